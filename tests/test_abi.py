"""The C ABI library loads (no GPU needed) and exports every function include/*.h declares;
the Python binding declares each with the header's argument count."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_prototypes():
    protos = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        for m in re.finditer(r"\n\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ipm_\w+|hykkt_\w+|mlp_\w+)\s*\(([^;{]*?)\)\s*;",
                             text):
            name, args = m.group(1), m.group(2).strip()
            n = 0 if args in ("", "void") else args.count(",") + 1
            protos[name] = n
    return protos


@pytest.fixture(scope="module")
def built():
    from paper_2405_14236_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(built):
    protos = header_prototypes()
    assert len(protos) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = sorted(set(protos) - exported)
    assert not missing, missing


def test_library_loads_and_binding_matches_header(built):
    import paper_2405_14236_gb300 as cp
    L = cp.lib()  # dlopen works without a GPU
    protos = header_prototypes()
    for name, (res, args) in cp._SIGS.items():
        assert name in protos, name
        assert len(args) == protos[name], (name, len(args), protos[name])
        assert getattr(L, name) is not None
    assert set(protos) == set(cp._SIGS)
