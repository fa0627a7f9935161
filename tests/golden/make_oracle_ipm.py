"""Writes oracle_ipm.json: the oracle IPM's results on the large configurations.

Runs only the CPU oracle (oracle/ipm.py) on the seeded grids of synth/ and stores, per case,
the status, iteration count and final objective, with a digest of the grid's arrays so that a
test can tell when the stored values no longer belong to the generator's output.  The 80,000-bus
cases take minutes (HyKKT) to tens of minutes (LiftedKKT) on one core.

    python tests/golden/make_oracle_ipm.py [case ...]     (default: every case)
    python tests/golden/make_oracle_ipm.py --redigest     (digests only)
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "oracle_ipm.json")

# case -> (grid config name, KKT form, gamma)
CASES = {
    "planar10k-lifted": ("planar10k", "lifted", 1e6),
    "planar10k-hykkt": ("planar10k", "hykkt", 1e6),
    "planar80k-hykkt-g1e7": ("planar80k", "hykkt", 1e7),
    "planar80k-lifted": ("planar80k", "lifted", 1e6),
}


def grid_digest(g) -> dict:
    """Fingerprint of the grid's arrays: a hash of the integer arrays (topology, generator
    buses), and two weighted sums of each real array.  The real arrays come from linear algebra
    whose last bits differ between machines (the ratings solve a DC power flow), so the sums are
    compared with a relative tolerance (same_grid), not bit for bit."""
    h = hashlib.sha256()
    sums = {}
    for k, v in sorted(g.arrays().items()):
        if v.dtype.kind in "iu":
            h.update(k.encode())
            h.update(v.astype(np.int64).tobytes())
        else:
            w = 1.0 + (np.arange(len(v)) % 13)
            sums[k] = [float(v.sum()), float(v @ w)]
    return {"int_sha": h.hexdigest()[:16], "sums": sums}


def same_grid(a: dict, b: dict, rtol: float = 1e-9) -> bool:
    if a["int_sha"] != b["int_sha"] or set(a["sums"]) != set(b["sums"]):
        return False
    return all(abs(x - y) <= rtol * max(1.0, abs(y))
               for k in a["sums"] for x, y in zip(a["sums"][k], b["sums"][k]))


def main(names):
    from synth import config_grid
    from oracle.opf import OPFModel
    from oracle import ipm as oipm
    for name in names:
        grid, kkt, gamma = CASES[name]
        g = config_grid(grid)
        t0 = time.perf_counter()
        r = oipm.solve(OPFModel(g), oipm.Options(kkt=kkt, gamma=gamma))
        rec = dict(grid=grid, kkt=kkt, gamma=gamma, grid_digest=grid_digest(g), status=r.status,
                   iters=r.iters, obj=r.obj, kkt_error=r.kkt_error,
                   seconds=round(time.perf_counter() - t0, 1))
        print(name, rec, flush=True)
        # re-read before writing: several cases may run in separate processes
        out = json.load(open(OUT)) if os.path.exists(OUT) else {}
        out[name] = rec
        json.dump(out, open(OUT, "w"), indent=1, sort_keys=True)


def redigest():
    """Recomputes the grid digests of the stored records (after a change of the digest rule;
    the oracle results themselves are kept)."""
    from synth import config_grid
    out = json.load(open(OUT))
    for rec in out.values():
        rec["grid_digest"] = grid_digest(config_grid(rec["grid"]))
    json.dump(out, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    if sys.argv[1:] == ["--redigest"]:
        redigest()
    else:
        main(sys.argv[1:] or list(CASES))
