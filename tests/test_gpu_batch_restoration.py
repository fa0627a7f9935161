"""Feasibility restoration in the batched IPM (Waechter & Biegler 2006, Sec. 3.3, the
restoration phase of the filter method cited in Sec. 2.2): instances in the phase are advanced by
the same sweeps as the others, on the device.

Bars.  An instance whose grid carries more load than its generators can supply ends with the
phase converging to a stationary point of the violation (IPM_ERR_INFEASIBLE), as in the oracle
and in the single-problem IPM, while the feasible instances of the same batch converge to the
oracle's objectives (1e-6 relative).  Grids whose line search fails from the flat start without
the phase converge with it, to the oracle's objective with the phase.
"""
import dataclasses
import json
import pathlib

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import config_grid, scale_loads, mixed_grid
from oracle.opf import OPFModel
from oracle import ipm as oipm
import paper_2405_14236_gb300 as cp


def overloaded(g, f=3.0):
    return dataclasses.replace(g, pd=f * g.pd, qd=f * g.qd, name=g.name + "-x3")


@pytest.mark.parametrize("kkt", ["lifted", "hykkt", "regularized"])
def test_batch_reports_infeasible_instance(kkt):
    base = config_grid("ring30")
    grids = [overloaded(base), base, scale_loads(base, 7)]
    opfs = [cp.Opf(g) for g in grids]
    B = cp.Batch(opfs, kkt=kkt, gamma=1e6)
    B.run()
    r = B.results()
    assert r["status"][0] == cp.IPM_ERR_INFEASIBLE, r["status"]
    assert r["resto_phases"][0] >= 1 and r["resto_iters"][0] >= 1
    okind = {"lifted": "lifted", "hykkt": "hykkt", "regularized": "regularized"}[kkt]
    assert oipm.solve(OPFModel(grids[0]), oipm.Options(kkt=okind)).status == "infeasible"
    for i in (1, 2):
        ref = oipm.solve(OPFModel(grids[i]), oipm.Options(kkt=okind, gamma=1e6))
        assert ref.status == "converged"
        assert r["status"][i] == 1, r["status"]
        assert abs(r["obj"][i] - ref.obj) <= 1e-6 * abs(ref.obj)


def test_batch_matches_single_problem_on_infeasible_instance():
    """The batch follows the single-problem iteration: the same main iteration at which the
    first restoration phase starts, and the same final status."""
    g = overloaded(config_grid("ring30"))
    B = cp.Batch([cp.Opf(g)], kkt="lifted")
    B.run()
    rb = B.results()
    st = cp.IpmState(cp.Opf(g), kkt="lifted")
    first = None
    while True:
        info = st.step()
        if info.resto == 2 and first is None:
            first = info.k
        if info.status != 0:
            break
    assert info.status == cp.IPM_ERR_INFEASIBLE == rb["status"][0]
    assert first is not None
    # the batch's iteration count at the end includes the main iterations only (each phase
    # counts as one, as in ipm_step)
    assert abs(int(rb["iters"][0]) - info.k) <= max(3, info.k // 5)


def test_restoration_off_stops_at_the_failed_line_search():
    g = overloaded(config_grid("ring30"))
    B = cp.Batch([cp.Opf(g)], kkt="lifted", restoration=False)
    B.run()
    r = B.results()
    assert r["status"][0] == cp.IPM_ERR_RESTORATION
    assert r["resto_phases"][0] == 0
