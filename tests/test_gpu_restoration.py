"""Feasibility restoration phase of the single-problem GPU IPM (Waechter & Biegler 2006,
Sec. 3.3, the restoration phase of the filter method cited in Sec. 2.2) against the oracle's.

Bars.  From a start where the filter line search fails (random bus angles) both sides enter the
restoration phase and then converge to the optimum of the regular start (objectives within 1e-6
relative).  The trajectories after the first phase depend on rounding (the phase's own filter
line search is as sensitive to the last bits as the main one), so the counts of phases are not
compared; the main iteration at which the first phase starts is, within the usual tolerance.  On
an infeasible grid (loads above the generation capacity) both sides end with the phase
converging to a stationary point of the violation.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import config_grid
from oracle.opf import OPFModel
from oracle import ipm as oipm
import paper_2405_14236_gb300 as cp


def run(opf, x0=None, max_iter=3000, **opts):
    st = cp.IpmState(opf, x0=x0, **opts)
    hist = []
    main = 0
    while main <= max_iter:
        info = st.step().as_dict()
        hist.append(info)
        if info["status"] != 0:
            break
        main += info["resto"] != 1
    return st, hist


def bad_start(g, seed):
    m = OPFModel(g)
    x0 = m.x0().copy()
    x0[g.nb:2 * g.nb] = np.random.default_rng(seed).uniform(-3, 3, g.nb)
    return x0


@pytest.mark.parametrize("kkt", ["lifted", "hykkt"])
@pytest.mark.parametrize("seed", [0, 1])
def test_restoration_recovers_from_a_bad_start(kkt, seed):
    g = config_grid("ring30")
    m = OPFModel(g)
    x0 = bad_start(g, seed)
    ref = oipm.solve(m, oipm.Options(kkt=kkt))
    obad = oipm.solve(m, oipm.Options(kkt=kkt), x0=x0)
    assert ref.status == "converged" and obad.status == "converged"
    st, hist = run(cp.Opf(g), x0=x0, kkt=kkt, gamma=1e6)
    assert hist[-1]["status"] == 1, hist[-1]
    starts = [h["k"] for h in hist if h["resto"] == 2]
    assert len(starts) >= 1
    assert sum(h["resto"] == 1 for h in hist) >= 1
    first_ref = min(h["k"] for h in obad.history if "resto" in h)
    assert abs(starts[0] - first_ref) <= max(3, first_ref // 5), (starts[0], first_ref)
    assert abs(st.objective() - ref.obj) <= 1e-6 * abs(ref.obj)
    gx, hx = m.cons(st.x())
    assert np.abs(gx).max() <= (1e-5 if kkt == "lifted" else 1e-8)
    assert hx.max() <= 1e-6


@pytest.mark.parametrize("kkt", ["lifted", "hykkt"])
def test_infeasible_grid_is_reported(kkt):
    g = config_grid("ring30")
    g = dataclasses.replace(g, pd=3 * g.pd, qd=3 * g.qd)   # load above the generation capacity
    ref = oipm.solve(OPFModel(g), oipm.Options(kkt=kkt))
    assert ref.status == "infeasible"
    st, hist = run(cp.Opf(g), kkt=kkt, gamma=1e6)
    assert hist[-1]["status"] == cp.IPM_ERR_INFEASIBLE, hist[-1]
    assert any(h["resto"] == 2 for h in hist)


def test_regular_start_through_create_at_matches_the_flat_start():
    """ipm_state_create_at at the flat start's own point reproduces ipm_state_create."""
    g = config_grid("ring30")
    opf = cp.Opf(g)
    a = cp.ipm_solve_opf(opf, kkt="lifted")
    x0 = OPFModel(g).x0()
    st, hist = run(opf, x0=x0, kkt="lifted")
    assert hist[-1]["status"] == 1 and a["status"] == 1
    assert abs(hist[-1]["k"] - a["iters"]) <= 1
    assert abs(st.objective() - a["obj"]) <= 1e-9 * abs(a["obj"])
