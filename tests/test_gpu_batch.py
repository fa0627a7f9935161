"""Batched interior-point solves (ipm_batch_*) against the oracle IPM and the single-problem GPU
IPM on the same instances.

The batch mixes load scenarios of one grid (one shared symbolic analysis) with grids of other
sizes.  Bar: every instance converges to the 1e-6 scaled KKT tolerance at the oracle's objective
within 1e-6 relative, and follows the single-problem GPU iteration (iteration counts within 3,
the same objective to rounding): the batch runs the same algorithm per instance, and only the
order of floating-point additions (atomic scatters, block reductions) differs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import config_grid, scale_loads, mixed_grid
from oracle.opf import OPFModel
from oracle import ipm as oipm
import paper_2405_14236_gb300 as cp


def small_batch():
    base = config_grid("planar1k")
    return ([scale_loads(base, 1000 + k) for k in range(4)] +
            [mixed_grid(2000 + k) for k in (3, 9, 23)] + [config_grid("ring30")])


@pytest.fixture(scope="module")
def solved():
    grids = small_batch()
    opfs = [cp.Opf(g) for g in grids]
    B = cp.Batch(opfs)
    B.run(max_iter=200)
    return grids, opfs, B, B.results()


def test_batch_shares_symbolic_per_pattern(solved):
    grids, opfs, B, res = solved
    # 4 scenarios of one grid share a pattern; 3 mixed grids and the ring have their own
    assert B.info()["patterns"] == 5


def test_batch_matches_oracle(solved):
    grids, opfs, B, res = solved
    for i, g in enumerate(grids):
        ref = oipm.solve(OPFModel(g), oipm.Options(kkt="lifted"))
        assert ref.status == "converged"
        assert res["status"][i] == 1, (i, g.name, res["status"][i], res["iters"][i])
        assert abs(res["obj"][i] - ref.obj) <= 1e-6 * abs(ref.obj), (i, g.name)
        assert res["kkt_err"][i] <= 1e-6
        m = OPFModel(g)
        gx, hx = m.cons(B.x(i))
        assert np.abs(gx).max() <= 1e-5 and hx.max() <= 1e-6


def test_batch_follows_single_problem_iteration(solved):
    grids, opfs, B, res = solved
    for i, g in enumerate(grids):
        single = cp.ipm_solve_opf(cp.Opf(g), max_iter=200, kkt="lifted")
        assert single["status"] == 1
        assert abs(res["iters"][i] - single["iters"]) <= 3, (g.name, res["iters"][i], single["iters"])
        assert abs(res["obj"][i] - single["obj"]) <= 1e-9 * abs(single["obj"])


def test_batch_reset_and_eager_launches_agree(solved):
    grids, opfs, B, res = solved
    B.reset()
    B.run(max_iter=200, use_graph=False)
    again = B.results()
    assert np.array_equal(again["status"], res["status"])
    assert np.all(np.abs(again["iters"] - res["iters"]) <= 3)
    assert np.allclose(again["obj"], res["obj"], rtol=1e-9, atol=0)


def test_batch_iteration_limit_reported():
    g = config_grid("ring30")
    B = cp.Batch([cp.Opf(g), cp.Opf(scale_loads(g, 7))])
    B.run(max_iter=3)
    r = B.results()
    assert np.all(r["status"] == cp.IPM_ERR_MAXITER)
    assert np.all(r["iters"] == 3)
