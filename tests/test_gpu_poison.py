"""No kernel reads a floating-point entry before writing it: with ipm_debug_poison_allocations on,
every floating-point buffer the library allocates starts as NaN, and the solves must still
converge to the objective they reach from ordinary allocations (single-problem IPM in both
formulations and every KKT form, FP32 factor included; the batched IPM, both formulations in one
batch, in every form, before and after a reset).  A read of an unwritten entry would carry NaN into the iterates."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import config_grid, scale_loads, mixed_grid
import paper_2405_14236_gb300 as cp


@pytest.fixture
def poisoned():
    cp.ipm_debug_poison_allocations(True)
    yield
    cp.ipm_debug_poison_allocations(False)


def close_its(kkt, a, b):
    # LiftedKKT's iteration count moves with the rounding of atomic sums (a few iterations);
    # the other forms take the same path every run
    return abs(a - b) <= (max(3, b // 10) if kkt == "lifted" else 1)


SINGLE = [("ring30", "compact", "lifted", 64), ("ring30", "flow", "hykkt", 64),
          ("planar1k", "compact", "hykkt", 64), ("planar1k", "compact", "regularized", 64),
          ("planar1k", "compact", "lifted", 32), ("planar1k", "flow", "lifted", 64),
          ("planar1k", "flow", "hykkt", 64), ("planar1k", "flow", "regularized", 64)]


@pytest.mark.parametrize("name,form,kkt,prec", SINGLE)
def test_single_problem_ignores_initial_buffer_contents(name, form, kkt, prec, poisoned):
    g = config_grid(name)
    run = lambda: cp.ipm_solve_opf(cp.Opf(g, form=form), kkt=kkt, gamma=1e6, precision=prec)
    cp.ipm_debug_poison_allocations(False)
    ref = run()
    cp.ipm_debug_poison_allocations(True)
    res = run()
    assert ref["status"] == 1 and res["status"] == 1, (ref["history"][-1], res["history"][-1])
    assert np.isfinite(res["x"]).all()
    assert abs(res["obj"] - ref["obj"]) <= 1e-6 * abs(ref["obj"])
    assert close_its(kkt, res["iters"], ref["iters"]), (res["iters"], ref["iters"])


@pytest.mark.parametrize("kkt,prec", [("lifted", 64), ("hykkt", 64), ("regularized", 64),
                                      ("lifted", 32)])
def test_batch_ignores_initial_buffer_contents(kkt, prec, poisoned):
    base = config_grid("planar1k")
    grids = ([scale_loads(base, 1000 + k) for k in range(3)] +
             [mixed_grid(2000 + k) for k in (3, 9)] + [config_grid("ring30")])
    # the last two instances in the branch-flow formulation
    forms = ["compact"] * len(grids) + ["flow", "flow"]
    grids += [scale_loads(base, 1003), config_grid("ring30")]
    opfs = lambda: [cp.Opf(g, form=f) for g, f in zip(grids, forms)]
    cp.ipm_debug_poison_allocations(False)
    R = cp.Batch(opfs(), kkt=kkt, gamma=1e6, precision=prec)
    R.run(max_iter=200)
    ref = R.results()
    del R
    cp.ipm_debug_poison_allocations(True)
    B = cp.Batch(opfs(), kkt=kkt, gamma=1e6, precision=prec)
    for rnd in range(2):
        if rnd:
            B.reset()   # the second run starts from the first run's leftovers
        B.run(max_iter=200)
        res = B.results()
        assert (res["status"] == 1).all() and (ref["status"] == 1).all(), (res["status"],
                                                                          ref["status"])
        np.testing.assert_allclose(res["obj"], ref["obj"], rtol=1e-6)
        for a, b in zip(res["iters"], ref["iters"]):
            assert close_its(kkt, int(a), int(b)), (res["iters"], ref["iters"])
