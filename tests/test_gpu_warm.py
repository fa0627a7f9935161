"""Learned warm start of the batched IPM: a network trained (on the GPU, by the library's own
kernels) on batched-IPM points of load scenarios of the 1,000-bus grid starts held-out
scenarios.  Bar: every warm-started instance converges to the 1e-6 tolerance at the objective
of its cold start (1e-6 relative) and the warm starts take fewer iterations on average than the
cold starts of the same instances."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import config_grid, scale_loads
import paper_2405_14236_gb300 as cp
from paper_2405_14236_gb300 import warm


@pytest.mark.parametrize("kkt", ["lifted"])
def test_warm_start_saves_iterations(kkt):
    base = config_grid("planar1k")
    train_grids = [scale_loads(base, 10000 + k) for k in range(640)]
    test_grids = [scale_loads(base, 30000 + k) for k in range(32)]
    T, ok = warm.collect(train_grids, tol=1e-3, kkt=kkt)
    assert ok.mean() > 0.95
    keep = np.nonzero(ok)[0]
    X = warm.input_rows([train_grids[i] for i in keep])
    Tk = T[torch.as_tensor(keep, device="cuda")].contiguous()
    model, losses = warm.train(X, Tk, steps=600, batch=128, lr=1e-3, log_every=100)
    assert losses[-1][1] < losses[0][1]
    opfs = [cp.Opf(g) for g in test_grids]
    B = cp.Batch(opfs, kkt=kkt, gamma=1e6)
    B.run(max_iter=300)
    cold = B.results()
    B.reset()
    used = model.start(B, warm.input_rows(test_grids))
    assert used.all()
    B.run(max_iter=300)
    hot = B.results()
    both = (cold["status"] == 1) & (hot["status"] == 1)
    assert both.mean() >= 0.9, (cold["status"], hot["status"])
    rel = np.abs(hot["obj"][both] - cold["obj"][both]) / np.abs(cold["obj"][both])
    assert rel.max() <= 1e-6
    assert hot["iters"][both].mean() < cold["iters"][both].mean(), (hot["iters"], cold["iters"])


def test_non_finite_prediction_keeps_the_cold_start():
    base = config_grid("planar1k")
    grids = [scale_loads(base, 30100 + k) for k in range(3)]
    B = cp.Batch([cp.Opf(g) for g in grids])
    B.run(max_iter=300)
    cold = B.results()
    rows = B.state_rows()  # the solutions themselves as "predictions" (unnormalized)
    rows[1, 5] = float("nan")
    B.reset()
    used = B.warm_start(rows)
    assert used.tolist() == [1, 0, 1]
    B.run(max_iter=300)
    hot = B.results()
    assert (hot["status"] == 1).all()
    # instance 1 repeats its cold solve (up to the reordered sums of the batched kernels, the
    # tolerance of the other batch tests); the others start at their own solution
    assert abs(hot["iters"][1] - cold["iters"][1]) <= max(3, cold["iters"][1] // 10)
    assert hot["iters"][0] < cold["iters"][0] and hot["iters"][2] < cold["iters"][2]
    assert np.allclose(hot["obj"], cold["obj"], rtol=1e-6)


@pytest.mark.parametrize("kkt", ["regularized", "hykkt"])
def test_state_rows_carry_the_equality_multipliers(kkt):
    """HyKKT and dual-regularized batches append y to the state rows; a batch started from the
    rows of its own iterates at tolerance 1e-3 (an exact prediction, y included) converges at the
    cold start's objective in fewer iterations, and the rows have the documented width."""
    base = config_grid("planar1k")
    grids = [scale_loads(base, 1000 + k) for k in range(6)]
    opfs = [cp.Opf(g) for g in grids]
    B = cp.Batch(opfs, kkt=kkt, gamma=1e6, tol=1e-3)
    B.run(max_iter=300)
    rows = B.state_rows()
    n, mi, me = opfs[0].n, opfs[0].m_i, opfs[0].m_e
    assert rows.shape[1] == 3 * n + 2 * mi + me
    assert torch.isfinite(rows).all() and float(rows[:, 3 * n + 2 * mi:].abs().max()) > 0
    C = cp.Batch(opfs, kkt=kkt, gamma=1e6)
    C.run(max_iter=300)
    cold = C.results()
    C.reset()
    used = C.warm_start(rows)
    assert np.asarray(used).all()
    C.run(max_iter=300)
    hot = C.results()
    assert (cold["status"] == 1).all() and (hot["status"] == 1).all(), (cold["status"], hot["status"])
    assert np.allclose(hot["obj"], cold["obj"], rtol=1e-6, atol=0)
    assert hot["iters"].mean() < cold["iters"].mean(), (hot["iters"], cold["iters"])
