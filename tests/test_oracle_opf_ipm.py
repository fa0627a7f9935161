"""Pins for the oracle AC-OPF model and interior-point method (no GPU)."""
import dataclasses

import numpy as np
import pytest
import scipy.sparse as sp

from synth import config_grid, kkt_point, ring_grid
from oracle.opf import OPFModel
from oracle import ipm


def fd_jacobian(m, x, eps=1e-7):
    cols = []
    for k in range(m.n):
        e = np.zeros(m.n)
        e[k] = eps
        gp, hp = m.cons(x + e)
        gm, hm = m.cons(x - e)
        cols.append((np.concatenate([gp, hp]) - np.concatenate([gm, hm])) / (2 * eps))
    return np.array(cols).T


def test_derivatives_match_finite_differences():
    g = config_grid("ring30")
    m = OPFModel(g)
    p = kkt_point(g, 7)
    x, y, z = p["x"], p["y"], p["z"]
    J = m.jacobian(x).toarray()
    assert np.abs(J - fd_jacobian(m, x)).max() < 1e-6 * max(1, np.abs(J).max())
    sf = 0.3
    W = m.hessian(x, y, z, sf).toarray()
    eps = 1e-6
    Wfd = np.zeros_like(W)
    lag = lambda xx: sf * m.grad(xx) + m.jacobian(xx).T @ np.concatenate([y, z])
    for k in range(m.n):
        e = np.zeros(m.n)
        e[k] = eps
        Wfd[:, k] = (lag(x + e) - lag(x - e)) / (2 * eps)
    assert np.abs(W - Wfd).max() < 1e-5 * max(1, np.abs(W).max())
    assert np.abs(W - W.T).max() <= 1e-13 * np.abs(W).max()


def test_branch_physics():
    """Lossless lines transfer power exactly; resistive lines only lose power."""
    g = ring_grid(12, 3, 3, seed=5)
    g0 = dataclasses.replace(g, r=np.zeros(g.nbr), b=np.zeros(g.nbr))
    m0 = OPFModel(g0)
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(0.9, 1.1, g.nb), rng.uniform(-0.3, 0.3, g.nb),
                        np.zeros(2 * g.ng)])
    (_, _, Pf, Qf, *_), (_, _, Pt, Qt, *_) = m0._flows(x)
    np.testing.assert_allclose(Pf + Pt, 0.0, atol=1e-12)
    m1 = OPFModel(dataclasses.replace(g, b=np.zeros(g.nbr)))
    (_, _, Pf, _, *_), (_, _, Pt, _, *_) = m1._flows(x)
    assert np.all(Pf + Pt >= -1e-12)


class QP:
    """min 1/2 x^T Q x + c^T x  s.t.  A x = b,  xl <= x <= xu."""

    def __init__(self, Q, c, A, b, xl, xu):
        self.Q, self.c, self.A, self.b = sp.csr_matrix(Q), c, sp.csr_matrix(A), b
        self.n, self.m_e, self.m_i = len(c), A.shape[0], 0
        self.xl, self.xu = xl, xu

    def x0(self):
        return np.zeros(self.n)

    def objective(self, x):
        return float(0.5 * x @ (self.Q @ x) + self.c @ x)

    def grad(self, x):
        return self.Q @ x + self.c

    def cons(self, x):
        return self.A @ x - self.b, np.zeros(0)

    def jacobian(self, x):
        return self.A.copy()

    def hessian(self, x, y, z, sigma_f=1.0):
        return (sigma_f * self.Q).tocsr()


def test_equality_qp_closed_form():
    rng = np.random.default_rng(1)
    n, me = 12, 4
    M = rng.standard_normal((n, n))
    Q = M @ M.T + np.eye(n)
    c = rng.standard_normal(n)
    A = rng.standard_normal((me, n))
    b = rng.standard_normal(me)
    inf = np.full(n, np.inf)
    r = ipm.solve(QP(Q, c, A, b, -inf, inf), ipm.Options(kkt="hykkt", gamma=1e4))
    kkt = np.block([[Q, A.T], [A, np.zeros((me, me))]])
    ref = np.linalg.solve(kkt, np.concatenate([-c, b]))[:n]
    assert r.status == "converged"
    np.testing.assert_allclose(r.x, ref, rtol=1e-6, atol=1e-7)


def test_box_qp_is_clipped_minimizer():
    rng = np.random.default_rng(2)
    n = 20
    q = rng.uniform(0.5, 2.0, n)
    c = rng.standard_normal(n) * 3
    xl, xu = np.full(n, -1.0), np.full(n, 1.0)
    xl[::5] = -np.inf
    prob = QP(np.diag(q), c, np.zeros((0, n)), np.zeros(0), xl, xu)
    for kkt in ("hykkt", "lifted"):
        r = ipm.solve(prob, ipm.Options(kkt=kkt))
        assert r.status == "converged"
        np.testing.assert_allclose(r.x, np.clip(-c / q, xl, xu), atol=1e-5)


@pytest.mark.parametrize("kkt", ["hykkt", "lifted"])
def test_ring30_converges(kkt):
    g = config_grid("ring30")
    r = ipm.solve(OPFModel(g), ipm.Options(kkt=kkt, gamma=1e6))
    assert r.status == "converged"
    assert r.kkt_error <= 1e-6
    gx, hx = OPFModel(g).cons(r.x)
    assert np.abs(gx).max() <= (1e-5 if kkt == "lifted" else 1e-8)
    assert hx.max() <= 1e-6


def test_lifted_optimum_within_tau_of_hykkt():
    """Section 3.2: the relaxation error is of the order of the tolerance tau."""
    g = config_grid("ring30")
    rh = ipm.solve(OPFModel(g), ipm.Options(kkt="hykkt", gamma=1e6))
    rl = ipm.solve(OPFModel(g), ipm.Options(kkt="lifted"))
    tau = 1e-6
    assert abs(rl.obj - rh.obj) <= 1e3 * tau * max(1.0, abs(rh.obj))


def test_auto_gamma_is_the_norm_ratio_when_the_bound_is_exact():
    # H with one entry per row, W + Sigma diagonal and non-negative, D >= 0: the row-sum bound of
    # ||K||_inf is the exact infinity norm of K = W + Sigma + H^T D H
    import scipy.sparse as sp
    from oracle.ipm import auto_gamma
    rng = np.random.default_rng(7)
    n = 6
    W = sp.diags(rng.uniform(0.5, 2.0, n)).tocsr()
    sig = rng.uniform(0, 1, n)
    H = sp.csr_matrix((rng.normal(size=4), ([0, 1, 2, 3], [0, 2, 2, 5])), shape=(4, n))
    Ds = rng.uniform(0.1, 3.0, 4)
    G = sp.csr_matrix(rng.normal(size=(2, n)))
    Kd = W.toarray() + np.diag(sig) + H.toarray().T @ np.diag(Ds) @ H.toarray()
    expect = np.linalg.norm(Kd, np.inf) / np.linalg.norm(G.toarray(), np.inf) ** 2
    assert np.isclose(auto_gamma(W, sig, G, H, Ds), expect, rtol=1e-14)


def test_dual_regularized_form_converges_near_hykkt():
    from synth import config_grid
    g = config_grid("ring30")
    hy = ipm.solve(OPFModel(g), ipm.Options(kkt="hykkt", gamma=1e6))
    for gam in (1e6, 0.0):
        r = ipm.solve(OPFModel(g), ipm.Options(kkt="regularized", gamma=gam))
        assert r.status == "converged"
        # delta_c = 1/gamma perturbs the dual update only: same optimum to O(delta_c)
        assert abs(r.obj - hy.obj) <= 1e-6 * abs(hy.obj)


def test_flow_model_derivatives_by_finite_differences():
    from oracle.opf import FlowOPFModel
    g = config_grid("ring30")
    m = FlowOPFModel(g)
    rng = np.random.default_rng(3)
    x = m.x0() + rng.normal(0, 0.02, m.n)
    y, z = rng.normal(size=m.m_e), rng.normal(size=m.m_i)
    J = m.jacobian(x).toarray()
    h = 1e-6
    fd = np.zeros_like(J)
    for j in range(m.n):
        e = np.zeros(m.n)
        e[j] = h
        gp, hp = m.cons(x + e)
        gm, hm = m.cons(x - e)
        fd[:, j] = (np.concatenate([gp, hp]) - np.concatenate([gm, hm])) / (2 * h)
    assert np.allclose(J, fd, atol=1e-6)

    def lag_grad(xx):
        return 0.7 * m.grad(xx) + m.jacobian(xx).T @ np.concatenate([y, z])
    W = m.hessian(x, y, z, 0.7).toarray()
    fdw = np.zeros_like(W)
    for j in range(m.n):
        e = np.zeros(m.n)
        e[j] = h
        fdw[:, j] = (lag_grad(x + e) - lag_grad(x - e)) / (2 * h)
    assert np.allclose(W, fdw, atol=1e-5)
    assert np.allclose(W, W.T)


def test_flow_model_has_the_compact_optimum():
    # the flow variables only name the branch flows: the same feasible set after projection,
    # so HyKKT (exact equalities) reaches the same objective on both formulations
    from oracle.opf import FlowOPFModel
    g = config_grid("ring30")
    a = ipm.solve(OPFModel(g), ipm.Options(kkt="hykkt", gamma=1e6))
    b = ipm.solve(FlowOPFModel(g), ipm.Options(kkt="hykkt", gamma=1e6))
    assert a.status == b.status == "converged"
    assert abs(a.obj - b.obj) <= 1e-6 * abs(a.obj)
    m = FlowOPFModel(g)
    assert (m.n, m.m_e, m.m_i) == (2 * g.nb + 2 * g.ng + 4 * g.nbr, 2 * g.nb + 1 + 4 * g.nbr, 2 * g.nbr)
