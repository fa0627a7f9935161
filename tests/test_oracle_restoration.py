"""Pins for the oracle's feasibility restoration (Waechter & Biegler 2006, Sec. 3.3, the
restoration phase of the filter method cited in Sec. 2.2) (no GPU)."""
import numpy as np
import pytest
import scipy.sparse as sp

from synth import config_grid
from oracle.opf import OPFModel
from oracle import ipm


def test_resto_pq_hand_values_and_stationarity():
    # mu = rho = 1, c = 1: p - q = 1 and 1/p + 1/q = 2 -> q = 1/sqrt(2), p = 1 + 1/sqrt(2)
    p, q = ipm.resto_pq(np.array([1.0]), 1.0, rho=1.0)
    assert p[0] == pytest.approx(1 + 2 ** -0.5, rel=1e-15)
    assert q[0] == pytest.approx(2 ** -0.5, rel=1e-15)
    # c = 0: p = q = mu / rho
    p, q = ipm.resto_pq(np.array([0.0]), 0.1, rho=1000.0)
    assert p[0] == pytest.approx(1e-4) and q[0] == pytest.approx(1e-4)
    # over many decades of c (both signs), the minimizer of rho (p + q) - mu log(p q) on p - q = c:
    # p - q = c and 2 rho = mu / p + mu / q, without cancellation where |c| >> mu / rho
    c = np.concatenate([-np.logspace(-10, 4, 29), [0.0], np.logspace(-10, 4, 29)])
    mu, rho = 0.1, 1000.0
    p, q = ipm.resto_pq(c, mu, rho)
    assert (p > 0).all() and (q > 0).all()
    np.testing.assert_allclose(p - q, c, rtol=1e-14, atol=1e-14 * mu / rho)
    np.testing.assert_allclose(mu / p + mu / q, 2 * rho, rtol=1e-12)


def test_restoration_model_derivatives():
    g = config_grid("ring30")
    base = ipm.ScaledModel(OPFModel(g), OPFModel(g).x0())
    rng = np.random.default_rng(3)
    xr = base.x0() + rng.normal(0, 0.05, base.n)
    R = ipm.RestorationModel(base, xr, zeta=0.3)
    m = R.mr
    w = np.concatenate([xr + rng.normal(0, 0.02, base.n), rng.uniform(0.1, 1, m), rng.uniform(0.1, 1, m)])
    eps = 1e-7
    # gradient of the objective
    gfd = np.array([(R.objective(w + eps * e) - R.objective(w - eps * e)) / (2 * eps)
                    for e in np.eye(R.n)])
    # (the objective is ~1e5 here: central differences carry ~1e-4 of rounding)
    np.testing.assert_allclose(R.grad(w), gfd, rtol=1e-6, atol=5e-4)
    # Jacobian of the rows c(x) - p + q
    J = R.jacobian(w).toarray()
    def c_of(ww):
        ge, hi = R.cons(ww)
        return np.concatenate([ge, hi])
    Jfd = np.array([(c_of(w + eps * e) - c_of(w - eps * e)) / (2 * eps) for e in np.eye(R.n)]).T
    np.testing.assert_allclose(J, Jfd, rtol=1e-5, atol=1e-6)
    # Hessian of the Lagrangian sigma * objective + lambda^T c
    y, z = rng.normal(size=R.m_e), rng.normal(size=R.m_i)
    lam = np.concatenate([y, z])
    lag = lambda ww: 0.7 * R.grad(ww) + R.jacobian(ww).T @ lam
    Hfd = np.array([(lag(w + eps * e) - lag(w - eps * e)) / (2 * eps) for e in np.eye(R.n)]).T
    np.testing.assert_allclose(R.hessian(w, y, z, 0.7).toarray(), Hfd, rtol=1e-5, atol=1e-5)


class LinearEquality:
    """min x1^2 + x2^2  s.t.  a . x = b  (one equality, no bounds)."""

    def __init__(self, a, b):
        self.a, self.b = np.asarray(a, float), float(b)
        self.n, self.m_e, self.m_i = 2, 1, 0
        self.xl = np.full(2, -np.inf)
        self.xu = np.full(2, np.inf)

    def x0(self):
        return np.zeros(2)

    def objective(self, x):
        return float(x @ x)

    def grad(self, x):
        return 2 * x

    def cons(self, x):
        return np.array([self.a @ x - self.b]), np.zeros(0)

    def jacobian(self, x):
        return sp.csr_matrix(self.a.reshape(1, 2))

    def hessian(self, x, y, z, sigma_f=1.0):
        return sp.csr_matrix(2.0 * sigma_f * np.eye(2))


def test_restoration_step_follows_the_weighted_normal():
    """For a linear constraint the restoration problem's x-stationarity is
    zeta D_R^2 (x - xr) + a lambda = 0, so every step of its IPM from xr moves x along
    D_R^{-2} a (D_R = min(1, 1/|xr|)): the point it returns lies on that line from xr and has
    at most 0.9 times the violation."""
    M = LinearEquality([1.0, 2.0], 1.0)
    xr = np.array([3.0, 0.5])   # D_R = (1/3, 1); a.xr - b = 3 > 0: direction -(9 a1, a2) = -(9, 2)
    theta_at = lambda x, s: float(abs(M.a @ x - M.b))
    phi_at = lambda x, s: M.objective(x)
    theta = theta_at(xr, None)
    rec = ipm._restoration(M, ipm.Options(kkt="hykkt"), xr, np.zeros(0), np.zeros(0),
                           np.zeros(2), np.zeros(2), 0.1, theta, 1e4, [], theta_at, phi_at)
    assert rec["status"] == "ok"
    d = rec["x"] - xr
    direction = -np.array([9.0, 2.0])
    cosang = d @ direction / (np.linalg.norm(d) * np.linalg.norm(direction))
    assert cosang == pytest.approx(1.0, abs=1e-10)
    assert theta_at(rec["x"], None) <= 0.9 * theta


@pytest.mark.parametrize("kkt", ["lifted", "hykkt"])
def test_restoration_recovers_from_a_bad_start(kkt):
    """30-bus grid started with random bus angles: the filter line search fails early; with the
    restoration phase the IPM reaches the same optimum as from the regular start, without it it
    stops."""
    g = config_grid("ring30")
    m = OPFModel(g)
    x0 = m.x0().copy()
    x0[g.nb:2 * g.nb] = np.random.default_rng(0).uniform(-3, 3, g.nb)
    ref = ipm.solve(m, ipm.Options(kkt=kkt))
    bad = ipm.solve(m, ipm.Options(kkt=kkt, restoration=False), x0=x0)
    assert bad.status == "restoration_needed"
    res = ipm.solve(m, ipm.Options(kkt=kkt), x0=x0)
    assert res.status == "converged"
    assert sum(1 for h in res.history if h.get("resto_status") == "ok") >= 1
    assert abs(res.obj - ref.obj) <= 1e-6 * abs(ref.obj)


def _late_iterate(g, kkt, k):
    """The oracle IPM's iterate after k iterations from the regular start (the model as solve
    builds it)."""
    base = OPFModel(g)
    opt = ipm.Options(kkt=kkt)
    model = ipm.ScaledModel(base, ipm._push(base.x0(), base.xl, base.xu))
    if kkt == "lifted":
        model = ipm.RelaxedModel(model, opt.tol)
    hl, hu = np.isfinite(model.xl), np.isfinite(model.xu)
    x = ipm._push(model.x0(), model.xl, model.xu)
    sig_f = min(1.0, 100.0 / max(np.abs(model.grad(x)).max(), 1e-300))
    gx, hx = model.cons(x)
    start = dict(x=x, s=np.maximum(-hx, ipm.KAPPA1), y=np.zeros(model.m_e), z=np.ones(model.m_i),
                 v=np.ones(model.m_i), zl=np.where(hl, 1.0, 0.0), zu=np.where(hu, 1.0, 0.0))
    r = ipm._ipm(model, opt, start, opt.mu0, sig_f, max_iter=k)
    return model, opt, r


def test_restoration_at_a_feasible_point_is_not_infeasibility():
    """Called at a late iterate of a feasible problem (violation at rounding level), the
    restoration problem is solved by the point itself; that is no evidence of infeasibility (a
    local minimizer of the violation with a positive violation), so the phase reports failure."""
    g = config_grid("ring30")
    model, opt, r = _late_iterate(g, "lifted", 30)
    gx, hx = model.cons(r.x)
    assert max(np.abs(gx).max(initial=0), np.abs(hx + r.s).max()) <= opt.tol
    theta_at = lambda xx, sx: float(np.abs(model.cons(xx)[0]).sum()
                                    + np.abs(model.cons(xx)[1] + sx).sum())
    phi_at = lambda xx, sx: float(model.objective(xx))
    rec = ipm._restoration(model, opt, r.x, r.s, r.v, r.zl, r.zu, r.mu, theta_at(r.x, r.s), 1e4,
                           [], theta_at, phi_at)
    assert rec["status"] == "restoration_failed"


@pytest.mark.parametrize("kkt", ["lifted", "hykkt"])
def test_overloaded_grid_is_locally_infeasible(kkt):
    """Total load three times the nominal one exceeds the generators' capacity (twice the nominal
    load): no point satisfies the power balances, and the restoration phase ends at a minimizer
    of the violation whose violation stays well above the tolerance."""
    import dataclasses
    g = config_grid("ring30")
    assert 3 * g.pd.sum() > g.pmax.sum()
    g3 = dataclasses.replace(g, pd=3 * g.pd, qd=3 * g.qd)
    res = ipm.solve(OPFModel(g3), ipm.Options(kkt=kkt))
    assert res.status == "infeasible"


def test_failed_line_search_at_a_feasible_point_recomputes_a_regularized_direction(monkeypatch):
    """A line search that fails at a point feasible within the tolerance cannot be helped by
    the restoration phase; the iteration's direction is computed again with the next delta_w of
    its inertia-correction schedule.  Pinned by planting an ascent direction (the negated
    Newton step of the unregularized system) at a late, feasible iterate of the 30-bus solve:
    the line search rejects every trial, the retry at delta_w = 1e-4 (the schedule's first
    candidate when no earlier iteration needed one) is accepted, and the solve reaches the same
    optimum.  Without the retry the same run stops there."""
    g = config_grid("ring30")
    ref = ipm.solve(OPFModel(g), ipm.Options(kkt="lifted"))
    assert ref.status == "converged"
    assert all(h["delta_w"] == 0 for h in ref.history[:31])
    k_star = 30
    orig = ipm.K.lifted_solve
    calls = {"n": 0}

    def planted(F, A, J, d, a, b, **kw):
        dx, dz, hist = orig(F, A, J, d, a, b, **kw)
        calls["n"] += 1
        if calls["n"] == k_star + 1:      # the first direction of iteration k_star
            return -dx, -dz, hist
        return dx, dz, hist

    monkeypatch.setattr(ipm.K, "lifted_solve", planted)
    res = ipm.solve(OPFModel(g), ipm.Options(kkt="lifted"))
    assert res.status == "converged"
    assert abs(res.obj - ref.obj) <= 1e-8 * abs(ref.obj)
    h = [e for e in res.history if e["k"] == k_star][0]
    assert h["delta_w"] == 1e-4 and h["nfac"] >= 2, h
    assert all(e["k"] != k_star or "resto" not in e for e in res.history)
    calls["n"] = 0
    monkeypatch.setattr(ipm, "MAX_LS_REGULARIZE", 0)
    res0 = ipm.solve(OPFModel(g), ipm.Options(kkt="lifted"))
    assert res0.status == "restoration_failed" and res0.iters == k_star
