"""Oracle primal-dual filter line-search interior-point method (FP64, TEST ONLY).

Follows Section 2 of the paper: problem (2) with slacks h(x) + s = 0, s >= 0,
the barrier system F_mu = 0 (Eq. (5)), Newton steps from the augmented system
(K_2) solved in condensed form (K_1) by LiftedKKT (Section 3.2) or HyKKT
(Section 3.1), and a step that keeps (x, s, v) strictly interior.  The paper
leaves the line search, barrier update and inertia correction to Ipopt
(Waechter & Biegler 2006, cited in Section 2.2); their published constants are
used and written out below.  Variable bounds xl <= x <= xu are handled as in
Ipopt by bound multipliers (zl, zu) that are eliminated into
Sigma_x = Zl (X - Xl)^{-1} + Zu (Xu - X)^{-1} on the diagonal of K.

A model provides: n, m_e, m_i, xl, xu, x0(), objective, grad, cons -> (g, h),
jacobian -> CSR [G; H] with a fixed pattern, hessian(x, y, z, sigma_f) -> full
symmetric CSR with a fixed pattern.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

from . import kkt as K

# Ipopt constants (Waechter & Biegler 2006)
KAPPA1 = KAPPA2 = 1e-2      # initial push into the bounds
KAPPA_EPS = 10.0            # barrier stop test E_mu <= kappa_eps mu
KAPPA_MU, THETA_MU = 0.2, 1.5
TAU_MIN = 0.99
S_MAX = 100.0
GAMMA_THETA, GAMMA_PHI = 1e-5, 1e-8
S_THETA, S_PHI, DELTA = 1.1, 2.3, 1.0
ETA_PHI = 1e-8
GAMMA_ALPHA = 0.05
KAPPA_SIGMA = 1e10
# rounding margin of barrier-function comparisons: phi is known only to about
# 10 eps_mach |phi|, so a trial whose phi differs by less than that counts as equal
PHI_MARGIN = 10.0 * np.finfo(np.float64).eps
SOFT_RESTO_REDUCTION = 1e-4   # required relative decrease of E_mu in a soft-restoration step
MAX_LS_REGULARIZE = 8         # recomputed directions (larger delta_w) after a line search that
                              # fails at a point feasible within the tolerance


def filter_accept(theta, phi, gphi, alpha, tht, pht, filt, theta_min, theta_max):
    """Acceptance of a trial point in the filter line search (Waechter & Biegler 2006,
    Sec. 2.3-2.4, cited in Sec. 2.2 of the paper).

    theta, phi: constraint violation and barrier function at the current iterate; gphi: the
    directional derivative of phi along the step; (tht, pht): the trial point at step alpha;
    filt: list of filter entries (theta_f, phi_f).  Returns (accepted, f_type): f_type is True
    when the trial was accepted by the Armijo condition in the switching case (such steps do
    not augment the filter).  Every comparison of barrier-function values allows the rounding
    margin PHI_MARGIN * |phi| (a reading: the paper is silent; Ipopt relaxes its Armijo and
    sufficient-decrease tests in the same way, applied here to the filter entries as well).
    """
    margin = PHI_MARGIN * abs(phi)
    if not (tht < theta_max and np.isfinite(pht)):
        return False, False
    for tf, pf in filt:
        if not (tht < tf or pht - pf < margin):
            return False, False
    switching = bool(gphi < 0 and alpha * (-gphi) ** S_PHI > DELTA * theta ** S_THETA)
    if switching and theta <= theta_min:
        return bool(pht - phi <= ETA_PHI * alpha * gphi + margin), True
    return bool(tht <= (1 - GAMMA_THETA) * theta or pht - phi <= -GAMMA_PHI * theta + margin), False


def barrier_update(mu, tol):
    """Monotone barrier decrease mu+ = max(tol / 10, min(kappa_mu mu, mu^theta_mu))
    (Waechter & Biegler 2006, Eq. (7))."""
    return max(tol / 10.0, min(KAPPA_MU * mu, mu ** THETA_MU))


@dataclasses.dataclass
class Options:
    kkt: str = "lifted"          # "lifted" | "hykkt" | "regularized"
    tol: float = 1e-6
    gamma: float = 1e6           # HyKKT gamma; "regularized": delta_c = 1 / gamma; <= 0: automatic
    tau: float | None = None     # LiftedKKT relaxation; None -> tol
    max_iter: int = 3000
    mu0: float = 0.1
    cg_rtol: float = 1e-10
    max_refine: int = 10
    soft_restoration: bool = False  # Ipopt's E_mu-decrease fallback before the restoration phase
    restoration: bool = True        # feasibility restoration phase when that fails too
    verbose: bool = False


class RelaxedModel:
    """LiftedKKT problem (12): -tau <= g(x) <= tau written as two inequality
    rows g - tau <= 0 and -g - tau <= 0 in front of h <= 0."""

    def __init__(self, base, tau):
        self.base, self.tau = base, tau
        self.n, self.m_e, self.m_i = base.n, 0, 2 * base.m_e + base.m_i
        self.xl, self.xu = base.xl, base.xu

    def x0(self):
        return self.base.x0()

    def objective(self, x):
        return self.base.objective(x)

    def grad(self, x):
        return self.base.grad(x)

    def cons(self, x):
        g, h = self.base.cons(x)
        return np.zeros(0), np.concatenate([g - self.tau, -g - self.tau, h])

    def jacobian(self, x):
        J = self.base.jacobian(x)
        me = self.base.m_e
        G, H = J[:me], J[me:]
        return sp.vstack([G, -G, H]).tocsr()

    def hessian(self, x, y, z, sigma_f=1.0):
        me = self.base.m_e
        return self.base.hessian(x, z[:me] - z[me:2 * me], z[2 * me:], sigma_f)


class ScaledModel:
    """Ipopt's gradient-based scaling of the constraint rows: row i is multiplied
    by min(1, 100 / ||grad c_i(x0)||_inf), computed once at the starting point."""

    def __init__(self, base, x0):
        self.base = base
        self.n, self.m_e, self.m_i = base.n, base.m_e, base.m_i
        self.xl, self.xu = base.xl, base.xu
        J = sp.csr_matrix(abs(base.jacobian(x0)))
        rmax = np.zeros(J.shape[0])
        nz = np.diff(J.indptr) > 0
        rmax[nz] = np.maximum.reduceat(J.data, J.indptr[:-1][nz])
        self.d = np.minimum(1.0, 100.0 / np.maximum(rmax, 1e-300))
        self.de, self.di = self.d[:base.m_e], self.d[base.m_e:]

    def x0(self):
        return self.base.x0()

    def objective(self, x):
        return self.base.objective(x)

    def grad(self, x):
        return self.base.grad(x)

    def cons(self, x):
        g, h = self.base.cons(x)
        return g * self.de, h * self.di

    def jacobian(self, x):
        # row scaling on the stored values: the structure (explicit zeros included) must stay the
        # pattern the symbolic analysis was made for
        J = self.base.jacobian(x).tocsr(copy=True)
        J.data *= np.repeat(self.d, np.diff(J.indptr))
        return J

    def hessian(self, x, y, z, sigma_f=1.0):
        return self.base.hessian(x, y * self.de, z * self.di, sigma_f)


RHO_RESTO = 1000.0        # penalty of the restoration objective (Waechter & Biegler 2006, Sec. 3.3)
KAPPA_RESTO = 0.9         # required reduction of theta before leaving the restoration phase


class RestorationModel:
    """The feasibility restoration problem of Waechter & Biegler 2006, Sec. 3.3 (the restoration
    phase of the filter method cited in Sec. 2.2) for a model at the reference point xr:

        min  rho sum(p + q) + zeta/2 ||D_R (x - xr)||_2^2
        s.t. g(x) - p_g + q_g = 0,  h(x) - p_h + q_h <= 0,  xl <= x <= xu,  p, q >= 0,

    with D_R = diag(min(1, 1/|xr_j|)); one pair (p, q) per constraint row.  Variables are
    [x, p, q] (n + 2 m); the inequality rows keep their slacks in the IPM."""

    def __init__(self, base, xr, zeta, rho=RHO_RESTO):
        self.base, self.xr, self.zeta, self.rho = base, xr.copy(), zeta, rho
        self.nx = base.n
        self.mr = base.m_e + base.m_i
        self.n, self.m_e, self.m_i = base.n + 2 * self.mr, base.m_e, base.m_i
        self.xl = np.concatenate([base.xl, np.zeros(2 * self.mr)])
        self.xu = np.concatenate([base.xu, np.full(2 * self.mr, np.inf)])
        self.dr2 = np.minimum(1.0, 1.0 / np.maximum(np.abs(xr), 1e-300)) ** 2

    def split(self, w):
        n, m = self.nx, self.mr
        return w[:n], w[n:n + m], w[n + m:]

    def x0(self):
        return np.concatenate([self.xr, np.ones(2 * self.mr)])

    def objective(self, w):
        x, p, q = self.split(w)
        return float(self.rho * (p.sum() + q.sum()) + 0.5 * self.zeta * (self.dr2 * (x - self.xr) ** 2).sum())

    def grad(self, w):
        x, p, q = self.split(w)
        return np.concatenate([self.zeta * self.dr2 * (x - self.xr), np.full(2 * self.mr, self.rho)])

    def cons(self, w):
        x, p, q = self.split(w)
        g, h = self.base.cons(x)
        c = np.concatenate([g, h]) - p + q
        return c[:self.m_e], c[self.m_e:]

    def jacobian(self, w):
        x, p, q = self.split(w)
        I = sp.identity(self.mr, format="csr")
        return sp.hstack([self.base.jacobian(x), -I, I]).tocsr()

    def hessian(self, w, y, z, sigma_f=1.0):
        x, p, q = self.split(w)
        Wx = self.base.hessian(x, y, z, 0.0) + sp.diags(sigma_f * self.zeta * self.dr2)
        return sp.block_diag([Wx, sp.csr_matrix((2 * self.mr, 2 * self.mr))]).tocsr()


def resto_pq(c, mu, rho=RHO_RESTO):
    """Starting p, q of the restoration problem for the row residuals c: for each row the
    minimizer of rho (p + q) - mu (log p + log q) subject to p - q = c, i.e. the positive root q
    of 2 rho q^2 + 2 (rho c - mu) q - mu c = 0 (Waechter & Biegler 2006, Eq. (33)) and p = c + q,
    the positive root of 2 rho p^2 - 2 (rho c + mu) p + mu c = 0.  Each root is evaluated in the
    form that does not cancel (through the product of the roots when the linear coefficient
    has the other sign); both discriminants equal mu^2 + rho^2 c^2."""
    c = np.asarray(c, dtype=np.float64)
    sd = np.sqrt(mu * mu + (rho * c) ** 2)
    bq, bp = mu - rho * c, mu + rho * c
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.where(bq >= 0, (bq + sd) / (2.0 * rho), -mu * c / (bq - sd))
        p = np.where(bp >= 0, (bp + sd) / (2.0 * rho), mu * c / (bp - sd))
    return p, q


@dataclasses.dataclass
class Result:
    status: str
    iters: int
    x: np.ndarray
    s: np.ndarray
    y: np.ndarray
    z: np.ndarray
    v: np.ndarray
    zl: np.ndarray
    zu: np.ndarray
    obj: float
    kkt_error: float
    mu: float
    history: list


def _push(x, xl, xu):
    """Initial point moved strictly inside the bounds (Ipopt bound push)."""
    hl, hu = np.isfinite(xl), np.isfinite(xu)
    x = x.copy()
    both = hl & hu
    pl = np.where(hl, KAPPA1 * np.maximum(1.0, np.abs(np.where(hl, xl, 0.0))), 0.0)
    pu = np.where(hu, KAPPA1 * np.maximum(1.0, np.abs(np.where(hu, xu, 0.0))), 0.0)
    width = np.where(both, xu - xl, np.inf)
    pl = np.where(both, np.minimum(pl, KAPPA2 * width), pl)
    pu = np.where(both, np.minimum(pu, KAPPA2 * width), pu)
    x = np.where(hl, np.maximum(x, np.where(hl, xl, 0.0) + pl), x)
    x = np.where(hu, np.minimum(x, np.where(hu, xu, 0.0) - pu), x)
    return x


def auto_gamma(W, sigma_x, G, H, Ds):
    """gamma = ||K|| / ||G||^2 (Golub & Greif, recommended in Sec. 3.1), infinity norms, with
    ||K|| bounded by the row sums of |W + Sigma_x| + |H|^T |D_s| |H| (delta_w = 0)."""
    import scipy.sparse as sps
    ones = np.ones(W.shape[0])
    full = abs(W + sps.diags(sigma_x)) @ ones
    rows = np.asarray(abs(H) @ np.ones(H.shape[1])).ravel()
    kn = float(np.max(full + abs(H).T @ (np.abs(Ds) * rows)))
    gn = float(np.max(np.asarray(abs(G) @ np.ones(G.shape[1])).ravel())) if G.shape[0] else 0.0
    return kn / (gn * gn) if gn > 0 else 1.0


def schedule_from(kmat, solver, delta, grow):
    """The inertia-correction schedule continued from the candidate delta: delta, delta grow,
    ... until the factorization of kmat(delta_w) succeeds (RuntimeError at 1e40).  Returns
    (delta_w, factor, factorizations)."""
    nf = 0
    while delta < 1e40:
        nf += 1
        F = solver.factor(kmat(delta))
        if F.ok:
            return delta, F, nf
        delta *= grow
    raise RuntimeError("inertia correction failed")


def solve(model, opt: Options | None = None, x0=None):
    """The IPM on a model: Ipopt's gradient scaling at the start, LiftedKKT's relaxation
    (Sec. 3.2) for kkt = "lifted", the flat starting point (|V| = 1, theta = 0, equal dispatch), then
    the filter line-search iterations (_ipm)."""
    opt = opt or Options()
    base = model
    model = ScaledModel(base, _push(base.x0() if x0 is None else x0, base.xl, base.xu))
    if opt.kkt == "lifted":
        model = RelaxedModel(model, opt.tau if opt.tau is not None else opt.tol)
    hl, hu = np.isfinite(model.xl), np.isfinite(model.xu)
    x = _push(model.x0() if x0 is None else x0, model.xl, model.xu)
    sig_f = min(1.0, 100.0 / max(np.abs(model.grad(x)).max(), 1e-300))
    g, h = model.cons(x)
    start = dict(x=x, s=np.maximum(-h, KAPPA1), y=np.zeros(model.m_e), z=np.ones(model.m_i),
                 v=np.ones(model.m_i), zl=np.where(hl, 1.0, 0.0), zu=np.where(hu, 1.0, 0.0))
    res = _ipm(model, opt, start, opt.mu0, sig_f)
    res.obj = base.objective(res.x)
    return res


def _ipm(model, opt, start, mu, sig_f, exit_check=None, restore=True, max_iter=None):
    """Filter line-search interior-point iterations on `model` (scaling and relaxation already
    applied) from the primal-dual point `start` with barrier parameter mu.  exit_check(x, s),
    when given, is asked after every accepted step and ends the iterations with status
    "exited" (the restoration phase's return test).  restore: call the restoration phase when
    the line search and the soft restoration fail."""
    max_iter = opt.max_iter if max_iter is None else max_iter
    n, me, mi = model.n, model.m_e, model.m_i
    xl, xu = model.xl, model.xu
    hl, hu = np.isfinite(xl), np.isfinite(xu)
    xlf, xuf = np.where(hl, xl, 0.0), np.where(hu, xu, 0.0)
    x, s, y, z, v, zl, zu = (np.array(start[k], dtype=np.float64)
                             for k in ("x", "s", "y", "z", "v", "zl", "zu"))
    tau = max(TAU_MIN, 1.0 - mu)
    nl, nu = int(hl.sum()), int(hu.sum())

    J = model.jacobian(x)
    W = model.hessian(x, y, z, sig_f)
    solver = K.CondensedSolver(W, J)
    filt = []
    delta_last = 0.0
    hist = []
    theta0 = None
    n_resto = 0

    def theta_of(gx, hx, sx):
        return float(np.abs(gx).sum() + np.abs(hx + sx).sum())

    def theta_at(xx, sx):
        gx, hx = model.cons(xx)
        return theta_of(gx, hx, sx)

    def phi_of(xx, sx, mu_):
        val = sig_f * model.objective(xx) - mu_ * np.log(sx).sum()
        val -= mu_ * np.log((xx - xlf)[hl]).sum() + mu_ * np.log((xuf - xx)[hu]).sum()
        return float(val)

    def errors(gradf, J, g, h, mu_):
        return errors_at(x, s, y, z, v, zl, zu, gradf, J, g, h, mu_)

    def errors_at(x, s, y, z, v, zl, zu, gradf, J, g, h, mu_):
        G, H = J[:me], J[me:]
        gl = gradf * sig_f + G.T @ y + H.T @ z - zl + zu
        sd = max(S_MAX, (np.abs(y).sum() + np.abs(z).sum() + np.abs(v).sum() + np.abs(zl).sum()
                         + np.abs(zu).sum()) / max(me + 2 * mi + nl + nu, 1)) / S_MAX
        sc = max(S_MAX, (np.abs(v).sum() + np.abs(zl).sum() + np.abs(zu).sum())
                 / max(mi + nl + nu, 1)) / S_MAX
        dual = max(np.abs(gl).max(initial=0.0), np.abs(z - v).max(initial=0.0)) / sd
        prim = max(np.abs(g).max(initial=0.0), np.abs(h + s).max(initial=0.0))
        comp = max(np.abs(s * v - mu_).max(initial=0.0),
                   np.abs(((x - xlf) * zl - mu_)[hl]).max(initial=0.0),
                   np.abs(((xuf - x) * zu - mu_)[hu]).max(initial=0.0)) / sc
        return max(dual, prim, comp)

    status = "max_iter"
    it = 0
    for it in range(max_iter + 1):
        g, h = model.cons(x)
        gradf = model.grad(x)
        J = model.jacobian(x)
        e0 = errors(gradf, J, g, h, 0.0)
        if theta0 is None:
            theta0 = theta_of(g, h, s)
            theta_max = 1e4 * max(1.0, theta0)
            theta_min = 1e-4 * max(1.0, theta0)
        if e0 <= opt.tol:
            status = "converged"
            break
        if it == max_iter:
            break
        first = True
        while errors(gradf, J, g, h, mu) <= KAPPA_EPS * mu and (first or it == 0):
            mu = barrier_update(mu, opt.tol)
            tau = max(TAU_MIN, 1.0 - mu)
            filt = []
            first = False
        W = model.hessian(x, y, z, sig_f)
        G, H = J[:me], J[me:]
        dxl = np.where(hl, x - xlf, 1.0)
        dxu = np.where(hu, xuf - x, 1.0)
        sigma_x = np.where(hl, zl / dxl, 0.0) + np.where(hu, zu / dxu, 0.0)
        Ds = v / s
        r1 = sig_f * gradf + G.T @ y + H.T @ z - np.where(hl, mu / dxl, 0.0) + np.where(hu, mu / dxu, 0.0)
        r2 = z - mu / s
        r3 = g
        r4 = h + s

        gamma = opt.gamma if opt.gamma > 0 else auto_gamma(W, sigma_x, G, H, Ds)

        def kmat(dw):
            dh = Ds + dw
            d = np.concatenate([np.full(me, gamma), dh]) if opt.kkt != "lifted" else dh
            return K.condensed_matrix(W, sigma_x, J, d, dw)

        # delta_w of this iteration from the inertia-correction schedule (Sec. 2.2); after a line
        # search that fails at a point feasible within the tolerance the schedule goes on from its
        # next candidate (sched = (delta, growth)) and the direction is recomputed
        delta_last0 = delta_last
        grow0 = 8.0 if delta_last0 > 0 else 100.0
        sched = None
        n_reg = 0
        outcome = None
        while True:
            try:
                if sched is None:
                    dw, F, nfac = K.inertia_schedule(kmat, solver, delta_last)
                else:
                    dw, F, nf2 = schedule_from(kmat, solver, *sched)
                    nfac += nf2
            except RuntimeError:      # no delta_w up to 1e40 gives a positive definite matrix
                outcome = "inertia_failed"
                break
            if dw > 0:
                delta_last = dw
            dh = Ds + dw
            a = -r1

            def direction(r3_, r4_):
                """Newton direction for the constraint residuals (r3_, r4_) with the factor of this
                iteration."""
                bH = -r4_ + r2 / dh
                cg_its_ = 0
                if opt.kkt == "hykkt":
                    b = np.concatenate([-r3_, bH])
                    dx_, dy_, dz_, cg_its_, _ = K.hykkt_solve(F, W, sigma_x, J, dh, me, dw, gamma, a, b,
                                                              rtol=opt.cg_rtol)
                    eta_ = K.backward_error(K.aug_matrix(W, sigma_x, J, dh, me, dw),
                                            np.concatenate([dx_, dy_, dz_]), np.concatenate([a, b]))
                elif opt.kkt == "regularized":
                    # dual regularization delta_c = 1/gamma (Remark in Sec. 3): one condensed solve
                    # of (K + G^T G / delta_c) dx = r1bar + G^T r2bar / delta_c, dy = (G dx - r2bar)
                    # / delta_c, refined on the augmented system with -delta_c I in the equality block
                    b = np.concatenate([-r3_, bH])
                    d = np.concatenate([np.full(me, gamma), dh])
                    A = K.aug_matrix(W, sigma_x, J, d, 0, dw)
                    dx_, dzall, eh = K.lifted_solve(F, A, J, d, a, b, max_refine=opt.max_refine)
                    dy_, dz_ = dzall[:me], dzall[me:]
                    eta_ = eh[-1]
                else:
                    A = K.aug_matrix(W, sigma_x, J, dh, 0, dw)
                    dx_, dz_, eh = K.lifted_solve(F, A, J, dh, a, bH, max_refine=opt.max_refine)
                    dy_ = np.zeros(0)
                    eta_ = eh[-1]
                ds_ = -(r2 + dz_) / dh
                dv_ = (mu - v * ds_) / s - v
                dzl_ = np.where(hl, mu / dxl - zl - zl / dxl * dx_, 0.0)
                dzu_ = np.where(hu, mu / dxu - zu + zu / dxu * dx_, 0.0)
                return dx_, dy_, dz_, ds_, dv_, dzl_, dzu_, cg_its_, eta_

            dx, dy, dz, ds, dv, dzl, dzu, cg_its, eta = direction(r3, r4)

            # fraction to the boundary
            def ftb(val, dval):
                neg = dval < 0
                if not neg.any():
                    return 1.0
                return float(min(1.0, np.min(-tau * val[neg] / dval[neg])))

            amax = min(ftb(x[hl] - xl[hl], dx[hl]), ftb(xu[hu] - x[hu], -dx[hu]), ftb(s, ds))
            az = min(ftb(v, dv), ftb(zl[hl], dzl[hl]), ftb(zu[hu], dzu[hu]))

            theta = theta_of(g, h, s)
            phi = phi_of(x, s, mu)
            gphi = (sig_f * gradf @ dx - mu * np.sum(ds / s) - mu * np.sum((dx / dxl)[hl])
                    + mu * np.sum((dx / dxu)[hu]))
            if gphi < 0:
                amin = GAMMA_ALPHA * min(GAMMA_THETA, GAMMA_PHI * theta / -gphi,
                                         DELTA * theta ** S_THETA / (-gphi) ** S_PHI)
            else:
                amin = GAMMA_ALPHA * GAMMA_THETA
            alpha = amax
            accepted = False
            ls = 0

            while True:
                xt = x + alpha * dx
                st = s + alpha * ds
                gt, ht = model.cons(xt)
                tht = theta_of(gt, ht, st)
                pht = phi_of(xt, st, mu)
                accepted, ftype = filter_accept(theta, phi, gphi, alpha, tht, pht, filt, theta_min,
                                                theta_max)
                if accepted:
                    break
                ls += 1
                alpha *= 0.5
                if alpha < amin:
                    break
            soft = False
            if not accepted and opt.soft_restoration:
                # soft restoration (Ipopt's fallback before its restoration phase): the step damped
                # only by the fraction to the boundary (alpha_max, and az for the bound duals) is
                # taken if it reduces the primal-dual error of the barrier problem, E_mu, by the
                # factor 1 - 1e-4; the filter is left as it is
                xt = x + amax * dx
                st = s + amax * ds
                gt, ht = model.cons(xt)
                e_now = errors(gradf, J, g, h, mu)
                e_try = errors_at(xt, st, y + amax * dy, z + amax * dz, v + az * dv, zl + az * dzl,
                                  zu + az * dzu, model.grad(xt), model.jacobian(xt), gt, ht, mu)
                if e_try <= (1.0 - SOFT_RESTO_REDUCTION) * e_now:
                    accepted = soft = True
                    alpha = amax
                    ftype = True
            if (not accepted and restore and opt.restoration
                    and max(np.abs(g).max(initial=0.0), np.abs(h + s).max(initial=0.0)) <= opt.tol):
                # a failed line search at a point that is feasible within the tolerance: the
                # restoration phase cannot reduce a violation that is already at rounding level, and
                # its problem is solved by the point itself.  The direction is computed again
                # with the next delta_w of the iteration's inertia-correction schedule (a
                # better conditioned, more gradient-like step), at most MAX_LS_REGULARIZE times,
                # before the method stops there (reading)
                if n_reg < MAX_LS_REGULARIZE:
                    n_reg += 1
                    # the schedule's candidate after the accepted delta_w
                    nxt = (dw * grow0 if dw > 0 else
                           (max(1e-20, delta_last0 / 3.0) if delta_last0 > 0 else 1e-4))
                    sched = (nxt, grow0)
                    continue
                outcome = "restoration_failed"
                break
            if not accepted and restore and opt.restoration:
                # feasibility restoration (Waechter & Biegler 2006, Sec. 3.3): the current point
                # enters the filter, a point acceptable to it with a smaller constraint violation is
                # sought by an IPM on the restoration problem, and the iterations go on from there
                entry = ((1 - GAMMA_THETA) * theta, phi - GAMMA_PHI * theta)
                rec = _restoration(model, opt, x, s, v, zl, zu, mu, theta, theta_max,
                                   filt + [entry], theta_at, lambda xx, sx: phi_of(xx, sx, mu))
                n_resto += 1
                hist.append(dict(k=it, mu=mu, e0=e0, alpha=0.0, delta_w=dw, nfac=nfac, cg=cg_its,
                                 eta=eta, ls=ls, obj=model.objective(x), gamma=gamma, soft=False,
                                 resto=rec["iters"], resto_status=rec["status"]))
                if rec["status"] != "ok":
                    outcome = rec["status"]
                    break
                filt.append(entry)
                # constraint multipliers start again from zero, bound multipliers are kept (as in
                # Ipopt after its restoration phase)
                x, s, v, zl, zu = rec["x"], rec["s"], rec["v"], rec["zl"], rec["zu"]
                y = np.zeros(me)
                z = np.zeros(mi)
                outcome = "restored"
                break
            break
        if outcome == "restored":
            continue
        if outcome is not None:
            status = outcome
            break
        if not accepted:
            status = "restoration_needed"
            break
        if not ftype:
            filt.append(((1 - GAMMA_THETA) * theta, phi - GAMMA_PHI * theta))
        x = xt
        s = st
        y = y + alpha * dy
        z = z + alpha * dz
        v = v + az * dv
        zl = zl + az * dzl
        zu = zu + az * dzu
        # bound-multiplier safeguard (Ipopt Eq. (16))
        dxl = np.where(hl, x - xlf, 1.0)
        dxu = np.where(hu, xuf - x, 1.0)
        zl = np.where(hl, np.clip(zl, mu / (KAPPA_SIGMA * dxl), KAPPA_SIGMA * mu / dxl), 0.0)
        zu = np.where(hu, np.clip(zu, mu / (KAPPA_SIGMA * dxu), KAPPA_SIGMA * mu / dxu), 0.0)
        v = np.clip(v, mu / (KAPPA_SIGMA * s), KAPPA_SIGMA * mu / s)
        hist.append(dict(k=it, mu=mu, e0=e0, alpha=alpha, delta_w=dw, nfac=nfac, cg=cg_its,
                         eta=eta, ls=ls, obj=model.objective(x), gamma=gamma, soft=soft))
        if exit_check is not None and exit_check(x, s):
            status = "exited"
            break
        if opt.verbose:
            print(f"{it:4d} mu={mu:.1e} E0={e0:.2e} a={alpha:.2e} dw={dw:.1e} cg={cg_its} eta={eta:.1e}")
    g, h = model.cons(x)
    J = model.jacobian(x)
    return Result(status=status, iters=it, x=x, s=s, y=y, z=z, v=v, zl=zl, zu=zu,
                  obj=model.objective(x), kkt_error=errors(model.grad(x), J, g, h, 0.0), mu=mu,
                  history=hist)


def _restoration(model, opt, x, s, v, zl, zu, mu, theta, theta_max, filt, theta_at, phi_at):
    """The restoration phase (Waechter & Biegler 2006, Sec. 3.3): an IPM on RestorationModel
    at the reference point x, with mu_R = max(mu, ||c||_inf), zeta = sqrt(mu_R), p and q from
    resto_pq, the constraint multipliers at zero and the bound multipliers capped at rho.  It
    returns (status "ok") at the first restoration iterate whose x and s reduce the original
    constraint violation to at most KAPPA_RESTO theta and are acceptable to the original filter
    (which holds the point the phase started from); "infeasible" when it converges to a
    stationary point of the restoration problem first (a local minimizer of the violation) whose
    violation ||c||_inf exceeds the tolerance; "restoration_failed" otherwise (the phase's own
    line search or iteration limit, or convergence at a point feasible within the tolerance
    that the filter still rejects)."""
    n, me, mi = model.n, model.m_e, model.m_i
    g, h = model.cons(x)
    c = np.concatenate([g, h + s])
    mu_r = max(mu, float(np.abs(c).max()))
    R = RestorationModel(model, x, np.sqrt(mu_r))
    p, q = resto_pq(c, mu_r)
    m = len(c)
    start = dict(x=np.concatenate([x, p, q]), s=s.copy(), y=np.zeros(me), z=np.zeros(mi),
                 v=np.minimum(RHO_RESTO, v),
                 zl=np.concatenate([np.minimum(RHO_RESTO, zl), mu_r / p, mu_r / q]),
                 zu=np.concatenate([np.minimum(RHO_RESTO, zu), np.zeros(2 * m)]))

    def exit_check(w, sk):
        xk = w[:n]
        th = theta_at(xk, sk)
        if not th <= KAPPA_RESTO * theta:
            return False
        ph = phi_at(xk, sk)
        return th < theta_max and all(th < tf or ph < pf for tf, pf in filt)

    ropt = dataclasses.replace(opt, restoration=False)
    rr = _ipm(R, ropt, start, mu_r, 1.0, exit_check=exit_check, restore=False, max_iter=500)
    out = dict(iters=rr.iters)
    if rr.status != "exited":
        infeasible = False
        if rr.status == "converged":
            gk, hk = model.cons(rr.x[:n])
            cinf = max(np.abs(gk).max(initial=0.0), np.abs(hk + rr.s).max(initial=0.0))
            infeasible = cinf > opt.tol
        out["status"] = "infeasible" if infeasible else "restoration_failed"
        return out
    reset = lambda a: np.where(a > 1e3, 1.0, a)   # large bound multipliers reset (Ipopt)
    out.update(status="ok", x=rr.x[:n].copy(), s=rr.s.copy(), v=reset(rr.v),
               zl=reset(rr.zl[:n]), zu=reset(rr.zu[:n]))
    return out
