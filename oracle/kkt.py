"""Oracle KKT solves in FP64 (TEST INFRASTRUCTURE ONLY).

Notation follows Section 2.2 and Section 3 of the paper.  J = [G; H] stacks the
m_e equality rows G over the m_i inequality rows H.  With the slack block of the
augmented system (K_2) eliminated (it is diagonal: D_s + delta_w I), what remains
is the augmented system

    [ W + Sigma_x + delta_w I   G^T    H^T      ] [dx]   [a  ]
    [ G                          0      0        ] [dy] = [b_G]          (AUG)
    [ H                          0   -D_H^{-1}   ] [dz]   [b_H]

with D_H = D_s + delta_w (delta_c = 0, so C = I in Eq. (K_1)).  Eliminating dz
gives the condensed system (K_1):
    K dx + G^T dy = a + H^T D_H b_H,   G dx = b_G,   K = W + Sigma_x + delta_w I + H^T D_H H,
and dz = D_H (H dx - b_H).

* LiftedKKT (Section 3.2, Eq. (12)-(13)): every row is an inequality (the
  equalities relaxed to -tau <= g <= tau), so m_e = 0 and K_tau dx = a + J^T D b.
  Iterative refinement (Richardson) runs on (AUG) in FP64 (Section 2.2,
  "Iterative refinement"; Section 3.2 last paragraph).
* HyKKT (Section 3.1, Eq. (9)-(10)): K_gamma = K + gamma G^T G is factored by
  Cholesky and the Schur system (G K_gamma^{-1} G^T) dy = G K_gamma^{-1}
  (r1bar + gamma G^T r2bar) - r2bar is solved by CG; then
  K_gamma dx = r1bar + gamma G^T r2bar - G^T dy.

Readings where the paper is silent:
  CG starts at dy = 0 and stops when ||r_k||_2 <= max(rtol ||r_0||_2, atol);
  refinement stops at backward error <= 1e-10, when the error stops halving,
  or after 10 steps (LiftedKKT) or 3 HyKKT re-solves (HyKKT).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .sparse import Symbolic, Cholesky, condensed_pattern


def lower(W: sp.spmatrix) -> sp.csr_matrix:
    return sp.tril(sp.csr_matrix(W), format="csr")


def full_from_lower(Wl: sp.spmatrix) -> sp.csr_matrix:
    Wl = sp.csr_matrix(Wl)
    return (Wl + sp.tril(Wl, -1).T).tocsr()


def condensed_matrix(W, sigma_x, J, d, delta_w):
    """K = W + diag(sigma_x + delta_w) + J^T diag(d) J  (Eq. (K_1), (9), (13))."""
    n = J.shape[1]
    K = W + sp.diags(sigma_x + delta_w) + J.T @ sp.diags(d) @ J
    K = sp.csr_matrix(K)
    K.sum_duplicates()
    return K


def aug_matrix(W, sigma_x, J, d_h, m_e, delta_w):
    """The augmented matrix (AUG) above, rows/cols ordered (x, y, z)."""
    n = J.shape[1]
    m = J.shape[0]
    E = np.zeros(m)
    E[m_e:] = -1.0 / d_h
    top = sp.hstack([W + sp.diags(sigma_x + delta_w), J.T])
    bot = sp.hstack([J, sp.diags(E)])
    return sp.vstack([top, bot]).tocsr()


def backward_error(A, sol, rhs) -> float:
    """eta = ||A sol - rhs||_inf / (||A||_inf ||sol||_inf + ||rhs||_inf)."""
    r = A @ sol - rhs
    nA = abs(A).sum(axis=1).max()
    return float(np.abs(r).max() / (nA * np.abs(sol).max() + np.abs(rhs).max()))


class CondensedSolver:
    """Symbolic analysis once per pattern, then factor / solve per iteration."""

    def __init__(self, W_pattern, J_pattern):
        self.P = condensed_pattern(W_pattern, J_pattern)
        self.sym = Symbolic(self.P)

    def factor(self, K):
        # the C factorization writes only the columns the analysis allocated: an entry of K
        # outside the analysed pattern is a caller error, reported here
        Kp = sp.csr_matrix((np.ones(K.nnz), K.indices, K.indptr), shape=K.shape)
        Pp = sp.csr_matrix((np.ones(self.P.nnz), self.P.indices, self.P.indptr), shape=self.P.shape)
        if (Kp - Kp.multiply(Pp)).count_nonzero():
            raise ValueError("K has entries outside the analysed pattern")
        return Cholesky(K, self.sym)


def inertia_schedule(K_of_delta, solver, delta_last=0.0):
    """Primal regularization search (Section 2.2, inertia correction of
    Waechter & Biegler Section 3.1, Cholesky success replacing the inertia test
    as in Section 3): try delta_w = 0; then delta_last/3 (or 1e-4 the first time),
    growing by 8 (after a previous success) or 100 (first time) until the
    Cholesky factorization succeeds.  Returns (delta_w, factor, n_factorizations)."""
    nf = 1
    F = solver.factor(K_of_delta(0.0))
    if F.ok:
        return 0.0, F, nf
    delta = max(1e-20, delta_last / 3.0) if delta_last > 0 else 1e-4
    grow = 8.0 if delta_last > 0 else 100.0
    while delta < 1e40:
        nf += 1
        F = solver.factor(K_of_delta(delta))
        if F.ok:
            return delta, F, nf
        delta *= grow
    raise RuntimeError("inertia correction failed")


def lifted_solve(F, A, J, d, a, b, max_refine=10, tol=1e-10):
    """LiftedKKT solve of (AUG) with m_e = 0: condensed solve + Richardson refinement."""
    n = J.shape[1]

    def csolve(ra, rb):
        dx = F.solve(ra + J.T @ (d * rb))
        dz = d * (J @ dx - rb)
        return np.concatenate([dx, dz])

    rhs = np.concatenate([a, b])
    sol = csolve(a, b)
    eta = backward_error(A, sol, rhs)
    hist = [eta]
    for _ in range(max_refine):
        if eta <= tol:
            break
        res = rhs - A @ sol
        corr = csolve(res[:n], res[n:])
        eta_new = backward_error(A, sol + corr, rhs)
        hist.append(eta_new)
        if not eta_new <= eta:      # the correction made it worse: keep the previous solution
            break
        sol = sol + corr
        stalled = eta_new > 0.5 * eta
        eta = eta_new
        if stalled:
            break
    if np.isfinite(eta) and eta > tol and max_refine > 0:
        # Richardson stagnated: conjugate gradients on K dx = a + J^T (d o b) preconditioned by
        # the factor, from the refined dx; dz = d o (J dx - b); the better solution is kept
        x = pcg_condensed(F, A[:n, :n], J, d, a + J.T @ (d * b), sol[:n].copy(), 50,
                          normwise=False)
        alt = np.concatenate([x, d * (J @ x - b)])
        eta_alt = backward_error(A, alt, rhs)
        hist.append(eta_alt)
        if eta_alt < eta:
            sol = alt
    return sol[:n], sol[n:], hist


def pcg_condensed(F, Axx, J, d, t, x, maxit, normwise=True):
    """Preconditioned CG on K x = t, K v = Axx v + J^T (d o (J v)), M^{-1} = the factor F,
    from the given x; stops at ||r||_2 <= 1e-14 ||t||_2 or (normwise) a normwise backward error
    ||r||_inf <= 1e-14 (||K||_inf ||x||_inf + ||t||_inf) (||K||_inf bounded by the row sums of
    |Axx| + |J|^T |d| |J|), after maxit iterations, or at negative curvature.  After stagnating
    refinement the normwise test is off: with large d it is far looser than the backward error
    of the augmented system."""
    kv = lambda v: Axx @ v + J.T @ (d * (J @ v))
    knorm = float(np.max(abs(Axx) @ np.ones(Axx.shape[0]) +
                         abs(J).T @ (np.abs(d) * (abs(J) @ np.ones(J.shape[1])))))
    tn, tinf = np.linalg.norm(t), np.abs(t).max()
    r = t - kv(x)
    z = F.solve(r)
    p = z.copy()
    rz = float(r @ z)
    for _ in range(maxit):
        if (np.linalg.norm(r) <= 1e-14 * tn or
                (normwise and np.abs(r).max() <= 1e-14 * (knorm * np.abs(x).max() + tinf))):
            break
        Ap = kv(p)
        pap = float(p @ Ap)
        if not pap > 0:
            break
        al = rz / pap
        x = x + al * p
        r = r - al * Ap
        z = F.solve(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x


def hykkt_cg(F, G, gamma, r1bar, r2bar, rtol=1e-10, atol=1e-14, maxit=None):
    """Eq. (10): CG on S_gamma = G K_gamma^{-1} G^T, then the primal back-solve."""
    m_e = G.shape[0]
    if maxit is None:
        maxit = max(m_e, 1)
    rhs1 = r1bar + gamma * (G.T @ r2bar)
    w = F.solve(rhs1)
    rhs = G @ w - r2bar
    dy = np.zeros(m_e)
    r = rhs.copy()
    p = r.copy()
    rr = float(r @ r)
    r0 = np.sqrt(rr)
    stop = max(rtol * r0, atol)
    it = 0
    while np.sqrt(rr) > stop and it < maxit:
        Sp = G @ F.solve(G.T @ p)
        alpha = rr / float(p @ Sp)
        dy += alpha * p
        r -= alpha * Sp
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    dx = F.solve(rhs1 - G.T @ dy)
    return dx, dy, it, float(np.sqrt(rr) / max(r0, 1e-300))


def hykkt_solve(F, W, sigma_x, J, d_h, m_e, delta_w, gamma, a, b, max_refine=3, tol=1e-10,
                **cg):
    """HyKKT solve of (AUG): condense H, CG on the Schur complement, recover dz; then, while the
    backward error on (AUG) exceeds tol, Richardson refinement on (AUG) with the same HyKKT
    procedure solving for the residual (Section 2.2, iterative refinement on the original
    system; at most max_refine corrections, stopping when the error fails to halve).
    Returns dx, dy, dz, the CG iterations of all solves, and the first CG's final relative
    residual."""
    G = J[:m_e]
    H = J[m_e:]
    n = J.shape[1]

    def once(ra, rb):
        r1bar = ra + H.T @ (d_h * rb[m_e:])
        dx_, dy_, it_, rel_ = hykkt_cg(F, G, gamma, r1bar, rb[:m_e], **cg)
        dz_ = d_h * (H @ dx_ - rb[m_e:])
        return np.concatenate([dx_, dy_, dz_]), it_, rel_

    A = aug_matrix(W, sigma_x, J, d_h, m_e, delta_w)
    rhs = np.concatenate([a, b])
    sol, it, rel = once(a, b)
    eta = backward_error(A, sol, rhs)
    for _ in range(max_refine):
        if eta <= tol:
            break
        res = rhs - A @ sol
        # solve for the residual scaled to unit size (the CG's absolute floor must not end the
        # correction early), then scale the correction back
        sc = float(np.abs(res).max()) or 1.0
        corr, it2, _ = once(res[:n] / sc, res[n:] / sc)
        it += it2
        eta_new = backward_error(A, sol + sc * corr, rhs)
        if not eta_new <= eta:      # worse: keep the previous solution
            break
        sol = sol + sc * corr
        stalled = eta_new > 0.5 * eta
        eta = eta_new
        if stalled:
            break
    return sol[:n], sol[n:n + m_e], sol[n + m_e:], it, rel
