"""Pins for the oracle's sparse Cholesky and KKT solves (no GPU)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle.sparse import Symbolic, Cholesky, condensed_pattern
from oracle import kkt as K


def random_spd(n, density, seed, shift=1.0):
    A = sp.random(n, n, density=density, random_state=seed, format="csr")
    return (A @ A.T + shift * sp.identity(n)).tocsr()


@pytest.mark.parametrize("n,seed", [(5, 0), (50, 1), (200, 2)])
def test_cholesky_matches_dense(n, seed):
    Kmat = random_spd(n, 0.05, seed)
    S = Symbolic(Kmat)
    F = Cholesky(Kmat, S)
    assert F.ok
    L = F.to_csc().toarray()
    C = Kmat.toarray()[np.ix_(S.perm, S.perm)]
    np.testing.assert_allclose(L, np.linalg.cholesky(C), rtol=1e-12, atol=1e-12)
    b = np.random.default_rng(seed).standard_normal(n)
    np.testing.assert_allclose(F.solve(b), np.linalg.solve(Kmat.toarray(), b), rtol=1e-9)


def test_cholesky_backward_error_bound():
    """||P K P^T - L L^T|| / ||K|| within a small multiple of n u (Assumption 4.2)."""
    Kmat = random_spd(300, 0.02, 3)
    S = Symbolic(Kmat)
    F = Cholesky(Kmat, S)
    L = F.to_csc().toarray()
    C = Kmat.toarray()[np.ix_(S.perm, S.perm)]
    err = np.abs(C - L @ L.T).max() / np.abs(C).max()
    assert err < 300 * np.finfo(float).eps


def test_cholesky_failure_column_is_first_indefinite_minor():
    rng = np.random.default_rng(4)
    n = 40
    A = rng.standard_normal((n, n))
    Kd = A @ A.T + 0.1 * np.eye(n)
    Kd[25, 25] -= 200.0
    Kd[30, 30] -= 500.0
    Kmat = sp.csr_matrix(Kd)
    S = Symbolic(Kmat)
    F = Cholesky(Kmat, S)
    assert not F.ok
    C = Kd[np.ix_(S.perm, S.perm)]
    first = next(k for k in range(n) if np.linalg.eigvalsh(C[:k + 1, :k + 1]).min() <= 0)
    assert F.fail == first


def small_kkt(n=30, me=8, mi=20, seed=0, convex=True):
    rng = np.random.default_rng(seed)
    J = sp.random(me + mi, n, density=0.2, random_state=seed, format="csr")
    J = (J + sp.eye(me + mi, n, format="csr")).tocsr()
    Wd = rng.standard_normal((n, n))
    Wd = (Wd + Wd.T) / 2
    if convex:
        Wd = Wd @ Wd.T / n + 0.1 * np.eye(n)
    W = sp.csr_matrix(Wd * (np.abs(Wd) > 0.8))
    W = (W + W.T) / 2
    sigma = 10.0 ** rng.uniform(-4, 4, n)
    dh = 10.0 ** rng.uniform(-4, 4, mi)
    return J, W, sigma, dh


def test_condensed_solution_equals_augmented():
    """Eliminating (d_s, d_z) gives the condensed system (K_1) with the same d_x."""
    n, me, mi = 30, 0, 25
    J, W, sigma, dh = small_kkt(n, me, mi, 1)
    rng = np.random.default_rng(7)
    a, b = rng.standard_normal(n), rng.standard_normal(mi)
    solver = K.CondensedSolver(W, J)
    dw, F, _ = K.inertia_schedule(lambda d: K.condensed_matrix(W, sigma, J, dh, d), solver)
    A = K.aug_matrix(W, sigma, J, dh, 0, dw)
    dx, dz, hist = K.lifted_solve(F, A, J, dh, a, b)
    ref = np.linalg.solve(A.toarray(), np.concatenate([a, b]))
    np.testing.assert_allclose(np.concatenate([dx, dz]), ref, rtol=1e-8, atol=1e-10)
    assert hist[-1] <= 1e-10


def test_augmented_is_k2_with_slacks_eliminated():
    """(K_2) with the d_s block solved out equals the system the oracle builds."""
    n, me, mi = 12, 4, 9
    J, W, sigma, dh_unused = small_kkt(n, me, mi, 2)
    rng = np.random.default_rng(3)
    Ds = 10.0 ** rng.uniform(-2, 2, mi)
    dw = 0.3
    G, H = J[:me].toarray(), J[me:].toarray()
    Z = np.zeros
    K2 = np.block([
        [W.toarray() + np.diag(sigma + dw), Z((n, mi)), G.T, H.T],
        [Z((mi, n)), np.diag(Ds + dw), Z((mi, me)), np.eye(mi)],
        [G, Z((me, mi)), Z((me, me)), Z((me, mi))],
        [H, np.eye(mi), Z((mi, me)), Z((mi, mi))]])
    r1, r2, r3, r4 = (rng.standard_normal(k) for k in (n, mi, me, mi))
    sol = np.linalg.solve(K2, -np.concatenate([r1, r2, r3, r4]))
    dx, ds, dy, dz = np.split(sol, np.cumsum([n, mi, me]))
    DH = Ds + dw
    A = K.aug_matrix(W, sigma, J, DH, me, dw).toarray()
    rhs = np.concatenate([-r1, -r3, -r4 + r2 / DH])
    sol2 = np.linalg.solve(A, rhs)
    np.testing.assert_allclose(sol2, np.concatenate([dx, dy, dz]), rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(-(r2 + dz) / DH, ds, rtol=1e-9, atol=1e-11)


def test_inertia_equivalence():
    """Eq. (7) with m_e = 0: inertia(AUG) = (n, m_i, 0) iff K is positive definite."""
    n, mi = 20, 15
    for seed in range(6):
        J, W, sigma, dh = small_kkt(n, 0, mi, seed, convex=False)
        sigma = sigma * 1e-4
        for dw in (0.0, 0.5, 5.0):
            Kc = K.condensed_matrix(W, sigma, J, dh, dw).toarray()
            pd = np.linalg.eigvalsh(Kc).min() > 0
            A = K.aug_matrix(W, sigma, J, dh, 0, dw).toarray()
            _, D, _ = sla.ldl(A)
            ev = np.linalg.eigvalsh(D)
            inertia_ok = (ev > 0).sum() == n and (ev < 0).sum() == mi
            assert pd == inertia_ok


def test_hykkt_matches_dense_and_cg_trends():
    n, me, mi = 40, 10, 25
    J, W, sigma, dh = small_kkt(n, me, mi, 5)
    rng = np.random.default_rng(9)
    a, b = rng.standard_normal(n), rng.standard_normal(me + mi)
    A = K.aug_matrix(W, sigma, J, dh, me, 0.0).toarray()
    ref = np.linalg.solve(A, np.concatenate([a, b]))
    solver = K.CondensedSolver(W, J)
    its, spread = [], []
    G = J[:me]
    for gamma in (1e2, 1e4, 1e6, 1e8):
        d = np.concatenate([np.full(me, gamma), dh])
        F = solver.factor(K.condensed_matrix(W, sigma, J, d, 0.0))
        assert F.ok
        dx, dy, dz, it, rel = K.hykkt_solve(F, W, sigma, J, dh, me, 0.0, gamma, a, b)
        np.testing.assert_allclose(np.concatenate([dx, dy, dz]), ref, rtol=1e-6 * max(1, gamma / 1e4),
                                   atol=1e-8)
        its.append(it)
        Kg = K.condensed_matrix(W, sigma, J, d, 0.0).toarray()
        S = G.toarray() @ np.linalg.solve(Kg, G.toarray().T)
        ev = np.linalg.eigvalsh(S)
        spread.append(np.abs(gamma * ev - 1).max())
    # Section 3.1: eigenvalues of S_gamma converge to 1/gamma, fewer CG iterations
    assert all(x >= y for x, y in zip(its, its[1:]))
    assert all(x > y for x, y in zip(spread, spread[1:]))
    assert spread[-1] < 1e-3


def test_dual_regularized_solve_equals_dense_and_tends_to_k2():
    """The dual-regularized condensed form (Remark in Sec. 3: delta_c > 0 on the equality block,
    condensed with weight gamma = 1/delta_c on the G rows): the oracle's refined condensed solve
    equals the dense solve of the augmented system whose equality block is -delta_c I, and as
    delta_c -> 0 that solution tends to the solution of the unregularized system (equalities
    kept exactly) with an error of order delta_c."""
    n, me, mi = 30, 6, 20
    J, W, sigma, dh = small_kkt(n, me, mi, 4)
    rng = np.random.default_rng(11)
    a, b = rng.standard_normal(n), rng.standard_normal(me + mi)
    solver = K.CondensedSolver(W, J)
    exact = np.linalg.solve(K.aug_matrix(W, sigma, J, dh, me, 0.0).toarray(),
                            np.concatenate([a, b]))
    errs = []
    for gamma in (1e2, 1e4, 1e6):
        d = np.concatenate([np.full(me, gamma), dh])
        dw, F, _ = K.inertia_schedule(lambda dd: K.condensed_matrix(W, sigma, J, d, dd), solver)
        assert dw == 0.0
        A = K.aug_matrix(W, sigma, J, d, 0, 0.0)
        dx, dz, hist = K.lifted_solve(F, A, J, d, a, b)
        sol = np.concatenate([dx, dz])
        ref = np.linalg.solve(A.toarray(), np.concatenate([a, b]))
        np.testing.assert_allclose(sol, ref, rtol=1e-7, atol=1e-9)
        assert hist[-1] <= 1e-10
        errs.append(np.abs(sol - exact).max() / np.abs(exact).max())
    # first order in delta_c = 1/gamma: a hundredfold smaller delta_c, a hundredfold smaller gap
    assert errs[0] > 30 * errs[1] > 900 * errs[2], errs
    assert errs[2] < 1e-4
