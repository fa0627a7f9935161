"""Why the FP32 factor is used without symmetric equilibration: Cholesky's rounding is invariant
under a symmetric diagonal scaling by powers of two, so scaling K to a unit-sized diagonal before
rounding it to FP32 changes neither whether the FP32 factorization succeeds nor the factor (up to
that scaling), and a scaling by the exact 1 / sqrt(diag K) changes it only at rounding level.
Checked with LAPACK's FP32 Cholesky on condensed matrices of the 30-bus and 1,000-bus KKT cases
(late-iteration shape: Sigma_x and D over sixteen decades) and on random SPD matrices with the
same spread of diagonal scales (test infrastructure; no GPU)."""
import numpy as np
import pytest

from tests.cases import kkt_case
from oracle import kkt as K


def fp32_chol(A):
    try:
        return np.linalg.cholesky(A.astype(np.float32))
    except np.linalg.LinAlgError:
        return None


def pow2_scaling(A):
    """D = 2^-round(log2 sqrt(a_jj)): D A D has diagonal entries in [0.5, 2]."""
    return np.exp2(-np.round(np.log2(np.sqrt(np.diag(A)))))


def random_spd(n, seed, spread=8.0):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n)) / np.sqrt(n)
    s = 10.0 ** rng.uniform(-spread, spread, n)
    return (B @ B.T + 1e-3 * np.eye(n)) * np.sqrt(np.outer(s, s))


def condensed(name):
    c = kkt_case(name)
    return K.condensed_matrix(c["Wf"], c["sigma"], c["J"], c["d"], c["dw"]).toarray()


CASES = [("ring30", None), ("planar1k", None)] + [(None, s) for s in range(6)]


@pytest.mark.parametrize("name,seed", CASES)
def test_power_of_two_equilibration_leaves_fp32_cholesky_unchanged(name, seed):
    A = condensed(name) if name else random_spd(120, seed)
    d = pow2_scaling(A)
    As = A * np.outer(d, d)
    L, Ls = fp32_chol(A), fp32_chol(As)
    assert (L is None) == (Ls is None)
    if L is not None:
        # the factor of the scaled matrix is the scaled factor, bit for bit
        np.testing.assert_array_equal(Ls, (L * d[:, None]).astype(np.float32))


def refine_rate(A, L, rng):
    """Mean contraction factor of FP64 Richardson refinement with the FP32 factor L of A."""
    b = rng.standard_normal(A.shape[0])
    x = np.zeros_like(b)
    rn = [np.linalg.norm(b)]
    for _ in range(6):
        r = b - A @ x
        y = np.linalg.solve(L.astype(np.float64), r)
        x = x + np.linalg.solve(L.astype(np.float64).T, y)
        rn.append(np.linalg.norm(b - A @ x))
    rn = np.array(rn)
    return float(np.exp(np.mean(np.log(rn[1:] / rn[:-1]))))


@pytest.mark.parametrize("seed", range(4))
def test_jacobi_equilibration_changes_fp32_refinement_only_at_rounding_level(seed):
    A = random_spd(120, seed, spread=4.0)
    d = 1.0 / np.sqrt(np.diag(A))
    As = A * np.outer(d, d)
    L, Ls = fp32_chol(A), fp32_chol(As)
    assert L is not None and Ls is not None
    rng = np.random.default_rng(seed)
    r0 = refine_rate(A, L, rng)
    r1 = refine_rate(As, Ls, np.random.default_rng(seed))
    # both contract (the FP32 factor preconditions either matrix), at the same rate within 4x
    assert r0 < 0.5 and r1 < 0.5
    assert max(r0, r1) <= 4 * min(r0, r1) + 1e-12, (r0, r1)
