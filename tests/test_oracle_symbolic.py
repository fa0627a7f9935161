"""Pins for the oracle's symbolic analysis (no GPU).

Brute-force boolean Gaussian elimination is the definition of the filled graph:
eliminating column j connects all its later neighbours.  The elimination tree is
parent(j) = min{i > j : L_ij != 0}, column counts are |struct(L_j)| + 1, and a
supernode is a run of columns whose structures nest.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.sparse import Symbolic


def random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    A = rng.random((n, n)) < p
    A = np.triu(A, 1)
    A = A | A.T
    return sp.csr_matrix(A.astype(float) + np.eye(n))


def brute_force_fill(Pdense, perm):
    n = len(perm)
    B = Pdense[np.ix_(perm, perm)] != 0
    B = B.copy()
    for j in range(n):
        nb = np.nonzero(B[j + 1:, j])[0] + j + 1
        for a in nb:
            B[nb, a] = True
            B[a, nb] = True
    L = np.tril(B)
    return L


@pytest.mark.parametrize("n,p,seed", [(10, 0.3, 0), (25, 0.15, 1), (40, 0.08, 2), (60, 0.05, 3),
                                      (60, 0.3, 4), (150, 0.02, 5), (200, 0.015, 6)])
def test_fill_etree_counts_match_brute_force(n, p, seed):
    P = random_graph(n, p, seed)
    S = Symbolic(P)
    assert sorted(S.perm.tolist()) == list(range(n))
    L = brute_force_fill(P.toarray(), S.perm)
    for j in range(n):
        rows = np.nonzero(L[j + 1:, j])[0] + j + 1
        assert S.cc[j] == len(rows) + 1
        np.testing.assert_array_equal(S.rowind[S.colptr[j]:S.colptr[j + 1]], rows)
        assert S.parent[j] == (rows[0] if len(rows) else -1)


def test_supernodes_have_nested_structures():
    P = random_graph(150, 0.03, 11)
    S = Symbolic(P)
    assert S.sptr[0] == 0 and S.sptr[-1] == S.n
    for s in range(S.nsuper):
        f, l = S.sptr[s], S.sptr[s + 1]
        assert 1 <= l - f <= 64
        for j in range(f, l - 1):
            sj = set(S.rowind[S.colptr[j]:S.colptr[j + 1]].tolist())
            sj1 = set(S.rowind[S.colptr[j + 1]:S.colptr[j + 2]].tolist())
            assert sj == {j + 1} | sj1
        # maximality: the next column does not continue this supernode unless width capped
        if l < S.n and l - f < 64:
            assert not (S.parent[l - 1] == l and S.cc[l - 1] == S.cc[l] + 1)


def test_components_ordered_by_smallest_vertex():
    # three disjoint paths, vertex ids interleaved
    n = 90
    rows, cols = [], []
    for c in range(3):
        vs = list(range(c, n, 3))
        for a, b in zip(vs[:-1], vs[1:]):
            rows += [a, b]
            cols += [b, a]
    P = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n)) + sp.identity(n)
    S = Symbolic(P.tocsr())
    comp = S.perm % 3
    np.testing.assert_array_equal(comp, np.repeat([0, 1, 2], 30))


def test_dense_row_fills_everything():
    """A single dense row of the inequality Jacobian makes J^T J dense
    (Section 2.3): the filled graph is complete, nnz(L) = n(n+1)/2."""
    n = 80
    J = sp.random(60, n, density=0.02, random_state=1, format="csr")
    J = sp.vstack([J, sp.csr_matrix(np.ones((1, n)))]).tocsr()
    from oracle.sparse import condensed_pattern
    P = condensed_pattern(sp.identity(n, format="csr"), J)
    S = Symbolic(P)
    assert S.nnz_l == n * (n + 1) // 2


def test_fill_quality_on_lattice():
    """Nested dissection of a k x k lattice keeps fill far below the natural
    (banded) order, whose factor has about n*k entries."""
    k = 40
    n = k * k
    idx = np.arange(n).reshape(k, k)
    rows = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    cols = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    A = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    P = (A + A.T + sp.identity(n)).tocsr()
    S = Symbolic(P)
    natural = n * k
    assert S.nnz_l < 0.5 * natural
    assert S.nnz_l < 12 * n * np.log2(n)
