"""Pins for the oracle's symbolic analysis (no GPU).

Brute-force boolean Gaussian elimination is the definition of the filled graph:
eliminating column j connects all its later neighbours.  The elimination tree is
parent(j) = min{i > j : L_ij != 0}, column counts are |struct(L_j)| + 1, and the relaxed
supernodes follow their rule written out over the brute-force structures.
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


def relaxed_partition(struct, parent, maxw=64, relax_w=8, relax_den=5):
    """The relaxed supernode rule written out from its definition: a supernode is a run f..l of
    a chain (parent(k) = k+1); column l+1 joins it when parent(l) = l+1, the width stays <= maxw,
    and the width is <= relax_w or the panel's explicit zeros are <= 1/relax_den of its entries
    (panel column k holds rows k..l and struct(L_l))."""
    n = len(struct)
    starts = [0]
    for j in range(1, n):
        f = starts[-1]
        if parent[j - 1] == j:
            w = j - f + 1
            entries = sum((j - k + 1) + len(struct[j]) for k in range(f, j + 1))
            nz = sum(1 + len(struct[k]) for k in range(f, j + 1))
            zeros = entries - nz
            if w <= maxw and (w <= relax_w or zeros == 0 or
                              (relax_den > 0 and relax_den * zeros <= entries)):
                continue
        starts.append(j)
    return starts + [n]


@pytest.mark.parametrize("n,p,seed", [(60, 0.05, 3), (150, 0.03, 11), (200, 0.015, 6),
                                      (120, 0.2, 7)])
@pytest.mark.parametrize("relax", [(8, 5), (1, 0), (4, 10), (64, 1)])
def test_relaxed_supernodes_match_definition(n, p, seed, relax):
    P = random_graph(n, p, seed)
    S = Symbolic(P, relax=relax)
    L = brute_force_fill(P.toarray(), S.perm)
    struct = [set((np.nonzero(L[j + 1:, j])[0] + j + 1).tolist()) for j in range(n)]
    parent = [min(st) if st else -1 for st in struct]
    expect = relaxed_partition(struct, parent, relax_w=relax[0], relax_den=relax[1])
    np.testing.assert_array_equal(S.sptr, expect)
    for s_ in range(S.nsuper):
        f, l = S.sptr[s_], S.sptr[s_ + 1]
        assert 1 <= l - f <= 64
        for k in range(f, l - 1):
            assert parent[k] == k + 1                      # a chain of the elimination tree
            assert struct[k] <= set(range(k + 1, l)) | struct[l - 1]   # panel rows cover L_k
    fundamental = sum(1 for j in range(n) if j == 0 or parent[j - 1] != j or
                      len(struct[j - 1]) != len(struct[j]) + 1)
    assert S.nsuper <= fundamental + n // 64 + 1
    if relax == (1, 0):   # no explicit zeros at all: the fundamental supernodes
        for s_ in range(S.nsuper):
            f, l = S.sptr[s_], S.sptr[s_ + 1]
            for k in range(f, l - 1):
                assert struct[k] == {k + 1} | struct[k + 1]


def test_relaxed_supernodes_on_a_path_and_a_star():
    """Small cases: a path of 10 vertices (its elimination tree under the analysis' ordering
    has short chains) and a star of 8 vertices (the centre is eliminated last, every leaf is its
    child and only the leaf just before it forms a chain with it; width <= 8 merges them)."""
    n = 10
    A = sp.diags([np.ones(n - 1), np.ones(n - 1)], [-1, 1], shape=(n, n)) + sp.identity(n)
    S = Symbolic(sp.csr_matrix(A))
    L = brute_force_fill(A.toarray(), S.perm)
    struct = [set((np.nonzero(L[j + 1:, j])[0] + j + 1).tolist()) for j in range(n)]
    parent = [min(st) if st else -1 for st in struct]
    np.testing.assert_array_equal(S.sptr, relaxed_partition(struct, parent))
    # star: centre 0 joined to 1..7
    m = 8
    B = sp.lil_matrix((m, m))
    B.setdiag(1.0)
    for v in range(1, m):
        B[0, v] = B[v, 0] = 1.0
    S2 = Symbolic(B.tocsr())
    L2 = brute_force_fill(B.toarray(), S2.perm)
    st2 = [set((np.nonzero(L2[j + 1:, j])[0] + j + 1).tolist()) for j in range(m)]
    par2 = [min(st) if st else -1 for st in st2]
    np.testing.assert_array_equal(S2.sptr, relaxed_partition(st2, par2))
    assert S2.sptr[-2] <= m - 2   # the centre shares its supernode with a leaf


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
