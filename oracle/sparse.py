"""Oracle sparse symbolic analysis and Cholesky (Python side of the plain C code).

TEST INFRASTRUCTURE ONLY.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from ._clib import lib, ptr


def condensed_pattern(W: sp.spmatrix, J: sp.spmatrix) -> sp.csr_matrix:
    """Structural pattern of K = W + diag + J^T D J (Eq. (K_1), (9), (13)):
    pat(W) united with the diagonal and pat(J^T J).  Built from all-ones copies so
    that no numerical cancellation can remove an entry."""
    n = J.shape[1]
    Jp = sp.csr_matrix((np.ones(J.nnz), J.indices, J.indptr), shape=J.shape)
    Wp = sp.csr_matrix((np.ones(W.nnz), W.indices, W.indptr), shape=W.shape)
    Wp = Wp + Wp.T
    P = (Jp.T @ Jp + Wp + sp.identity(n, format="csr")).tocsr()
    P.sum_duplicates()
    P.sort_indices()
    return P


def adjacency(P: sp.csr_matrix):
    """Symmetric adjacency (no self loops) as int32 CSR arrays."""
    P = P.tocoo()
    keep = P.row != P.col
    A = sp.csr_matrix((np.ones(keep.sum()), (P.row[keep], P.col[keep])), shape=P.shape)
    A = ((A + A.T) > 0).astype(np.float64).tocsr()
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32)


class Symbolic:
    """Ordering, elimination tree, column structures and supernodes of a pattern."""

    def __init__(self, P: sp.csr_matrix, relax=(8, 5)):
        self.n = P.shape[0]
        ap, ai = adjacency(P)
        L = lib()
        h = L.osym_analyze_relaxed(self.n, ptr(ap), ptr(ai), int(relax[0]), int(relax[1]))
        ns = np.zeros(1, np.int32)
        nnz = np.zeros(1, np.int64)
        L.osym_sizes(h, ptr(ns), ptr(nnz))
        n = self.n
        self.perm = np.zeros(n, np.int32)
        self.parent = np.zeros(n, np.int32)
        self.cc = np.zeros(n, np.int32)
        self.sptr = np.zeros(int(ns[0]) + 1, np.int32)
        self.colptr = np.zeros(n + 1, np.int64)
        self.rowind = np.zeros(max(int(nnz[0]), 1), np.int32)
        L.osym_export(h, ptr(self.perm), ptr(self.parent), ptr(self.cc), ptr(self.sptr),
                      ptr(self.colptr), ptr(self.rowind))
        L.osym_free(h)
        self.rowind = self.rowind[:int(nnz[0])]
        self.iperm = np.empty(n, np.int32)
        self.iperm[self.perm] = np.arange(n, dtype=np.int32)
        self.nsuper = int(ns[0])

    @property
    def nnz_l(self) -> int:
        """Entries of L including the diagonal."""
        return int(self.cc.sum())

    def factor_flops(self) -> float:
        """Textbook count sum_j eta_j (eta_j + 3), eta_j = off-diagonal count of column j."""
        eta = self.cc.astype(np.float64) - 1.0
        return float(np.sum(eta * (eta + 3.0)))

    def supernode_rows(self, s: int) -> np.ndarray:
        """Row structure of supernode s: its columns, then the rows below them."""
        f, l = self.sptr[s], self.sptr[s + 1]
        below = self.rowind[self.colptr[l - 1]:self.colptr[l]]
        return np.concatenate([np.arange(f, l, dtype=np.int32), below])


class Cholesky:
    """LL^T of P K P^T using the oracle symbolic; ``ok`` is False on a failed pivot."""

    def __init__(self, K: sp.spmatrix, sym: Symbolic):
        self.sym = sym
        n = sym.n
        C = sp.csc_matrix(K)[sym.perm][:, sym.perm]
        C = sp.triu(C, format="csc")
        C.sort_indices()
        Cp = C.indptr.astype(np.int64)
        Ci = C.indices.astype(np.int32)
        Cx = C.data.astype(np.float64)
        self.Lp = np.zeros(n + 1, np.int64)
        self.Lp[1:] = np.cumsum(sym.cc)
        self.Li = np.zeros(int(self.Lp[-1]), np.int32)
        self.Lx = np.zeros(int(self.Lp[-1]), np.float64)
        self.fail = lib().ochol_factor(n, ptr(Cp), ptr(Ci), ptr(Cx), ptr(sym.parent),
                                       ptr(self.Lp), ptr(self.Li), ptr(self.Lx))
        self.ok = self.fail < 0

    def solve(self, b: np.ndarray) -> np.ndarray:
        assert self.ok
        y = np.ascontiguousarray(b[self.sym.perm], dtype=np.float64).copy()
        lib().ochol_solve(self.sym.n, ptr(self.Lp), ptr(self.Li), ptr(self.Lx), ptr(y))
        x = np.empty_like(y)
        x[self.sym.perm] = y
        return x

    def to_csc(self) -> sp.csc_matrix:
        n = self.sym.n
        return sp.csc_matrix((self.Lx, self.Li, self.Lp), shape=(n, n))
