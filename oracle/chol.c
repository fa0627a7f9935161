/*
 * Oracle sparse Cholesky (TEST INFRASTRUCTURE; shares no code with the CUDA path).
 *
 * Plain up-looking LL^T of an SPD matrix C (already permuted), row by row: row k of
 * L solves L[0:k,0:k] l = C[0:k,k] on the row's elimination-tree reach, and
 * L_kk = sqrt(C_kk - l.l).  The factorization fails, returning the column k, as soon
 * as a pivot C_kk - l.l is not positive or not finite: this is the positive-definite
 * test that replaces the inertia check for the condensed matrices (Section 3,
 * Eq. (9), (13)).  Returns -1 on success.
 *
 * Cp/Ci/Cx: upper triangle of C by columns (rows i <= k in column k).
 * Lp: column pointers of L with the diagonal first in each column (from the
 *     column counts of the symbolic analysis); Li/Lx receive rows/values.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static int cmp_int(const void *a, const void *b) {
  int x = *(const int *)a, y = *(const int *)b;
  return (x > y) - (x < y);
}

int ochol_factor(int n, const int64_t *Cp, const int *Ci, const double *Cx, const int *parent,
                 const int64_t *Lp, int *Li, double *Lx) {
  double *x = (double *)calloc(n + 1, sizeof(double));
  int *mark = (int *)malloc(sizeof(int) * (n + 1));
  int *pat = (int *)malloc(sizeof(int) * (n + 1));
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
  int fail = -1;
  for (int j = 0; j < n; ++j) {
    mark[j] = -1;
    fill[j] = Lp[j] + 1;
  }
  for (int k = 0; k < n && fail < 0; ++k) {
    int np = 0;
    double d = 0.0;
    mark[k] = k;
    for (int64_t p = Cp[k]; p < Cp[k + 1]; ++p) {
      int i = Ci[p];
      if (i == k) { d += Cx[p]; continue; }
      if (i > k) continue;
      x[i] += Cx[p];
      for (int j = i; j != -1 && mark[j] != k; j = parent[j]) {
        mark[j] = k;
        pat[np++] = j;
      }
    }
    qsort(pat, np, sizeof(int), cmp_int);
    for (int t = 0; t < np; ++t) {
      int j = pat[t];
      double lkj = x[j] / Lx[Lp[j]];
      x[j] = 0.0;
      for (int64_t p = Lp[j] + 1; p < fill[j]; ++p) x[Li[p]] -= Lx[p] * lkj;
      d -= lkj * lkj;
      Li[fill[j]] = k;
      Lx[fill[j]] = lkj;
      fill[j]++;
    }
    if (!(d > 0.0) || !isfinite(d)) {
      fail = k;
      break;
    }
    Li[Lp[k]] = k;
    Lx[Lp[k]] = sqrt(d);
  }
  free(x);
  free(mark);
  free(pat);
  free(fill);
  return fail;
}

/* Solve L L^T x = b in place (b overwritten by x). */
void ochol_solve(int n, const int64_t *Lp, const int *Li, const double *Lx, double *b) {
  for (int j = 0; j < n; ++j) {
    b[j] /= Lx[Lp[j]];
    for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; ++p) b[Li[p]] -= Lx[p] * b[j];
  }
  for (int j = n - 1; j >= 0; --j) {
    double s = b[j];
    for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; ++p) s -= Lx[p] * b[Li[p]];
    b[j] = s / Lx[Lp[j]];
  }
}
