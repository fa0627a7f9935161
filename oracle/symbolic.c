/*
 * Oracle symbolic analysis for the condensed KKT matrix (TEST INFRASTRUCTURE).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg load this
 * file's library.  It shares no code with the CUDA path.
 *
 * The paper leaves the fill-reducing ordering to the sparse solver (cuDSS does it on
 * the host; CHOLMOD uses AMD, Section 5).  Both sides of this project implement one
 * deterministic ordering so that the GPU result can be checked bit-exactly:
 *
 *   ND(P):  for each connected component C of G[P], in increasing order of its
 *           smallest vertex, place ND_conn(C) at the next free positions.
 *   ND_conn(C):
 *     |C| <= LEAF: minimum degree on the component's elimination graph; ties go to
 *                  the smallest vertex index.
 *     otherwise:   root = min(C); BFS level structure from root; up to REROOT times:
 *                  cand = smallest vertex of the last level, BFS from cand, and keep it
 *                  as root only if its eccentricity is larger (else stop).
 *                  k = first level whose cumulative size reaches ceil(|C|/2); if k is the
 *                  last level, k = k - 1.  S = vertices of level k with a neighbour in
 *                  level k+1.  A = levels < k plus (level k minus S), B = levels > k.
 *                  Positions: ND(A), then ND(B), then S in ascending vertex index.
 *
 * The elimination tree and the column structures of L follow their definitions
 * (symbolic elimination): struct(L_j) = {i > j : A_ij != 0} united with
 * struct(L_c) minus {j} over the children c of j; parent(j) = min struct(L_j).
 * Supernodes (relaxed): a supernode is a run of consecutive columns f..l in which
 * parent(k) = k+1 for f <= k < l (a chain of the elimination tree).  Its panel holds, in
 * every column k, the rows k..l and the rows of struct(L_l); the entries of the panel that are
 * not in struct(L_k) are explicit zeros.  Scanning the columns in order, column l+1 joins the
 * supernode f..l when parent(l) = l+1, the width w = l+2-f stays <= SN_MAXW, and w <= relax_w,
 * or the panel has no explicit zero, or (relax_den > 0) the explicit zeros are at most
 * 1/relax_den of the panel's entries (E = w(w+1)/2 + w |struct(L_{l+1})|, zeros = E -
 * sum_k |L_k|); otherwise l+1 starts a new supernode.  (relax_w, relax_den) = (1, 0) gives the
 * fundamental supernodes; osym_analyze uses (8, 5).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define LEAF 64
#define REROOT 4
#define SN_MAXW 64

typedef struct {
  int n;
  const int *ap, *ai;
  int *perm;
  int *inpart; /* stamp: vertex belongs to the current part */
  int *vis;    /* stamp: visited in current BFS */
  int *lev;    /* BFS level */
  int stamp;
  int *queue;
  int next_pos;
} nd_ctx;

static int cmp_int(const void *a, const void *b) {
  int x = *(const int *)a, y = *(const int *)b;
  return (x > y) - (x < y);
}

/* BFS restricted to vertices v with inpart[v]==pst; returns number of vertices
   reached; queue holds them in BFS order, lev their level. *nlev = #levels. */
static int bfs(nd_ctx *c, int root, int pst, int *nlev) {
  int st = ++c->stamp;
  int head = 0, tail = 0;
  c->queue[tail++] = root;
  c->vis[root] = st;
  c->lev[root] = 0;
  int maxl = 0;
  while (head < tail) {
    int v = c->queue[head++];
    for (int p = c->ap[v]; p < c->ap[v + 1]; ++p) {
      int u = c->ai[p];
      if (c->inpart[u] != pst || c->vis[u] == st) continue;
      c->vis[u] = st;
      c->lev[u] = c->lev[v] + 1;
      if (c->lev[u] > maxl) maxl = c->lev[u];
      c->queue[tail++] = u;
    }
  }
  *nlev = maxl + 1;
  return tail;
}

/* minimum degree on a part of at most LEAF vertices (sorted ascending). */
static void min_degree(nd_ctx *c, int *vs, int cnt) {
  uint64_t adj[LEAF];
  int pst = ++c->stamp;
  for (int k = 0; k < cnt; ++k) c->inpart[vs[k]] = pst;
  for (int k = 0; k < cnt; ++k) {
    adj[k] = 0;
    int v = vs[k];
    for (int p = c->ap[v]; p < c->ap[v + 1]; ++p) {
      int u = c->ai[p];
      if (c->inpart[u] != pst) continue;
      /* local index of u: binary search in the sorted list */
      int lo = 0, hi = cnt - 1;
      while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (vs[mid] < u) lo = mid + 1; else hi = mid;
      }
      adj[k] |= (uint64_t)1 << lo;
    }
  }
  uint64_t alive = (cnt == 64) ? ~(uint64_t)0 : (((uint64_t)1 << cnt) - 1);
  for (int step = 0; step < cnt; ++step) {
    int best = -1, bestd = 1 << 30;
    for (int k = 0; k < cnt; ++k) {
      if (!((alive >> k) & 1)) continue;
      int d = __builtin_popcountll(adj[k] & alive & ~((uint64_t)1 << k));
      if (d < bestd) { bestd = d; best = k; }
    }
    c->perm[c->next_pos++] = vs[best];
    uint64_t nb = adj[best] & alive & ~((uint64_t)1 << best);
    alive &= ~((uint64_t)1 << best);
    for (int k = 0; k < cnt; ++k)
      if ((nb >> k) & 1) adj[k] |= nb & ~((uint64_t)1 << k);
  }
}

static void nd(nd_ctx *c, int *vs, int cnt);

static void nd_conn(nd_ctx *c, int *vs, int cnt) {
  if (cnt <= LEAF) {
    qsort(vs, cnt, sizeof(int), cmp_int);
    min_degree(c, vs, cnt);
    return;
  }
  int pst = ++c->stamp;
  int root = vs[0];
  for (int k = 0; k < cnt; ++k) {
    c->inpart[vs[k]] = pst;
    if (vs[k] < root) root = vs[k];
  }
  int nlev;
  bfs(c, root, pst, &nlev);
  for (int it = 0; it < REROOT; ++it) {
    int cand = -1;
    for (int k = 0; k < cnt; ++k) {
      int v = vs[k];
      if (c->lev[v] == nlev - 1 && (cand < 0 || v < cand)) cand = v;
    }
    int nlev2;
    /* BFS from cand overwrites lev; keep a copy of the old levels */
    int *old = (int *)malloc(sizeof(int) * cnt);
    for (int k = 0; k < cnt; ++k) old[k] = c->lev[vs[k]];
    bfs(c, cand, pst, &nlev2);
    if (nlev2 > nlev) {
      root = cand;
      nlev = nlev2;
      free(old);
    } else {
      for (int k = 0; k < cnt; ++k) c->lev[vs[k]] = old[k];
      free(old);
      break;
    }
  }
  /* level sizes and separator level k */
  int *lsize = (int *)calloc(nlev, sizeof(int));
  for (int k = 0; k < cnt; ++k) lsize[c->lev[vs[k]]]++;
  int half = (cnt + 1) / 2, cum = 0, ks = 0;
  for (ks = 0; ks < nlev; ++ks) {
    cum += lsize[ks];
    if (cum >= half) break;
  }
  if (ks == nlev - 1) ks = nlev - 2;
  free(lsize);
  /* classify: 0 = A, 1 = B, 2 = S */
  int *A = (int *)malloc(sizeof(int) * cnt), *B = (int *)malloc(sizeof(int) * cnt),
      *S = (int *)malloc(sizeof(int) * cnt);
  int na = 0, nbb = 0, ns = 0;
  for (int k = 0; k < cnt; ++k) {
    int v = vs[k], l = c->lev[v];
    if (l < ks) A[na++] = v;
    else if (l > ks) B[nbb++] = v;
    else {
      int sep = 0;
      for (int p = c->ap[v]; p < c->ap[v + 1]; ++p) {
        int u = c->ai[p];
        if (c->inpart[u] == pst && c->lev[u] == ks + 1) { sep = 1; break; }
      }
      if (sep) S[ns++] = v; else A[na++] = v;
    }
  }
  nd(c, A, na);
  nd(c, B, nbb);
  qsort(S, ns, sizeof(int), cmp_int);
  for (int k = 0; k < ns; ++k) c->perm[c->next_pos++] = S[k];
  free(A);
  free(B);
  free(S);
}

static void nd(nd_ctx *c, int *vs, int cnt) {
  if (cnt == 0) return;
  /* split into connected components ordered by smallest vertex */
  int *rest = (int *)malloc(sizeof(int) * cnt);
  int nrest = cnt;
  memcpy(rest, vs, sizeof(int) * cnt);
  qsort(rest, nrest, sizeof(int), cmp_int);
  while (nrest > 0) {
    int pst = ++c->stamp;
    for (int k = 0; k < nrest; ++k) c->inpart[rest[k]] = pst;
    int nlev;
    int got = bfs(c, rest[0], pst, &nlev);
    int *comp = (int *)malloc(sizeof(int) * got);
    memcpy(comp, c->queue, sizeof(int) * got);
    int vst = c->stamp; /* stamp of that BFS */
    int w = 0;
    for (int k = 0; k < nrest; ++k)
      if (c->vis[rest[k]] != vst) rest[w++] = rest[k];
    nrest = w;
    nd_conn(c, comp, got);
    free(comp);
  }
  free(rest);
}

typedef struct {
  int n, nsuper;
  int *perm, *iperm, *parent, *cc, *sptr;
  int64_t *colptr; /* column structure of L (rows > j), CSC */
  int *rowind;
  int64_t nnz_offdiag;
} osym;

/* ap/ai: symmetric adjacency (no self loops). */
osym *osym_analyze_relaxed(int n, const int *ap, const int *ai, int relax_w, int relax_den) {
  osym *s = (osym *)calloc(1, sizeof(osym));
  s->n = n;
  s->perm = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
  s->iperm = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
  s->parent = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
  s->cc = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
  s->sptr = (int *)malloc(sizeof(int) * (n + 1));
  nd_ctx c;
  c.n = n;
  c.ap = ap;
  c.ai = ai;
  c.perm = s->perm;
  c.inpart = (int *)calloc(n + 1, sizeof(int));
  c.vis = (int *)calloc(n + 1, sizeof(int));
  c.lev = (int *)calloc(n + 1, sizeof(int));
  c.queue = (int *)malloc(sizeof(int) * (n + 1));
  c.stamp = 0;
  c.next_pos = 0;
  int *all = (int *)malloc(sizeof(int) * (n + 1));
  for (int v = 0; v < n; ++v) all[v] = v;
  nd(&c, all, n);
  free(all);
  free(c.inpart);
  free(c.vis);
  free(c.lev);
  free(c.queue);
  for (int k = 0; k < n; ++k) s->iperm[s->perm[k]] = k;

  /* symbolic elimination in the new order */
  int64_t cap = 4 * (int64_t)(ap[n] + n) + 16, used = 0;
  int64_t *start = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
  int *len = (int *)calloc(n + 1, sizeof(int));
  int *buf = (int *)malloc(sizeof(int) * cap);
  int *mark = (int *)malloc(sizeof(int) * (n + 1));
  for (int j = 0; j < n; ++j) mark[j] = -1;
  int *head = (int *)malloc(sizeof(int) * (n + 1)), *nxt = (int *)malloc(sizeof(int) * (n + 1));
  for (int j = 0; j < n; ++j) head[j] = -1;
  int *tmp = (int *)malloc(sizeof(int) * (n + 1));
  for (int j = 0; j < n; ++j) {
    int cnt = 0;
    int v = s->perm[j];
    for (int p = ap[v]; p < ap[v + 1]; ++p) {
      int i = s->iperm[ai[p]];
      if (i > j && mark[i] != j) { mark[i] = j; tmp[cnt++] = i; }
    }
    for (int ch = head[j]; ch >= 0; ch = nxt[ch]) {
      for (int q = 0; q < len[ch]; ++q) {
        int i = buf[start[ch] + q];
        if (i != j && mark[i] != j) { mark[i] = j; tmp[cnt++] = i; }
      }
    }
    qsort(tmp, cnt, sizeof(int), cmp_int);
    if (used + cnt > cap) {
      while (used + cnt > cap) cap *= 2;
      buf = (int *)realloc(buf, sizeof(int) * cap);
    }
    start[j] = used;
    len[j] = cnt;
    memcpy(buf + used, tmp, sizeof(int) * cnt);
    used += cnt;
    s->cc[j] = cnt + 1;
    s->parent[j] = cnt > 0 ? tmp[0] : -1;
    if (cnt > 0) {
      int p = tmp[0];
      nxt[j] = head[p];
      head[p] = j;
    }
  }
  s->colptr = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
  s->rowind = (int *)malloc(sizeof(int) * (used > 0 ? used : 1));
  s->colptr[0] = 0;
  for (int j = 0; j < n; ++j) {
    s->colptr[j + 1] = s->colptr[j] + len[j];
    memcpy(s->rowind + s->colptr[j], buf + start[j], sizeof(int) * len[j]);
  }
  s->nnz_offdiag = used;
  free(start);
  free(len);
  free(buf);
  free(mark);
  free(head);
  free(nxt);
  free(tmp);

  /* supernodes (relaxed, see the header) */
  int ns = 0;
  int64_t nzsum = 0; /* sum of |L_k| (diagonal included) over the current supernode */
  for (int j = 0; j < n; ++j) {
    int join = 0;
    if (j > 0 && s->parent[j - 1] == j) {
      int64_t w = j - s->sptr[ns - 1] + 1; /* width with column j */
      int64_t below = s->cc[j] - 1;        /* |struct(L_j)|: the rows below the panel */
      int64_t entries = w * (w + 1) / 2 + w * below;
      int64_t zeros = entries - (nzsum + s->cc[j]);
      join = w <= SN_MAXW &&
             (w <= relax_w || zeros == 0 || (relax_den > 0 && relax_den * zeros <= entries));
    }
    if (!join) {
      s->sptr[ns++] = j;
      nzsum = 0;
    }
    nzsum += s->cc[j];
  }
  s->sptr[ns] = n;
  s->nsuper = ns;
  return s;
}

osym *osym_analyze(int n, const int *ap, const int *ai) {
  return osym_analyze_relaxed(n, ap, ai, 8, 5);
}

void osym_sizes(const osym *s, int *nsuper, int64_t *nnz_offdiag) {
  *nsuper = s->nsuper;
  *nnz_offdiag = s->nnz_offdiag;
}

void osym_export(const osym *s, int *perm, int *parent, int *cc, int *sptr, int64_t *colptr,
                 int *rowind) {
  int n = s->n;
  if (perm) memcpy(perm, s->perm, sizeof(int) * n);
  if (parent) memcpy(parent, s->parent, sizeof(int) * n);
  if (cc) memcpy(cc, s->cc, sizeof(int) * n);
  if (sptr) memcpy(sptr, s->sptr, sizeof(int) * (s->nsuper + 1));
  if (colptr) memcpy(colptr, s->colptr, sizeof(int64_t) * (n + 1));
  if (rowind) memcpy(rowind, s->rowind, sizeof(int) * s->nnz_offdiag);
}

void osym_free(osym *s) {
  if (!s) return;
  free(s->perm);
  free(s->iperm);
  free(s->parent);
  free(s->cc);
  free(s->sptr);
  free(s->colptr);
  free(s->rowind);
  free(s);
}

/* etree by Liu's definition-free check helper is not provided: the tests compare the
   result of osym_analyze against brute-force boolean elimination written in Python. */
