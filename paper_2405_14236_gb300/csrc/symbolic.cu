// GPU symbolic analysis of the condensed KKT matrix (once per sparsity pattern).
//
// The paper reuses one symbolic analysis across IPM iterations and re-solves (Section 6.1,
// Table 1: the cuDSS analysis, whose ordering runs on the host).  Here every step runs in
// this file's kernels:
//   1. graph of K = pat(W) + pat(J^T J) (per-vertex gather, block sort, unique)
//   2. nested-dissection ordering, one thread block per part, parts of a level in parallel:
//      component split, pseudo-peripheral BFS root, BFS-level separator, minimum degree on
//      parts of <= 64 vertices (bit masks in one warp)
//   3. elimination tree: Liu's path-compressed algorithm, run per nested-dissection node,
//      all nodes of one depth in parallel (their subtrees are disjoint)
//   4. column structures of L: struct(L_j) = adj_>j(j) + sum_children struct(L_c) - {j},
//      columns of one elimination-tree depth in parallel
//   5. supernodes, their row lists, panel offsets, condensation slot maps, level schedule.
// The ordering rule is a project definition (the paper leaves ordering to the solver); an
// independent CPU implementation of the same rule checks this one bit for bit.
#include <algorithm>
#include <climits>
#include <cmath>

#include "internal.cuh"

namespace cipm {

static constexpr int SORT_CAP = 4096;  // ints of shared memory for block sorts

// ---------------------------------------------------------------- small helpers
__global__ void k_fill_i32(int *a, int64_t n, int v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

__global__ void k_rowidx(const int *rowptr, int nrows, int *rowidx) {
  int r = blockIdx.x * blockDim.y + threadIdx.y;
  if (r >= nrows) return;
  for (int p = rowptr[r] + threadIdx.x; p < rowptr[r + 1]; p += blockDim.x) rowidx[p] = r;
}

__global__ void k_count_cols(const int *colind, int nnz, int *cnt) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nnz) atomicAdd(&cnt[colind[p]], 1);
}

__global__ void k_fill_cols(const int *colind, int nnz, const int *ptr, int *fill, int *ent) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nnz) {
    int c = colind[p];
    ent[ptr[c] + atomicAdd(&fill[c], 1)] = p;
  }
}

// Sort every segment ptr[s]..ptr[s+1] of data ascending (segments hold distinct values).
__global__ void k_sort_segments(int *data, const int *ptr, int nseg) {
  __shared__ int smem[SORT_CAP + 1];
  int s = blockIdx.x;
  if (s >= nseg) return;
  int b = ptr[s], len = ptr[s + 1] - b;
  if (len > 1) block_sort_unique(data + b, len, smem, SORT_CAP, INT_MIN);
}

// Transpose of a CSR pattern: for each column, the entry indices in increasing order.
static int build_transpose(const int *colind, int nnz, int ncols, int **ptr_out, int **ent_out,
                           cudaStream_t s) {
  int *cnt, *ptr, *ent, *fill;
  DevTemp t;
  CKR(t.alloc(&cnt, ncols + 1));
  CKR(t.alloc(&fill, ncols + 1));
  CKR(dev_alloc(&ptr, ncols + 1));
  CKR(dev_alloc(&ent, nnz));
  *ptr_out = ptr;
  *ent_out = ent;
  CK(cudaMemsetAsync(cnt, 0, sizeof(int) * (ncols + 1), s));
  CK(cudaMemsetAsync(fill, 0, sizeof(int) * (ncols + 1), s));
  if (nnz > 0) {
    k_count_cols<<<grid_for(nnz, 256), 256, 0, s>>>(colind, nnz, cnt);
    CKL();
  }
  CKR(exclusive_scan_i32(cnt, ptr, ncols, s));
  if (nnz > 0) {
    k_fill_cols<<<grid_for(nnz, 256), 256, 0, s>>>(colind, nnz, ptr, fill, ent);
    CKL();
    k_sort_segments<<<ncols, 128, 0, s>>>(ent, ptr, ncols);
    CKL();
  }
  CK(cudaStreamSynchronize(s));
  return IPM_OK;
}

// ---------------------------------------------------------------- 1. graph of K
__global__ void k_graph_count(int n, const int *JT_ptr, const int *JT_ent, const int *J_rowidx,
                              const int *J_rowptr, const int *W_rowptr, const int *WT_ptr,
                              int *ub) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int c = 0;
  for (int t = JT_ptr[v]; t < JT_ptr[v + 1]; ++t) {
    int r = J_rowidx[JT_ent[t]];
    c += J_rowptr[r + 1] - J_rowptr[r];
  }
  c += W_rowptr[v + 1] - W_rowptr[v] + WT_ptr[v + 1] - WT_ptr[v];
  ub[v] = c;
}

__global__ void k_graph_fill(int n, const int *JT_ptr, const int *JT_ent, const int *J_rowidx,
                             const int *J_rowptr, const int *J_colind, const int *W_rowptr,
                             const int *W_colind, const int *WT_ptr, const int *WT_ent,
                             const int *W_rowidx, const int64_t *cand_ptr, int *cand, int *deg) {
  __shared__ int smem[SORT_CAP + 1];
  int v = blockIdx.x;
  if (v >= n) return;
  int *c = cand + cand_ptr[v];
  int off = 0;
  for (int t = JT_ptr[v]; t < JT_ptr[v + 1]; ++t) {
    int r = J_rowidx[JT_ent[t]];
    int b = J_rowptr[r], len = J_rowptr[r + 1] - b;
    for (int k = threadIdx.x; k < len; k += blockDim.x) c[off + k] = J_colind[b + k];
    off += len;
  }
  {
    int b = W_rowptr[v], len = W_rowptr[v + 1] - b;
    for (int k = threadIdx.x; k < len; k += blockDim.x) c[off + k] = W_colind[b + k];
    off += len;
  }
  {
    int b = WT_ptr[v], len = WT_ptr[v + 1] - b;
    for (int k = threadIdx.x; k < len; k += blockDim.x) c[off + k] = W_rowidx[WT_ent[b + k]];
    off += len;
  }
  int d = block_sort_unique(c, off, smem, SORT_CAP, v);
  if (threadIdx.x == 0) deg[v] = d;
}

__global__ void k_graph_compact(int n, const int64_t *cand_ptr, const int *cand,
                                const int *adj_ptr, int *adj) {
  int v = blockIdx.x;
  if (v >= n) return;
  int len = adj_ptr[v + 1] - adj_ptr[v];
  for (int k = threadIdx.x; k < len; k += blockDim.x) adj[adj_ptr[v] + k] = cand[cand_ptr[v] + k];
}

// ---------------------------------------------------------------- 2. nested dissection
struct NDPart {
  int off, size, start, uid;
};
struct NDNode {
  int start, end, depth, pad;
};

struct NDArgs {
  int n;
  const int *adj_ptr, *adj;
  int *part_of;           // uid of the part holding each unplaced vertex, -1 once placed
  int *levA, *levB;       // BFS levels (two copies for the re-rooting comparison)
  int *qA, *qB;           // BFS queues (a part uses its own [off, off+size) range)
  const int *vcur;        // vertex lists of this round's parts
  int *vnext;             // vertex lists of the next round's parts
  const NDPart *parts;
  NDPart *next_parts;
  int *next_count;
  int *uid_counter;
  NDNode *nodes;
  int *node_count;
  int *perm;
  int depth;
};

__device__ __forceinline__ int block_min_int(int v, int *sred) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sred[w] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    int x = threadIdx.x < (int)(blockDim.x >> 5) ? sred[threadIdx.x] : INT_MAX;
    for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (threadIdx.x == 0) sred[32] = x;
  }
  __syncthreads();
  int r = sred[32];
  __syncthreads();
  return r;
}

// Level-synchronous BFS from root over vertices with part_of == uid; q receives the vertices
// in level order starting at q[qbase]; lev must be -1 on every unvisited part vertex.
// Returns the number of vertices reached; *nlev receives the number of levels.
__device__ int nd_bfs(const NDArgs &A, int uid, int root, int *lev, int *q, int qbase,
                      int *nlev_out, int *s_tail) {
  __syncthreads();
  if (threadIdx.x == 0) {
    lev[root] = 0;
    q[qbase] = root;
    *s_tail = qbase + 1;
  }
  __syncthreads();
  int head = qbase;
  int tail = *s_tail;
  int levels = 0;
  while (head < tail) {
    ++levels;
    for (int i = head + (int)threadIdx.x; i < tail; i += blockDim.x) {
      int v = q[i];
      int lv = lev[v] + 1;
      for (int p = A.adj_ptr[v]; p < A.adj_ptr[v + 1]; ++p) {
        int u = A.adj[p];
        if (A.part_of[u] != uid) continue;
        if (atomicCAS(&lev[u], -1, lv) == -1) q[atomicAdd(s_tail, 1)] = u;
      }
    }
    __syncthreads();
    head = tail;
    tail = *s_tail;
    __syncthreads();
  }
  *nlev_out = levels;
  return tail - qbase;
}

// Minimum degree on a connected part of at most 64 vertices, in warp 0.
__device__ void nd_min_degree(const NDArgs &A, int uid, const int *vs_sorted, int cnt,
                              int start, unsigned long long *adjm) {
  if (threadIdx.x >= 32) return;
  int lane = threadIdx.x;
  for (int li = lane; li < cnt; li += 32) {
    int v = vs_sorted[li];
    unsigned long long msk = 0ull;
    for (int p = A.adj_ptr[v]; p < A.adj_ptr[v + 1]; ++p) {
      int u = A.adj[p];
      if (A.part_of[u] != uid) continue;
      int lo = 0, hi = cnt - 1;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (vs_sorted[mid] < u) lo = mid + 1; else hi = mid;
      }
      msk |= 1ull << lo;
    }
    adjm[li] = msk;
  }
  __syncwarp();
  unsigned long long alive = (cnt == 64) ? ~0ull : ((1ull << cnt) - 1ull);
  for (int step = 0; step < cnt; ++step) {
    unsigned best = 0xffffffffu;
    for (int li = lane; li < cnt; li += 32) {
      if ((alive >> li) & 1ull) {
        unsigned d = (unsigned)__popcll(adjm[li] & alive & ~(1ull << li));
        unsigned key = (d << 8) | (unsigned)li;
        best = min(best, key);
      }
    }
    best = __reduce_min_sync(0xffffffffu, best);
    int k = (int)(best & 0xffu);
    unsigned long long nb = adjm[k] & alive & ~(1ull << k);
    alive &= ~(1ull << k);
    if (lane == 0) A.perm[start + step] = vs_sorted[k];
    __syncwarp();
    for (int li = lane; li < cnt; li += 32)
      if ((nb >> li) & 1ull) adjm[li] |= nb & ~(1ull << li);
    __syncwarp();
  }
}

__global__ void __launch_bounds__(512) k_nd_round(NDArgs A) {
  __shared__ int s_red[33];
  __shared__ int s_tail;
  __shared__ int s_cnt[3];
  __shared__ int s_sorted[CIPM_LEAF];
  __shared__ unsigned long long s_adjm[CIPM_LEAF];
  __shared__ int s_sort[SORT_CAP + 1];
  const NDPart P = A.parts[blockIdx.x];
  const int *vl = A.vcur + P.off;
  const int uid = P.uid;
  int *lev = A.levA, *levo = A.levB;
  int *q = A.qA, *qo = A.qB;
  for (int i = threadIdx.x; i < P.size; i += blockDim.x) {
    lev[vl[i]] = -1;
    levo[vl[i]] = -1;
  }
  int vmin = INT_MAX;
  for (int i = threadIdx.x; i < P.size; i += blockDim.x) vmin = min(vmin, vl[i]);
  int root = block_min_int(vmin, s_red);
  int nlev;
  int got = nd_bfs(A, uid, root, lev, q, P.off, &nlev, &s_tail);

  if (got < P.size) {
    // ---- split into connected components, in increasing order of smallest vertex
    int base = 0;
    while (true) {
      int csize = got;
      int cuid = 0;
      if (threadIdx.x == 0) {
        cuid = atomicAdd(A.uid_counter, 1);
        int slot = atomicAdd(A.next_count, 1);
        A.next_parts[slot] = NDPart{P.off + base, csize, P.start + base, cuid};
        s_red[0] = cuid;
      }
      __syncthreads();
      cuid = s_red[0];
      __syncthreads();
      for (int i = threadIdx.x; i < csize; i += blockDim.x) {
        int v = q[P.off + base + i];
        A.vnext[P.off + base + i] = v;
      }
      base += csize;
      if (base >= P.size) break;
      int vm = INT_MAX;
      for (int i = threadIdx.x; i < P.size; i += blockDim.x) {
        int v = vl[i];
        if (lev[v] == -1) vm = min(vm, v);
      }
      int r2 = block_min_int(vm, s_red);
      got = nd_bfs(A, uid, r2, lev, q, P.off + base, &nlev, &s_tail);
    }
    __syncthreads();
    // relabel after all BFS passes (they test part_of == uid)
    // component k occupies vnext[P.off + base_k, +size_k) and its uid was issued in order;
    // the uid of each vertex is recovered from the part table entries written above.
    return;
  }

  if (P.size <= CIPM_LEAF) {
    // ---- minimum degree leaf
    for (int i = threadIdx.x; i < P.size; i += blockDim.x) s_sorted[i] = vl[i];
    __syncthreads();
    bitonic_asc(s_sorted, P.size);
    nd_min_degree(A, uid, s_sorted, P.size, P.start, s_adjm);
    __syncthreads();
    for (int i = threadIdx.x; i < P.size; i += blockDim.x) A.part_of[vl[i]] = -1;
    if (threadIdx.x == 0) {
      int k = atomicAdd(A.node_count, 1);
      A.nodes[k] = NDNode{P.start, P.start + P.size, A.depth, 0};
    }
    return;
  }

  // ---- pseudo-peripheral root
  for (int it = 0; it < CIPM_REROOT; ++it) {
    int lastl = nlev - 1;
    int cm = INT_MAX;
    for (int i = threadIdx.x; i < P.size; i += blockDim.x) {
      int v = q[P.off + i];
      if (lev[v] == lastl) cm = min(cm, v);
    }
    int cand = block_min_int(cm, s_red);
    for (int i = threadIdx.x; i < P.size; i += blockDim.x) levo[vl[i]] = -1;
    int nlev2;
    nd_bfs(A, uid, cand, levo, qo, P.off, &nlev2, &s_tail);
    if (nlev2 > nlev) {
      int *t = lev; lev = levo; levo = t;
      t = q; q = qo; qo = t;
      nlev = nlev2;
    } else {
      break;
    }
  }
  // ---- separator level k: first level whose cumulative size reaches ceil(size/2)
  int half = (P.size + 1) / 2;
  int ks = lev[q[P.off + half - 1]];
  if (ks == nlev - 1) ks = nlev - 2;
  if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  // classify: 0 = A, 1 = B, 2 = S ; stash class in levo (free now)
  for (int i = threadIdx.x; i < P.size; i += blockDim.x) {
    int v = vl[i];
    int l = lev[v];
    int cls;
    if (l < ks) cls = 0;
    else if (l > ks) cls = 1;
    else {
      cls = 0;
      for (int p = A.adj_ptr[v]; p < A.adj_ptr[v + 1]; ++p) {
        int u = A.adj[p];
        if (A.part_of[u] == uid && lev[u] == ks + 1) { cls = 2; break; }
      }
    }
    levo[v] = cls;
    atomicAdd(&s_cnt[cls], 1);
  }
  __syncthreads();
  int na = s_cnt[0], nbb = s_cnt[1], ns = s_cnt[2];
  __syncthreads();
  if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < P.size; i += blockDim.x) {
    int v = vl[i];
    int cls = levo[v];
    int pos = atomicAdd(&s_cnt[cls], 1);
    int dst = cls == 0 ? pos : (cls == 1 ? na + pos : na + nbb + pos);
    A.vnext[P.off + dst] = v;
  }
  __syncthreads();
  int *sv = A.vnext + P.off + na + nbb;
  block_sort_unique(sv, ns, s_sort, SORT_CAP, -1);
  __syncthreads();
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    A.perm[P.start + na + nbb + i] = sv[i];
  }
  __syncthreads();
  // relabel: new parts A and B get fresh uids, separator vertices are placed
  if (threadIdx.x == 0) {
    int ua = -1, ub = -1;
    if (na > 0) {
      ua = atomicAdd(A.uid_counter, 1);
      A.next_parts[atomicAdd(A.next_count, 1)] = NDPart{P.off, na, P.start, ua};
    }
    if (nbb > 0) {
      ub = atomicAdd(A.uid_counter, 1);
      A.next_parts[atomicAdd(A.next_count, 1)] = NDPart{P.off + na, nbb, P.start + na, ub};
    }
    int k = atomicAdd(A.node_count, 1);
    A.nodes[k] = NDNode{P.start + na + nbb, P.start + P.size, A.depth, 0};
    s_red[0] = ua;
    s_red[1] = ub;
  }
  __syncthreads();
  int ua = s_red[0], ub = s_red[1];
  for (int i = threadIdx.x; i < P.size; i += blockDim.x) {
    int v = A.vnext[P.off + i];
    A.part_of[v] = i < na ? ua : (i < na + nbb ? ub : -1);
  }
}

// Relabel the vertices of every newly created part with its uid (component splits defer
// this so that their BFS passes can still test the old uid).
__global__ void k_nd_relabel(const NDPart *parts, int nparts, const int *vnext, int *part_of) {
  int k = blockIdx.x;
  if (k >= nparts) return;
  NDPart P = parts[k];
  for (int i = threadIdx.x; i < P.size; i += blockDim.x) part_of[vnext[P.off + i]] = P.uid;
}

// ---------------------------------------------------------------- 3. elimination tree
__global__ void k_liu(const NDNode *nodes, int nn, const int *adj_ptr, const int *adj,
                      const int *perm, const int *iperm, int *anc, int *parent) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nn) return;
  NDNode N = nodes[t];
  for (int i = N.start; i < N.end; ++i) {
    int v = perm[i];
    for (int p = adj_ptr[v]; p < adj_ptr[v + 1]; ++p) {
      int k = iperm[adj[p]];
      if (k >= i) continue;
      int r = k;
      while (anc[r] != -1 && anc[r] != i) {
        int nx = anc[r];
        anc[r] = i;
        r = nx;
      }
      if (anc[r] == -1) {
        anc[r] = i;
        parent[r] = i;
      }
    }
  }
}

__global__ void k_iperm(const int *perm, int n, int *iperm) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) iperm[perm[k]] = k;
}

// depth in a forest by pointer jumping (ping-pong buffers)
__global__ void k_depth_init(const int *parent, int n, int *d, int *a) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  a[j] = parent[j];
  d[j] = parent[j] < 0 ? 0 : 1;
}
__global__ void k_depth_step(int n, const int *d, const int *a, int *d2, int *a2, int *changed) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int aj = a[j];
  if (aj >= 0) {
    d2[j] = d[j] + d[aj];
    a2[j] = a[aj];
    *changed = 1;
  } else {
    d2[j] = d[j];
    a2[j] = -1;
  }
}

static int forest_depth(const int *parent, int n, int *depth_out, cudaStream_t s) {
  DevTemp t;
  int *d2, *a, *a2, *changed;
  CKR(t.alloc(&d2, n));
  CKR(t.alloc(&a, n));
  CKR(t.alloc(&a2, n));
  CKR(t.alloc(&changed, 1));
  int *d = depth_out;
  k_depth_init<<<grid_for(n, 256), 256, 0, s>>>(parent, n, d, a);
  CKL();
  for (int it = 0; it < 40; ++it) {
    int h = 0;
    CK(cudaMemsetAsync(changed, 0, sizeof(int), s));
    k_depth_step<<<grid_for(n, 256), 256, 0, s>>>(n, d, a, d2, a2, changed);
    CKL();
    std::swap(d, d2);
    std::swap(a, a2);
    CK(cudaMemcpyAsync(&h, changed, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!h) break;
  }
  if (d != depth_out) {
    CK(cudaMemcpyAsync(depth_out, d, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  return IPM_OK;
}

// bucket items 0..n-1 by key (0..nkeys-1): returns ptr[nkeys+1] and list (order within a
// bucket unspecified)
// (items with a negative key are left out)
__global__ void k_bucket_count(const int *key, int n, int *cnt) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n && key[j] >= 0) atomicAdd(&cnt[key[j]], 1);
}
__global__ void k_bucket_fill(const int *key, int n, const int *ptr, int *fill, int *list) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n && key[j] >= 0) {
    int k = key[j];
    list[ptr[k] + atomicAdd(&fill[k], 1)] = j;
  }
}

// key[j] -> ptr[nkeys+1], list; returns the bucket pointers also on the host if requested
static int bucket(const int *key, int n, int nkeys, int *ptr, int *list, int *scratch,
                  cudaStream_t s) {
  CK(cudaMemsetAsync(scratch, 0, sizeof(int) * (nkeys + 1), s));
  if (n > 0) k_bucket_count<<<grid_for(n, 256), 256, 0, s>>>(key, n, scratch);
  CKL();
  CKR(exclusive_scan_i32(scratch, ptr, nkeys, s));
  CK(cudaMemsetAsync(scratch, 0, sizeof(int) * (nkeys + 1), s));
  if (n > 0) k_bucket_fill<<<grid_for(n, 256), 256, 0, s>>>(key, n, ptr, scratch, list);
  CKL();
  return IPM_OK;
}

__global__ void k_level_key(const int *depth, int n, int maxd, int *key) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) key[j] = maxd - depth[j];
}

// ---------------------------------------------------------------- 4. column structures
__global__ void k_colstruct(const int *cols, int ncols, const int *adj_ptr, const int *adj,
                            const int *perm, const int *iperm, const int *ch_ptr,
                            const int *ch_list, int *cc, int64_t *cstart, int *pool,
                            unsigned long long *pool_top, int64_t pool_cap, int *overflow) {
  __shared__ int smem[SORT_CAP + 1];
  __shared__ long long s_base;
  int b = blockIdx.x;
  if (b >= ncols) return;
  int j = cols[b];
  int v = perm[j];
  if (threadIdx.x == 0) {
    int ub = adj_ptr[v + 1] - adj_ptr[v];
    for (int t = ch_ptr[j]; t < ch_ptr[j + 1]; ++t) ub += cc[ch_list[t]] - 1;
    unsigned long long base = atomicAdd(pool_top, (unsigned long long)ub);
    if ((int64_t)base + ub > pool_cap) {
      *overflow = 1;
      s_base = -1;
    } else {
      s_base = (long long)base;
    }
  }
  __syncthreads();
  if (s_base < 0) {
    if (threadIdx.x == 0) cc[j] = 1;
    return;
  }
  int *c = pool + s_base;
  int off = 0;
  {
    int b0 = adj_ptr[v], len = adj_ptr[v + 1] - b0;
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
      int i = iperm[adj[b0 + k]];
      c[k] = i > j ? i : j;
    }
    off = len;
  }
  for (int t = ch_ptr[j]; t < ch_ptr[j + 1]; ++t) {
    int ch = ch_list[t];
    const int *src = pool + cstart[ch];
    int len = cc[ch] - 1;
    for (int k = threadIdx.x; k < len; k += blockDim.x) c[off + k] = src[k];
    off += len;
  }
  int u = block_sort_unique(c, off, smem, SORT_CAP, j);
  if (threadIdx.x == 0) {
    cc[j] = u + 1;
    cstart[j] = s_base;
  }
}

__global__ void k_cc_minus1(const int *cc, int n, int *out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = cc[j] - 1;
}

__global__ void k_copy_struct(int n, const int64_t *cstart, const int *pool, const int64_t *colptr,
                              int *rowind) {
  int j = blockIdx.x;
  if (j >= n) return;
  int64_t len = colptr[j + 1] - colptr[j];
  for (int64_t k = threadIdx.x; k < len; k += blockDim.x) rowind[colptr[j] + k] = pool[cstart[j] + k];
}

// ---------------------------------------------------------------- 5. supernodes
// Relaxed supernodes: runs of consecutive columns f..l with parent(k) = k+1 (chains of the
// elimination tree), each panel holding rows k..l and struct(L_l) in every column k (explicit
// zeros where struct(L_k) lacks them).  Column j joins the supernode f..j-1 when parent(j-1) = j,
// the width w = j-f+1 is <= CIPM_SN_MAXW, and w <= relax_w, or the panel has no explicit zero, or
// (relax_den > 0) the explicit zeros are at most entries / relax_den (entries = w(w+1)/2 +
// w |struct(L_j)|, zeros = entries - sum |L_k|).  (relax_w, relax_den) = (1, 0) gives the
// fundamental supernodes.  One thread per chain scans it greedily from its first column;
// flag[j] = 1 where a supernode starts (every column belongs to exactly one chain, so every flag
// is written once).
__global__ void k_sn_relaxed(const int *parent, const int *cc, int n, int relax_w, int relax_den,
                             int *flag) {
  const int j0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (j0 >= n || (j0 > 0 && parent[j0 - 1] == j0)) return;  // not the first column of a chain
  int f = j0;
  long long nz = cc[j0];
  flag[j0] = 1;
  for (int j = j0 + 1; j < n && parent[j - 1] == j; ++j) {
    const long long w = j - f + 1, below = cc[j] - 1;
    const long long entries = w * (w + 1) / 2 + w * below;
    const long long zeros = entries - (nz + cc[j]);
    if (w <= CIPM_SN_MAXW &&
        (w <= relax_w || zeros == 0 || (relax_den > 0 && relax_den * zeros <= entries))) {
      flag[j] = 0;
      nz += cc[j];
    } else {
      flag[j] = 1;
      f = j;
      nz = cc[j];
    }
  }
}
__global__ void k_snode(const int *flag, const int *ex, int n, int *snode, int *sptr) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int s = ex[j] + flag[j] - 1;
  snode[j] = s;
  if (flag[j]) sptr[s] = j;
}
__global__ void k_sn_ld(const int *sptr, const int *cc, int ns, int n, int *ld, int64_t *area) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  int f = sptr[s], l = (s + 1 < ns) ? sptr[s + 1] : n;
  int w = l - f;
  int rows = w + cc[l - 1] - 1;
  ld[s] = rows;
  area[s] = (int64_t)rows * w;
}
__global__ void k_sn_rows(const int *sptr, int ns, int n, const int64_t *colptr, const int *rowind,
                          const int *srow_ptr, int *srow) {
  int s = blockIdx.x;
  if (s >= ns) return;
  int f = sptr[s], l = (s + 1 < ns) ? sptr[s + 1] : n;
  int w = l - f;
  int *dst = srow + srow_ptr[s];
  for (int t = threadIdx.x; t < w; t += blockDim.x) dst[t] = f + t;
  int64_t b = colptr[l - 1], len = colptr[l] - b;
  for (int64_t t = threadIdx.x; t < len; t += blockDim.x) dst[w + t] = rowind[b + t];
}
__global__ void k_sn_parent(const int *sptr, int ns, int n, const int *parent, const int *snode,
                            int *sparent) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  int l = (s + 1 < ns) ? sptr[s + 1] : n;
  int p = parent[l - 1];
  sparent[s] = p < 0 ? -1 : snode[p];
}

// ---------------------------------------------------------------- 6. condensation maps
__device__ __forceinline__ int64_t slot_of(int i, int j, const int *snode, const int *sptr,
                                           const int *srow_ptr, const int *srow,
                                           const int64_t *lptr) {
  if (i < j) {
    int t = i; i = j; j = t;
  }
  int s = snode[j];
  int b = srow_ptr[s], ld = srow_ptr[s + 1] - b;
  const int *rows = srow + b;
  int lo = 0, hi = ld - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (rows[mid] < i) lo = mid + 1; else hi = mid;
  }
  return lptr[s] + (int64_t)(j - sptr[s]) * ld + lo;
}

struct MapArgs {
  int m, nnzW;
  const int *J_rowptr, *J_colind, *W_rowidx, *W_colind, *iperm;
  const int *snode, *sptr, *srow_ptr, *srow;
  const int64_t *lptr;
  int *cnt;           // count pass: per-slot counts
  const int *slot_ptr;  // fill pass
  int *fill;
  int2 *items;
};

// one warp per J row: every pair (a >= b) of its entries adds J_a J_b d_r to one slot
template <bool Fill>
__global__ void k_map_j(MapArgs M) {
  int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (r >= M.m) return;
  int b = M.J_rowptr[r], len = M.J_rowptr[r + 1] - b;
  int64_t npair = (int64_t)len * (len + 1) / 2;
  for (int64_t t = lane; t < npair; t += 32) {
    // decode t -> (a, c) with c <= a: a = floor((sqrt(8t+1)-1)/2)
    int a = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)(a + 1) * (a + 2) / 2 <= t) ++a;
    while ((int64_t)a * (a + 1) / 2 > t) --a;
    int c = (int)(t - (int64_t)a * (a + 1) / 2);
    int pa = b + a, pc = b + c;
    int64_t sl = slot_of(M.iperm[M.J_colind[pa]], M.iperm[M.J_colind[pc]], M.snode, M.sptr,
                         M.srow_ptr, M.srow, M.lptr);
    if (!Fill) {
      atomicAdd(&M.cnt[sl], 1);
    } else {
      int pos = M.slot_ptr[sl] + atomicAdd(&M.fill[sl], 1);
      M.items[pos] = make_int2(max(pa, pc), min(pa, pc));
    }
  }
}

template <bool Fill>
__global__ void k_map_w(MapArgs M) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M.nnzW) return;
  int64_t sl = slot_of(M.iperm[M.W_rowidx[e]], M.iperm[M.W_colind[e]], M.snode, M.sptr,
                       M.srow_ptr, M.srow, M.lptr);
  if (!Fill) {
    atomicAdd(&M.cnt[sl], 1);
  } else {
    int pos = M.slot_ptr[sl] + atomicAdd(&M.fill[sl], 1);
    M.items[pos] = make_int2(e, -1);
  }
}

// canonical order inside each slot: sort by (p, q)
__global__ void k_sort_items(const int *slot_ptr, int64_t nslots, int2 *items) {
  int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= nslots) return;
  int b = slot_ptr[sl], e = slot_ptr[sl + 1];
  for (int i = b + 1; i < e; ++i) {
    int2 x = items[i];
    long long kx = ((long long)x.x << 32) | (unsigned)(x.y + 1);
    int k = i - 1;
    while (k >= b) {
      int2 y = items[k];
      long long ky = ((long long)y.x << 32) | (unsigned)(y.y + 1);
      if (ky <= kx) break;
      items[k + 1] = y;
      --k;
    }
    items[k + 1] = x;
  }
}

}  // namespace cipm

using namespace cipm;

static void free_sym(ipm_sym_t S) {
  if (!S) return;
  int *ip[] = {S->J_rowptr, S->J_colind, S->J_rowidx, S->W_rowptr, S->W_colind, S->W_rowidx,
               S->JT_ptr, S->JT_ent, S->WT_ptr, S->WT_ent, S->perm, S->iperm, S->parent, S->cc,
               S->rowind, S->sptr, S->snode, S->srow_ptr, S->srow, S->slot_ptr, S->level_sn};
  for (int *p : ip)
    if (p) cudaFree(p);
  if (S->colptr) cudaFree(S->colptr);
  if (S->lptr) cudaFree(S->lptr);
  if (S->items) cudaFree(S->items);
  if (S->panel_tasks) cudaFree(S->panel_tasks);
  if (S->dptr) cudaFree(S->dptr);
  if (S->ftasks) cudaFree(S->ftasks);
  if (S->upd_need) cudaFree(S->upd_need);
  if (S->fwd_need) cudaFree(S->fwd_need);
  if (S->upd_tasks) cudaFree(S->upd_tasks);
  delete S;
}

static int symbolic_impl(ipm_sym_t S, const int *J_rowptr, const int *J_colind,
                         const int *W_rowptr, const int *W_colind, cudaStream_t s) {
  const int n = S->n, m = S->m, nnzJ = S->nnzJ, nnzW = S->nnzW;
  // ---- copies of the patterns and their transposes
  CKR(dev_alloc(&S->J_rowptr, m + 1));
  CKR(dev_alloc(&S->J_colind, nnzJ));
  CKR(dev_alloc(&S->J_rowidx, nnzJ));
  CKR(dev_alloc(&S->W_rowptr, n + 1));
  CKR(dev_alloc(&S->W_colind, nnzW));
  CKR(dev_alloc(&S->W_rowidx, nnzW));
  CK(cudaMemcpyAsync(S->J_rowptr, J_rowptr, sizeof(int) * (m + 1), cudaMemcpyDefault, s));
  if (nnzJ) CK(cudaMemcpyAsync(S->J_colind, J_colind, sizeof(int) * nnzJ, cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(S->W_rowptr, W_rowptr, sizeof(int) * (n + 1), cudaMemcpyDefault, s));
  if (nnzW) CK(cudaMemcpyAsync(S->W_colind, W_colind, sizeof(int) * nnzW, cudaMemcpyDefault, s));
  {
    dim3 blk(32, 8);
    if (m > 0) k_rowidx<<<grid_for(m, 8), blk, 0, s>>>(S->J_rowptr, m, S->J_rowidx);
    CKL();
    k_rowidx<<<grid_for(n, 8), blk, 0, s>>>(S->W_rowptr, n, S->W_rowidx);
    CKL();
  }
  CKR(build_transpose(S->J_colind, nnzJ, n, &S->JT_ptr, &S->JT_ent, s));
  CKR(build_transpose(S->W_colind, nnzW, n, &S->WT_ptr, &S->WT_ent, s));

  DevTemp T;
  // ---- 1. graph of K
  int *ub, *deg, *adj_ptr, *adj, *cand;
  int64_t *cand_ptr;
  CKR(T.alloc(&ub, n + 1));
  CKR(T.alloc(&deg, n + 1));
  CKR(T.alloc(&cand_ptr, n + 1));
  CKR(T.alloc(&adj_ptr, n + 1));
  k_graph_count<<<grid_for(n, 256), 256, 0, s>>>(n, S->JT_ptr, S->JT_ent, S->J_rowidx,
                                                  S->J_rowptr, S->W_rowptr, S->WT_ptr, ub);
  CKL();
  CKR(exclusive_scan_i32_to_i64(ub, cand_ptr, n, s));
  int64_t ncand = 0;
  CK(cudaMemcpy(&ncand, cand_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost));
  CKR(T.alloc(&cand, ncand));
  k_graph_fill<<<n, 128, 0, s>>>(n, S->JT_ptr, S->JT_ent, S->J_rowidx, S->J_rowptr, S->J_colind,
                                 S->W_rowptr, S->W_colind, S->WT_ptr, S->WT_ent, S->W_rowidx,
                                 cand_ptr, cand, deg);
  CKL();
  CKR(exclusive_scan_i32(deg, adj_ptr, n, s));
  int nadj = 0;
  CK(cudaMemcpy(&nadj, adj_ptr + n, sizeof(int), cudaMemcpyDeviceToHost));
  CKR(T.alloc(&adj, nadj));
  S->nnz_k = (int64_t)nadj / 2 + n;
  k_graph_compact<<<n, 128, 0, s>>>(n, cand_ptr, cand, adj_ptr, adj);
  CKL();

  // ---- 2. nested dissection
  CKR(dev_alloc(&S->perm, n));
  CKR(dev_alloc(&S->iperm, n));
  int *part_of, *levA, *levB, *qA, *qB, *vA, *vB, *cnts;
  NDPart *pA, *pB;
  NDNode *nodes;
  CKR(T.alloc(&part_of, n));
  CKR(T.alloc(&levA, n));
  CKR(T.alloc(&levB, n));
  CKR(T.alloc(&qA, n));
  CKR(T.alloc(&qB, n));
  CKR(T.alloc(&vA, n));
  CKR(T.alloc(&vB, n));
  CKR(T.alloc(&pA, n + 1));
  CKR(T.alloc(&pB, n + 1));
  CKR(T.alloc(&nodes, n + 1));
  CKR(T.alloc(&cnts, 4));  // next_count, uid_counter, node_count
  {
    std::vector<int> iota(n);
    for (int i = 0; i < n; ++i) iota[i] = i;
    CK(cudaMemcpy(vA, iota.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    k_fill_i32<<<grid_for(n, 256), 256, 0, s>>>(part_of, n, 0);
    CKL();
    NDPart p0{0, n, 0, 0};
    CK(cudaMemcpy(pA, &p0, sizeof(NDPart), cudaMemcpyHostToDevice));
    int init[4] = {0, 1, 0, 0};
    CK(cudaMemcpy(cnts, init, sizeof(init), cudaMemcpyHostToDevice));
  }
  int nparts = n > 0 ? 1 : 0;
  int depth = 0;
  while (nparts > 0) {
    CK(cudaMemsetAsync(cnts, 0, sizeof(int), s));  // next_count
    NDArgs A;
    A.n = n;
    A.adj_ptr = adj_ptr;
    A.adj = adj;
    A.part_of = part_of;
    A.levA = levA;
    A.levB = levB;
    A.qA = qA;
    A.qB = qB;
    A.vcur = vA;
    A.vnext = vB;
    A.parts = pA;
    A.next_parts = pB;
    A.next_count = cnts;
    A.uid_counter = cnts + 1;
    A.nodes = nodes;
    A.node_count = cnts + 2;
    A.perm = S->perm;
    A.depth = depth;
    k_nd_round<<<nparts, 512, 0, s>>>(A);
    CKL();
    int nnext = 0;
    CK(cudaMemcpyAsync(&nnext, cnts, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (nnext > 0) {
      k_nd_relabel<<<nnext, 256, 0, s>>>(pB, nnext, vB, part_of);
      CKL();
    }
    std::swap(vA, vB);
    std::swap(pA, pB);
    nparts = nnext;
    ++depth;
    if (depth > 4 * n + 8) {
      set_error_msg("nested dissection did not terminate");
      return IPM_ERR_CUDA;
    }
  }
  k_iperm<<<grid_for(n, 256), 256, 0, s>>>(S->perm, n, S->iperm);
  CKL();

  // ---- 3. elimination tree (Liu), nested-dissection nodes deepest first
  CKR(dev_alloc(&S->parent, n));
  {
    int nn = 0;
    CK(cudaMemcpy(&nn, cnts + 2, sizeof(int), cudaMemcpyDeviceToHost));
    std::vector<NDNode> hn(nn);
    if (nn) CK(cudaMemcpy(hn.data(), nodes, sizeof(NDNode) * nn, cudaMemcpyDeviceToHost));
    std::stable_sort(hn.begin(), hn.end(),
                     [](const NDNode &a, const NDNode &b) { return a.depth > b.depth; });
    if (nn) CK(cudaMemcpy(nodes, hn.data(), sizeof(NDNode) * nn, cudaMemcpyHostToDevice));
    int *anc;
    CKR(T.alloc(&anc, n));
    k_fill_i32<<<grid_for(n, 256), 256, 0, s>>>(anc, n, -1);
    k_fill_i32<<<grid_for(n, 256), 256, 0, s>>>(S->parent, n, -1);
    CKL();
    int b = 0;
    while (b < nn) {
      int e = b;
      while (e < nn && hn[e].depth == hn[b].depth) ++e;
      k_liu<<<grid_for(e - b, 64), 64, 0, s>>>(nodes + b, e - b, adj_ptr, adj, S->perm, S->iperm,
                                               anc, S->parent);
      CKL();
      b = e;
    }
  }

  // ---- 4. column structures by elimination-tree depth, deepest first
  CKR(dev_alloc(&S->cc, n));
  int *dep, *ch_ptr, *ch_list, *lvl_ptr, *lvl_list, *tmpc, *overflow;
  int64_t *cstart;
  CKR(T.alloc(&dep, n));
  CKR(T.alloc(&ch_ptr, n + 1));
  CKR(T.alloc(&ch_list, n));
  CKR(T.alloc(&tmpc, n + 1));
  CKR(T.alloc(&cstart, n + 1));
  CKR(T.alloc(&overflow, 1));
  CKR(forest_depth(S->parent, n, dep, s));
  std::vector<int> hdep(n);
  CK(cudaMemcpy(hdep.data(), dep, sizeof(int) * n, cudaMemcpyDeviceToHost));
  int maxdep = 0;
  for (int j = 0; j < n; ++j) maxdep = std::max(maxdep, hdep[j]);
  CKR(T.alloc(&lvl_ptr, maxdep + 2));
  CKR(T.alloc(&lvl_list, n));
  // children lists (bucket by parent) and columns grouped by depth
  CKR(bucket(S->parent, n, n, ch_ptr, ch_list, tmpc, s));
  CKR(bucket(dep, n, maxdep + 1, lvl_ptr, lvl_list, tmpc, s));
  std::vector<int> hlp(maxdep + 2);
  CK(cudaMemcpy(hlp.data(), lvl_ptr, sizeof(int) * (maxdep + 2), cudaMemcpyDeviceToHost));
  int64_t pool_cap = 4 * ((int64_t)nadj + n) + 1024;
  int *pool = nullptr;
  unsigned long long *pool_top;
  CKR(T.alloc(&pool_top, 1));
  for (int attempt = 0; attempt < 8; ++attempt) {
    if (pool) cudaFree(pool);
    CKR(dev_alloc(&pool, pool_cap));
    CK(cudaMemsetAsync(pool_top, 0, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(overflow, 0, sizeof(int), s));
    for (int d = maxdep; d >= 0; --d) {
      int b = hlp[d], e = hlp[d + 1];
      if (e <= b) continue;
      k_colstruct<<<e - b, 128, 0, s>>>(lvl_list + b, e - b, adj_ptr, adj, S->perm, S->iperm,
                                        ch_ptr, ch_list, S->cc, cstart, pool, pool_top, pool_cap,
                                        overflow);
      CKL();
    }
    int ovf = 0;
    CK(cudaMemcpy(&ovf, overflow, sizeof(int), cudaMemcpyDeviceToHost));
    if (!ovf) break;
    pool_cap *= 4;
    if (attempt == 7) {
      cudaFree(pool);
      set_error_msg("column-structure pool overflow");
      return IPM_ERR_OOM;
    }
  }
  CKR(dev_alloc(&S->colptr, n + 1));
  k_cc_minus1<<<grid_for(n, 256), 256, 0, s>>>(S->cc, n, tmpc);
  CKL();
  CKR(exclusive_scan_i32_to_i64(tmpc, S->colptr, n, s));
  CK(cudaMemcpy(&S->nnz_offdiag, S->colptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost));
  CKR(dev_alloc(&S->rowind, S->nnz_offdiag));
  if (n) k_copy_struct<<<n, 128, 0, s>>>(n, cstart, pool, S->colptr, S->rowind);
  CKL();
  CK(cudaStreamSynchronize(s));
  cudaFree(pool);

  // ---- 5. supernodes
  int *flag, *ex, *ld, *sparent, *sdep;
  int64_t *area;
  CKR(T.alloc(&flag, n + 1));
  CKR(T.alloc(&ex, n + 1));
  k_sn_relaxed<<<grid_for(n, 256), 256, 0, s>>>(S->parent, S->cc, n, S->relax_w, S->relax_den,
                                                 flag);
  CKL();
  CKR(exclusive_scan_i32(flag, ex, n, s));
  CK(cudaMemcpy(&S->nsuper, ex + n, sizeof(int), cudaMemcpyDeviceToHost));
  const int ns = S->nsuper;
  CKR(dev_alloc(&S->sptr, ns + 1));
  CKR(dev_alloc(&S->snode, n));
  k_snode<<<grid_for(n, 256), 256, 0, s>>>(flag, ex, n, S->snode, S->sptr);
  CKL();
  CK(cudaMemcpy(S->sptr + ns, &n, sizeof(int), cudaMemcpyHostToDevice));
  CKR(T.alloc(&ld, ns + 1));
  CKR(T.alloc(&area, ns + 1));
  k_sn_ld<<<grid_for(ns, 256), 256, 0, s>>>(S->sptr, S->cc, ns, n, ld, area);
  CKL();
  CKR(dev_alloc(&S->srow_ptr, ns + 1));
  CKR(exclusive_scan_i32(ld, S->srow_ptr, ns, s));
  CKR(dev_alloc(&S->lptr, ns + 1));
  CKR(exclusive_scan_i64(area, S->lptr, ns, s));
  int nsrow = 0;
  CK(cudaMemcpy(&nsrow, S->srow_ptr + ns, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&S->panel_len, S->lptr + ns, sizeof(int64_t), cudaMemcpyDeviceToHost));
  CKR(dev_alloc(&S->srow, nsrow));
  k_sn_rows<<<ns, 128, 0, s>>>(S->sptr, ns, n, S->colptr, S->rowind, S->srow_ptr, S->srow);
  CKL();
  // supernodal tree levels
  CKR(T.alloc(&sparent, ns + 1));
  CKR(T.alloc(&sdep, ns + 1));
  k_sn_parent<<<grid_for(ns, 256), 256, 0, s>>>(S->sptr, ns, n, S->parent, S->snode, sparent);
  CKL();
  CKR(forest_depth(sparent, ns, sdep, s));
  {
    // levels of the supernodal tree, deepest first (level L = maxdepth - depth)
    std::vector<int> hsd(ns), hld(ns), hsp(ns + 1);
    CK(cudaMemcpy(hsd.data(), sdep, sizeof(int) * ns, cudaMemcpyDeviceToHost));
    int md = 0;
    for (int k = 0; k < ns; ++k) md = std::max(md, hsd[k]);
    S->nlevels = ns > 0 ? md + 1 : 0;
    int *lkey, *lptr_d, *lscr;
    CKR(T.alloc(&lkey, ns + 1));
    CKR(T.alloc(&lptr_d, md + 2));
    CKR(T.alloc(&lscr, md + 2));
    CKR(dev_alloc(&S->level_sn, ns));
    k_level_key<<<grid_for(ns, 256), 256, 0, s>>>(sdep, ns, md, lkey);
    CKL();
    CKR(bucket(lkey, ns, md + 1, lptr_d, S->level_sn, lscr, s));
    S->h_level_ptr.assign(S->nlevels + 1, 0);
    CK(cudaMemcpy(S->h_level_ptr.data(), lptr_d, sizeof(int) * (S->nlevels + 1),
                  cudaMemcpyDeviceToHost));
    // launch-shape bookkeeping: widest panel of each level
    CK(cudaMemcpy(hld.data(), ld, sizeof(int) * ns, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hsp.data(), S->sptr, sizeof(int) * (ns + 1), cudaMemcpyDeviceToHost));
    S->h_level_maxld.assign(S->nlevels, 0);
    S->h_level_maxw.assign(S->nlevels, 0);
    for (int k = 0; k < ns; ++k) {
      int L = md - hsd[k];
      S->h_level_maxld[L] = std::max(S->h_level_maxld[L], hld[k]);
      S->h_level_maxw[L] = std::max(S->h_level_maxw[L], hsp[k + 1] - hsp[k]);
      S->max_ld = std::max(S->max_ld, hld[k]);
      S->max_w = std::max(S->max_w, hsp[k + 1] - hsp[k]);
    }
    // factorization task lists (launch shapes of the numeric phase)
    std::vector<int> hlsn(ns);
    if (ns) CK(cudaMemcpy(hlsn.data(), S->level_sn, sizeof(int) * ns, cudaMemcpyDeviceToHost));
    std::vector<int4> pt, ut;
    S->h_panel_ptr.assign(S->nlevels + 1, 0);
    S->h_upd_ptr.assign(S->nlevels + 1, 0);
    for (int L = 0; L < S->nlevels; ++L) {
      S->h_panel_ptr[L] = (int)pt.size();
      S->h_upd_ptr[L] = (int)ut.size();
      for (int q = S->h_level_ptr[L]; q < S->h_level_ptr[L + 1]; ++q) {
        int sn = hlsn[q];
        int w = hsp[sn + 1] - hsp[sn];
        int B = hld[sn] - w;
        int T = B > 0 ? (B + CIPM_RB - 1) / CIPM_RB : 1;
        for (int rb = 0; rb < T; ++rb) pt.push_back(make_int4(sn, rb, 0, 0));
        if (B > 0)
          for (int ti = 0; ti < T; ++ti)
            for (int tj = 0; tj <= ti; ++tj) ut.push_back(make_int4(sn, ti, tj, 0));
      }
    }
    S->h_panel_ptr[S->nlevels] = (int)pt.size();
    // one topological order for the sync-free factorization: per level, its panel tasks then
    // its update tasks; dependency counts from the row structure (rows are sorted, so the
    // target supernodes of a row range appear in increasing runs)
    {
      std::vector<int> hsrp(ns + 1), hsrow(nsrow), hsn(n);
      CK(cudaMemcpy(hsrp.data(), S->srow_ptr, sizeof(int) * (ns + 1), cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(hsrow.data(), S->srow, sizeof(int) * nsrow, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(hsn.data(), S->snode, sizeof(int) * n, cudaMemcpyDeviceToHost));
      std::vector<int4> ft;
      std::vector<int> updn(ns, 0), fwdn(ns, 0);
      for (int L = 0; L < S->nlevels; ++L) {
        for (int q = S->h_level_ptr[L]; q < S->h_level_ptr[L + 1]; ++q) {
          int sn = hlsn[q];
          int w = hsp[sn + 1] - hsp[sn];
          int B = hld[sn] - w;
          int T = B > 0 ? (B + CIPM_RB - 1) / CIPM_RB : 1;
          for (int rb = 0; rb < T; ++rb) ft.push_back(make_int4(sn, rb, 0, 0));
          int last = -1;
          for (int i = w; i < w + B; ++i) {
            int t = hsn[hsrow[hsrp[sn] + i]];
            if (t != last) fwdn[t]++;
            last = t;
          }
        }
        for (int q = S->h_level_ptr[L]; q < S->h_level_ptr[L + 1]; ++q) {
          int sn = hlsn[q];
          int w = hsp[sn + 1] - hsp[sn];
          int B = hld[sn] - w;
          if (B <= 0) continue;
          int T = (B + CIPM_RB - 1) / CIPM_RB;
          for (int ti = 0; ti < T; ++ti)
            for (int tj = 0; tj <= ti; ++tj) {
              ft.push_back(make_int4(sn, ti, tj, 1));
              int j0 = w + tj * CIPM_RB, j1 = std::min(w + B, j0 + CIPM_RB);
              int last = -1;
              for (int j = j0; j < j1; ++j) {
                int t = hsn[hsrow[hsrp[sn] + j]];
                if (t != last) updn[t]++;
                last = t;
              }
            }
        }
      }
      S->nftasks = (int)ft.size();
      CKR(dev_alloc(&S->ftasks, (int64_t)ft.size()));
      CKR(dev_alloc(&S->upd_need, ns));
      CKR(dev_alloc(&S->fwd_need, ns));
      if (!ft.empty())
        CK(cudaMemcpy(S->ftasks, ft.data(), sizeof(int4) * ft.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(S->upd_need, updn.data(), sizeof(int) * ns, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(S->fwd_need, fwdn.data(), sizeof(int) * ns, cudaMemcpyHostToDevice));
    }
    S->h_upd_ptr[S->nlevels] = (int)ut.size();
    std::vector<int64_t> hdp(ns + 1, 0);
    for (int k = 0; k < ns; ++k) {
      int64_t w = hsp[k + 1] - hsp[k];
      hdp[k + 1] = hdp[k] + w * w + w;  // L11 (column-major) then its reciprocal diagonal
    }
    S->diag_len = hdp[ns];
    CKR(dev_alloc(&S->dptr, ns + 1));
    CK(cudaMemcpy(S->dptr, hdp.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice));
    CKR(dev_alloc(&S->panel_tasks, (int64_t)pt.size()));
    CKR(dev_alloc(&S->upd_tasks, (int64_t)ut.size()));
    if (!pt.empty())
      CK(cudaMemcpy(S->panel_tasks, pt.data(), sizeof(int4) * pt.size(), cudaMemcpyHostToDevice));
    if (!ut.empty())
      CK(cudaMemcpy(S->upd_tasks, ut.data(), sizeof(int4) * ut.size(), cudaMemcpyHostToDevice));
    std::vector<int> hcc(n);
    CK(cudaMemcpy(hcc.data(), S->cc, sizeof(int) * n, cudaMemcpyDeviceToHost));
    double fl = 0;
    for (int j = 0; j < n; ++j) fl += (double)(hcc[j] - 1) * (double)(hcc[j] + 2);
    S->flops = fl;
  }

  // ---- 6. condensation slot maps
  {
    int *cnt, *fillc;
    CKR(T.alloc(&cnt, S->panel_len + 1));
    CKR(T.alloc(&fillc, S->panel_len + 1));
    CK(cudaMemsetAsync(cnt, 0, sizeof(int) * (S->panel_len + 1), s));
    MapArgs M;
    M.m = m;
    M.nnzW = nnzW;
    M.J_rowptr = S->J_rowptr;
    M.J_colind = S->J_colind;
    M.W_rowidx = S->W_rowidx;
    M.W_colind = S->W_colind;
    M.iperm = S->iperm;
    M.snode = S->snode;
    M.sptr = S->sptr;
    M.srow_ptr = S->srow_ptr;
    M.srow = S->srow;
    M.lptr = S->lptr;
    M.cnt = cnt;
    M.slot_ptr = nullptr;
    M.fill = fillc;
    M.items = nullptr;
    if (m > 0) k_map_j<false><<<grid_for(m, 8), 256, 0, s>>>(M);
    CKL();
    if (nnzW > 0) k_map_w<false><<<grid_for(nnzW, 256), 256, 0, s>>>(M);
    CKL();
    CKR(dev_alloc(&S->slot_ptr, S->panel_len + 1));
    CKR(exclusive_scan_i32(cnt, S->slot_ptr, S->panel_len, s));
    int nit = 0;
    CK(cudaMemcpy(&nit, S->slot_ptr + S->panel_len, sizeof(int), cudaMemcpyDeviceToHost));
    S->nitems = nit;
    CKR(dev_alloc(&S->items, nit));
    CK(cudaMemsetAsync(fillc, 0, sizeof(int) * (S->panel_len + 1), s));
    M.slot_ptr = S->slot_ptr;
    M.items = S->items;
    if (m > 0) k_map_j<true><<<grid_for(m, 8), 256, 0, s>>>(M);
    CKL();
    if (nnzW > 0) k_map_w<true><<<grid_for(nnzW, 256), 256, 0, s>>>(M);
    CKL();
    k_sort_items<<<grid_for(S->panel_len, 256), 256, 0, s>>>(S->slot_ptr, S->panel_len, S->items);
    CKL();
  }
  CK(cudaStreamSynchronize(s));
  return IPM_OK;
}

extern "C" int ipm_symbolic(int n, int m, const int *J_rowptr, const int *J_colind, int nnzJ,
                            const int *W_rowptr, const int *W_colind, int nnzW,
                            cudaStream_t stream, ipm_sym_t *out) {
  return ipm_symbolic_relaxed(n, m, J_rowptr, J_colind, nnzJ, W_rowptr, W_colind, nnzW, 8, 5,
                              stream, out);
}

extern "C" int ipm_symbolic_relaxed(int n, int m, const int *J_rowptr, const int *J_colind,
                                    int nnzJ, const int *W_rowptr, const int *W_colind, int nnzW,
                                    int relax_w, int relax_den, cudaStream_t stream,
                                    ipm_sym_t *out) {
  NvtxRange nvtx_range("ipm_symbolic");
  if (!out || n <= 0 || m < 0 || nnzJ < 0 || nnzW < 0 || !J_rowptr || !W_rowptr ||
      (nnzJ > 0 && !J_colind) || (nnzW > 0 && !W_colind) || relax_w < 1 ||
      relax_w > CIPM_SN_MAXW || relax_den < 0) {
    set_error_msg("ipm_symbolic: bad argument");
    return IPM_ERR_BAD_ARG;
  }
  *out = nullptr;
  stream = setup_stream(stream);
  ipm_sym_t S = new ipm_sym_s();
  S->relax_w = relax_w;
  S->relax_den = relax_den;
  S->n = n;
  S->m = m;
  S->nnzJ = nnzJ;
  S->nnzW = nnzW;
  int rc = symbolic_impl(S, J_rowptr, J_colind, W_rowptr, W_colind, stream);
  if (cudaStreamSynchronize(stream) != cudaSuccess && rc == IPM_OK) rc = IPM_ERR_CUDA;
  if (rc != IPM_OK) {
    free_sym(S);
    return rc;
  }
  *out = S;
  return IPM_OK;
}

extern "C" int ipm_symbolic_info(ipm_sym_t S, int64_t *nnz_k, int *nsuper, int64_t *nnz_offdiag,
                                 int64_t *panel_len, int *nlevels, double *flops) {
  if (!S) return IPM_ERR_BAD_ARG;
  if (nnz_k) *nnz_k = S->nnz_k;
  if (nsuper) *nsuper = S->nsuper;
  if (nnz_offdiag) *nnz_offdiag = S->nnz_offdiag;
  if (panel_len) *panel_len = S->panel_len;
  if (nlevels) *nlevels = S->nlevels;
  if (flops) *flops = S->flops;
  return IPM_OK;
}

extern "C" int ipm_symbolic_export(ipm_sym_t S, int *perm, int *parent, int *sptr,
                                   int64_t *colptr, int *rowind) {
  if (!S) return IPM_ERR_BAD_ARG;
  int n = S->n;
  if (perm) CK(cudaMemcpy(perm, S->perm, sizeof(int) * n, cudaMemcpyDeviceToHost));
  if (parent) CK(cudaMemcpy(parent, S->parent, sizeof(int) * n, cudaMemcpyDeviceToHost));
  if (sptr) CK(cudaMemcpy(sptr, S->sptr, sizeof(int) * (S->nsuper + 1), cudaMemcpyDeviceToHost));
  if (colptr) CK(cudaMemcpy(colptr, S->colptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost));
  if (rowind && S->nnz_offdiag)
    CK(cudaMemcpy(rowind, S->rowind, sizeof(int) * S->nnz_offdiag, cudaMemcpyDeviceToHost));
  return IPM_OK;
}

extern "C" int ipm_symbolic_export_panels(ipm_sym_t S, int *srow_ptr, int *srow, int64_t *lptr) {
  if (!S) return IPM_ERR_BAD_ARG;
  int ns = S->nsuper;
  int nsrow = 0;
  CK(cudaMemcpy(&nsrow, S->srow_ptr + ns, sizeof(int), cudaMemcpyDeviceToHost));
  if (srow_ptr) CK(cudaMemcpy(srow_ptr, S->srow_ptr, sizeof(int) * (ns + 1), cudaMemcpyDeviceToHost));
  if (srow && nsrow) CK(cudaMemcpy(srow, S->srow, sizeof(int) * nsrow, cudaMemcpyDeviceToHost));
  if (lptr) CK(cudaMemcpy(lptr, S->lptr, sizeof(int64_t) * (ns + 1), cudaMemcpyDeviceToHost));
  return IPM_OK;
}

extern "C" void ipm_symbolic_destroy(ipm_sym_t S) { free_sym(S); }
