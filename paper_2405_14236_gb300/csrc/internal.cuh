// Library-internal layout of the symbolic and numeric handles.
#pragma once
#include "common.cuh"

// Project-defined ordering parameters (kept equal to the CPU checker's constants).
#define CIPM_LEAF 64     // parts of at most this many vertices are ordered by minimum degree
#define CIPM_REROOT 4    // pseudo-peripheral root search: at most this many re-roots
#define CIPM_SN_MAXW 64  // maximum supernode width

struct ipm_sym_s {
  int n = 0, m = 0, nnzJ = 0, nnzW = 0;
  int relax_w = 8, relax_den = 5;  // relaxed-supernode rule (ipm_symbolic_relaxed)
  // copies of the caller's patterns
  int *J_rowptr = nullptr, *J_colind = nullptr, *J_rowidx = nullptr;
  int *W_rowptr = nullptr, *W_colind = nullptr, *W_rowidx = nullptr;
  int *JT_ptr = nullptr, *JT_ent = nullptr;  // column j of J: J entry indices, by row
  int *WT_ptr = nullptr, *WT_ent = nullptr;  // column j of lower W: W entry indices
  // ordering and elimination tree (positions)
  int *perm = nullptr, *iperm = nullptr, *parent = nullptr, *cc = nullptr;
  int64_t *colptr = nullptr;
  int *rowind = nullptr;
  int64_t nnz_offdiag = 0;
  // supernodes
  int nsuper = 0;
  int *sptr = nullptr, *snode = nullptr;
  int *srow_ptr = nullptr, *srow = nullptr;  // rows of each supernode (own columns first)
  int64_t *lptr = nullptr;                   // panel offsets (column-major, ld = rows)
  int64_t panel_len = 0;
  int max_ld = 0, max_w = 0;
  // condensation: items per panel slot (p, q): J entries p, q (q >= 0) or W entry p (q = -1)
  int *slot_ptr = nullptr;
  int2 *items = nullptr;
  int64_t nitems = 0;
  // level schedule of the supernodal elimination tree, deepest level first
  int nlevels = 0;
  int *level_sn = nullptr;             // supernodes grouped by level
  std::vector<int> h_level_ptr;        // host copy, nlevels + 1 entries
  std::vector<int> h_level_maxld;      // max panel rows in each level
  std::vector<int> h_level_maxw;       // max supernode width in each level
  double flops = 0.0;
  int64_t nnz_k = 0;  // structural entries of tril(K)
  // factorization task lists per level: panel tasks (supernode, row block) and update tasks
  // (supernode, row block i, row block j <= i) of the rows below the diagonal block
  int4 *panel_tasks = nullptr, *upd_tasks = nullptr;
  int64_t *dptr = nullptr;  // offsets of the diagonal factors: w x w L11, then 1 / diag(L11)
  int64_t diag_len = 0;
  // sync-free schedule: all factorization tasks in one topological order (x = supernode,
  // y/z = row blocks, w = 0 panel / 1 update), dependency counts per supernode
  int4 *ftasks = nullptr;
  int nftasks = 0;
  int *upd_need = nullptr;  // update tasks that scatter into each supernode
  int *fwd_need = nullptr;  // supernodes whose rows below the diagonal reach each supernode
  std::vector<int> h_panel_ptr, h_upd_ptr;  // per level, nlevels + 1 entries
};

#define CIPM_RB 32  // rows per block of the below-diagonal part of a panel

struct ipm_num_s {
  ipm_sym_t sym = nullptr;
  int precision = 64;
  void *Lx = nullptr;  // panel values (double or float, by precision)
  void *Dx = nullptr;  // diagonal factors L11 + reciprocal pivots of every supernode
  void *tJ = nullptr;     // d_row(p) J_p per J entry (condensation workspace)
  // values of the last ipm_condense (caller-owned): the FP32 path multiplies by K in FP64
  const double *cW = nullptr, *cSig = nullptr, *cJ = nullptr, *cD = nullptr;
  double cDw = 0.0;
  int last_pcg_iters = 0;
  double last_eta = 0.0;  // backward error of the last hykkt_cg solve on the augmented system
  bool factored = false;  // panels hold L21 and Dx holds L11 (else panels hold K)
  // dependency counters of the sync-free kernels: [0,ns) update arrivals, [ns,2ns) panel
  // tasks done, [2ns,3ns) forward arrivals, [3ns,4ns) backward done flags, then tickets/status
  int *sync = nullptr;
  // workspaces (n or m sized), allocated once
  double *vn[12] = {nullptr};
  double *vm[8] = {nullptr};
  double *scal = nullptr;  // device scalars
  double *h_scal = nullptr;  // pinned host mirror
};

// the batched kernels (batch.cu) keep their own copy of the device spin limit
int batch_set_spin_limit(long long polls);
