// Device side of the AC-OPF model evaluation (per branch end, per generator), shared by the
// single-problem kernels (opf.cu) and the batched ones (batch.cu).
//
// Compact form (0): x = [V (nb) | theta (nb) | Pg (ng) | Qg (ng)];
// g = [P balance (nb) | Q balance (nb) | theta_ref]; h = [|S_from|^2 - rate^2 | |S_to|^2 - rate^2].
// Flow-variable form (1): x adds p_end (2 nbr) | q_end (2 nbr) (ends: from ends, then to ends),
// g = [P balance with -p_end | Q balance with -q_end | theta_ref | p_end - P_end(V, theta) |
// q_end - Q_end(V, theta)], h = [p_end^2 + q_end^2 - rate^2].
// Branch pi-model: series 1/(r + j x), shunt j b/2 per end, unit tap.  Cost on MW (base 100).
#pragma once
#include "opf.cuh"

namespace cipm {

static constexpr double BASE = 100.0;

struct OpfDims {
  int nb, nbr, ng, n, me, mi;
  int form;
};

// per-end term counts and offsets of the two forms (J: 12 or 14 terms per end after 2 per
// generator; W: 10 or 12 per end after 1 per generator)
__host__ __device__ __forceinline__ int jterms_per_end(const OpfDims &D) { return D.form ? 14 : 12; }
__host__ __device__ __forceinline__ int wterms_per_end(const OpfDims &D) { return D.form ? 12 : 10; }
__host__ __device__ __forceinline__ int flow_pvar(const OpfDims &D, int e) {
  return 2 * D.nb + 2 * D.ng + e;
}
__host__ __device__ __forceinline__ int flow_qvar(const OpfDims &D, int e) {
  return 2 * D.nb + 2 * D.ng + 2 * D.nbr + e;
}
__host__ __device__ __forceinline__ int flow_prow(const OpfDims &D, int e) { return 2 * D.nb + 1 + e; }
__host__ __device__ __forceinline__ int flow_qrow(const OpfDims &D, int e) {
  return 2 * D.nb + 1 + 2 * D.nbr + e;
}

__device__ __forceinline__ void end_vars(const OpfDims &D, const int *f_bus, const int *t_bus,
                                         int e, int *bus, int *vars) {
  int k = e % D.nbr;
  bool to = e >= D.nbr;
  int a = to ? t_bus[k] : f_bus[k], b = to ? f_bus[k] : t_bus[k];
  *bus = a;
  vars[0] = a;           // Va
  vars[1] = b;           // Vb
  vars[2] = D.nb + a;    // theta_a
  vars[3] = D.nb + b;    // theta_b
}

// lower-triangle pairs of the 4 x 4 Hessian block of a branch end (variables of end_vars)
static __device__ __constant__ int c_lowpairs[10][2] = {{0, 0}, {1, 0}, {1, 1}, {2, 0}, {2, 1},
                                                        {2, 2}, {3, 0}, {3, 1}, {3, 2}, {3, 3}};

__device__ __forceinline__ void block_sum_to(double *out, double v, double *sh) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double u = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    u = warp_sum(u);
    if (threadIdx.x == 0) *out = u;
  }
}

// g = -load on the balance rows, theta_ref row; zero J and W values (grid-stride from i)
__device__ __forceinline__ void eval_init_at(const OpfDims &D, const double *pd,
                                             const double *qd, const double *x, int ref,
                                             double *g, double *Jv, int nnzJ, double *Wv,
                                             int nnzW, int i, int stride) {
  for (int k = i; k < D.nb; k += stride) {
    g[k] = -pd[k];
    g[D.nb + k] = -qd[k];
  }
  if (i == 0) g[2 * D.nb] = x[D.nb + ref];
  if (Jv)
    for (int p = i; p < nnzJ; p += stride) Jv[p] = 0.0;
  if (Wv)
    for (int p = i; p < nnzW; p += stride) Wv[p] = 0.0;
}

// flow leaving bus a on branch end e and its derivatives / second derivatives in the local
// variable order (Va, Vb, theta_a, theta_b); lower-triangle second derivatives follow c_lowpairs
struct EndFlow {
  int bus, v[4];
  double P, Q, dP[4], dQ[4], hP[10], hQ[10];
};
__device__ __forceinline__ void end_flow_at(const OpfDims &D, const OpfData &M, const double *x,
                                            int e, EndFlow &F) {
  const int k = e % D.nbr;
  end_vars(D, M.f_bus, M.t_bus, e, &F.bus, F.v);
  double4_32a ad = M.adm[k];
  const double G1 = ad.x, B1 = ad.y, G2 = ad.z, B2 = ad.w;
  const double Va = x[F.v[0]], Vb = x[F.v[1]], ta = x[F.v[2]], tb = x[F.v[3]];
  double sn, cs;
  sincos(ta - tb, &sn, &cs);
  const double A = G2 * cs + B2 * sn, Bq = G2 * sn - B2 * cs;
  F.P = G1 * Va * Va + Va * Vb * A;
  F.Q = -B1 * Va * Va + Va * Vb * Bq;
  const double dP[4] = {2 * G1 * Va + Vb * A, Va * A, -Va * Vb * Bq, Va * Vb * Bq};
  const double dQ[4] = {-2 * B1 * Va + Vb * Bq, Va * Bq, Va * Vb * A, -Va * Vb * A};
  const double hP[10] = {2 * G1, A, 0.0, -Vb * Bq, -Va * Bq, -Va * Vb * A, Vb * Bq, Va * Bq,
                         Va * Vb * A, -Va * Vb * A};
  const double hQ[10] = {-2 * B1, Bq, 0.0, Vb * A, Va * A, -Va * Vb * Bq, -Vb * A, -Va * A,
                         Va * Vb * Bq, -Va * Vb * Bq};
  for (int c = 0; c < 4; ++c) {
    F.dP[c] = dP[c];
    F.dQ[c] = dQ[c];
  }
  for (int t = 0; t < 10; ++t) {
    F.hP[t] = hP[t];
    F.hQ[t] = hQ[t];
  }
}

// flow-variable form, branch end e (term order per end: balance P, balance Q, p definition
// (p_end, Va, Vb, theta_a, theta_b), q definition (q_end, ...), thermal (p_end, q_end); W: the 10
// lower pairs of the definition rows, then (p_end, p_end), (q_end, q_end))
__device__ __forceinline__ void eval_branch_flow_at(const OpfDims &D, const OpfData &M,
                                                    const double *x, const double *y,
                                                    const double *z, double *g, double *h,
                                                    double *Jv, double *Wv, int e) {
  EndFlow F;
  end_flow_at(D, M, x, e, F);
  const int pv = flow_pvar(D, e), qv = flow_qvar(D, e);
  const double p = x[pv], q = x[qv];
  atomicAdd(&g[F.bus], -p);
  atomicAdd(&g[D.nb + F.bus], -q);
  g[flow_prow(D, e)] = p - F.P;
  g[flow_qrow(D, e)] = q - F.Q;
  const double rt = M.rate[e % D.nbr];
  h[e] = p * p + q * q - rt * rt;
  if (Jv) {
    const int *je = M.jentry + 2 * D.ng + 14 * e;
    Jv[je[0]] = -1.0;
    Jv[je[1]] = -1.0;
    Jv[je[2]] = 1.0;
    Jv[je[7]] = 1.0;
    for (int c = 0; c < 4; ++c) {
      Jv[je[3 + c]] = -F.dP[c];
      Jv[je[8 + c]] = -F.dQ[c];
    }
    Jv[je[12]] = 2 * p;
    Jv[je[13]] = 2 * q;
  }
  if (Wv) {
    const double yp = y[flow_prow(D, e)], yq = y[flow_qrow(D, e)], zz = z[e];
    const int *we = M.wentry + D.ng + 12 * e;
    for (int t = 0; t < 10; ++t) atomicAdd(&Wv[we[t]], -yp * F.hP[t] - yq * F.hQ[t]);
    Wv[we[10]] = 2 * zz;
    Wv[we[11]] = 2 * zz;
  }
}

// branch end e: flows into the balance rows, thermal row, their derivatives, and the weighted
// second derivatives (y on the balance rows, z on the thermal row) into W
__device__ __forceinline__ void eval_branch_at(const OpfDims &D, const OpfData &M,
                                               const double *x, const double *y, const double *z,
                                               double *g, double *h, double *Jv, double *Wv,
                                               int e) {
  if (D.form) {
    eval_branch_flow_at(D, M, x, y, z, g, h, Jv, Wv, e);
    return;
  }
  int k = e % D.nbr;
  int bus, v[4];
  end_vars(D, M.f_bus, M.t_bus, e, &bus, v);
  double4_32a ad = M.adm[k];
  const double G1 = ad.x, B1 = ad.y, G2 = ad.z, B2 = ad.w;
  const double Va = x[v[0]], Vb = x[v[1]], ta = x[v[2]], tb = x[v[3]];
  double sn, cs;
  sincos(ta - tb, &sn, &cs);
  const double A = G2 * cs + B2 * sn, Bq = G2 * sn - B2 * cs;
  const double P = G1 * Va * Va + Va * Vb * A;
  const double Q = -B1 * Va * Va + Va * Vb * Bq;
  double dP[4] = {2 * G1 * Va + Vb * A, Va * A, -Va * Vb * Bq, Va * Vb * Bq};
  double dQ[4] = {-2 * B1 * Va + Vb * Bq, Va * Bq, Va * Vb * A, -Va * Vb * A};
  // lower-triangle second derivatives in the order of c_lowpairs
  double hP[10] = {2 * G1, A, 0.0, -Vb * Bq, -Va * Bq, -Va * Vb * A, Vb * Bq, Va * Bq, Va * Vb * A,
                   -Va * Vb * A};
  double hQ[10] = {-2 * B1, Bq, 0.0, Vb * A, Va * A, -Va * Vb * Bq, -Vb * A, -Va * A, Va * Vb * Bq,
                   -Va * Vb * Bq};
  atomicAdd(&g[bus], -P);
  atomicAdd(&g[D.nb + bus], -Q);
  const int hrow = e;
  const double rt = M.rate[k];
  h[hrow] = P * P + Q * Q - rt * rt;
  if (Jv) {
    const int *je = M.jentry + 2 * D.ng + 12 * e;
    for (int c = 0; c < 4; ++c) {
      atomicAdd(&Jv[je[c]], -dP[c]);
      atomicAdd(&Jv[je[4 + c]], -dQ[c]);
      Jv[je[8 + c]] = 2 * P * dP[c] + 2 * Q * dQ[c];
    }
  }
  if (Wv) {
    const double yP = y[bus], yQ = y[D.nb + bus], zz = z[hrow];
    const int *we = M.wentry + D.ng + 10 * e;
    for (int t = 0; t < 10; ++t) {
      int a = c_lowpairs[t][0], b = c_lowpairs[t][1];
      double hh = 2 * (dP[a] * dP[b] + P * hP[t] + dQ[a] * dQ[b] + Q * hQ[t]);
      atomicAdd(&Wv[we[t]], -yP * hP[t] - yQ * hQ[t] + zz * hh);
    }
  }
}

// generator gi: injections, its J entries, gradient and W entry; returns its cost
__device__ __forceinline__ double eval_gen_at(const OpfDims &D, const OpfData &M,
                                              const double *x, double sigma_f, double *g,
                                              double *grad, double *Jv, double *Wv, int gi) {
  int bus = M.gen_bus[gi];
  double pg = x[2 * D.nb + gi], qg = x[2 * D.nb + D.ng + gi];
  atomicAdd(&g[bus], pg);
  atomicAdd(&g[D.nb + bus], qg);
  if (Jv) {
    Jv[M.jentry[2 * gi]] = 1.0;
    Jv[M.jentry[2 * gi + 1]] = 1.0;
  }
  double pm = pg * BASE;
  if (grad) {
    grad[2 * D.nb + gi] = BASE * (2 * M.c2[gi] * pm + M.c1[gi]);
    grad[2 * D.nb + D.ng + gi] = 0.0;
  }
  if (Wv) atomicAdd(&Wv[M.wentry[gi]], sigma_f * 2 * M.c2[gi] * BASE * BASE);
  return M.c2[gi] * pm * pm + M.c1[gi] * pm;
}

// theta_ref row entry, the zero gradient on V, theta and the flow variables, f = sum of the
// block parts in order
__device__ __forceinline__ void eval_finish_at(const OpfDims &D, const OpfData &M,
                                               const double *fpart, int nparts, double *f,
                                               double *grad, double *Jv, int i, int stride) {
  if (grad) {
    for (int k = i; k < 2 * D.nb; k += stride) grad[k] = 0.0;
    // the branch-flow variables (flow form) do not enter the objective either
    for (int k = 2 * (D.nb + D.ng) + i; k < D.n; k += stride) grad[k] = 0.0;
  }
  if (i == 0) {
    if (Jv) Jv[M.jentry[2 * D.ng + 2 * jterms_per_end(D) * D.nbr]] = 1.0;
    if (f) {
      double s = 0.0;
      for (int p = 0; p < nparts; ++p) s += fpart[p];
      *f = s;
    }
  }
}

// flow-variable start: p_end, q_end = the flows of the voltages already in x
__device__ __forceinline__ void flow_start_at(const OpfDims &D, const OpfData &M, double *x, int e) {
  EndFlow F;
  end_flow_at(D, M, x, e, F);
  x[flow_pvar(D, e)] = F.P;
  x[flow_qvar(D, e)] = F.Q;
}

}  // namespace cipm
