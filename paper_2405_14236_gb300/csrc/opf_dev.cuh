// Device side of the AC-OPF model evaluation (per branch end, per generator), shared by the
// single-problem kernels (opf.cu) and the batched ones (batch.cu).
//
// Layout: x = [V (nb) | theta (nb) | Pg (ng) | Qg (ng)];
// g = [P balance (nb) | Q balance (nb) | theta_ref]; h = [|S_from|^2 - rate^2 | |S_to|^2 - rate^2].
// Branch pi-model: series 1/(r + j x), shunt j b/2 per end, unit tap.  Cost on MW (base 100).
#pragma once
#include "opf.cuh"

namespace cipm {

static constexpr double BASE = 100.0;

struct OpfDims {
  int nb, nbr, ng, n, me, mi;
};

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

// branch end e: flows into the balance rows, thermal row, their derivatives, and the weighted
// second derivatives (y on the balance rows, z on the thermal row) into W
__device__ __forceinline__ void eval_branch_at(const OpfDims &D, const OpfData &M,
                                               const double *x, const double *y, const double *z,
                                               double *g, double *h, double *Jv, double *Wv,
                                               int e) {
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

// theta_ref row entry, the zero gradient on V and theta, f = sum of the block parts in order
__device__ __forceinline__ void eval_finish_at(const OpfDims &D, const OpfData &M,
                                               const double *fpart, int nparts, double *f,
                                               double *grad, double *Jv, int i, int stride) {
  if (grad)
    for (int k = i; k < 2 * D.nb; k += stride) grad[k] = 0.0;
  if (i == 0) {
    if (Jv) Jv[M.jentry[2 * D.ng + 24 * D.nbr]] = 1.0;
    if (f) {
      double s = 0.0;
      for (int p = 0; p < nparts; ++p) s += fpart[p];
      *f = s;
    }
  }
}

}  // namespace cipm
