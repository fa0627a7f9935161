// Per-element arithmetic of one primal-dual interior-point iteration, shared by the
// single-problem kernels (ipm.cu) and the batched kernels (batch.cu).
//
// Problem (2) of the paper with slacks h(x) + s = 0, s >= 0 and Ipopt-style variable bounds
// (bound multipliers zl, zu eliminated into Sigma_x on the diagonal of K).  LiftedKKT
// (Section 3.2) relaxes the equalities to -tau <= g <= tau, i.e. rows g - tau <= 0 and
// -g - tau <= 0 in front of h <= 0; HyKKT (Section 3.1) keeps them as equalities.  Constants are
// those of Ipopt (Waechter & Biegler 2006, cited in Section 2.2).
#pragma once
#include "common.cuh"

namespace cipm {

static constexpr double KAPPA1 = 1e-2, KAPPA_EPS = 10.0, KAPPA_MU = 0.2, THETA_MU = 1.5;
static constexpr double TAU_MIN = 0.99, S_MAX = 100.0, GAMMA_THETA = 1e-5, GAMMA_PHI = 1e-8;
static constexpr double S_THETA = 1.1, S_PHI = 2.3, DELTA_SW = 1.0, ETA_PHI = 1e-8;
static constexpr double GAMMA_ALPHA = 0.05, KAPPA_SIGMA = 1e10, KAPPA_SIGMA_INV = 1.0 / KAPPA_SIGMA;
// rounding margin of barrier-function comparisons: phi is known to about 10 eps_mach |phi|, so
// values closer than that compare as equal (the Armijo test, the sufficient decrease and the
// filter entries alike)
static constexpr double PHI_MARGIN = 10.0 * 2.220446049250313e-16;
// directions recomputed with the next delta_w of the iteration's inertia-correction schedule
// after a line search that fails at a point feasible within the tolerance (where the
// restoration phase cannot help), before the method stops there
static constexpr int MAX_LS_REGULARIZE = 8;

// Filter acceptance of a trial point (tht, pht) at step alpha from (theta, phi) with directional
// derivative gphi (Waechter & Biegler 2006, Sec. 2.3-2.4): the filter (nfilter interleaved
// (theta, phi) pairs) and theta_max first, then, when the switching condition holds at
// theta <= theta_min, the Armijo test on phi (*ftype = 1: the step leaves the filter as is), else
// sufficient decrease in theta or in phi against the current iterate (*ftype = 0).
__host__ __device__ inline bool filter_accept(double theta, double phi, double gphi, double alpha,
                                              double tht, double pht, const double *filt,
                                              int nfilter, double theta_min, double theta_max,
                                              int *ftype) {
  *ftype = 0;
  const double margin = PHI_MARGIN * fabs(phi);
  if (!(tht < theta_max) || !isfinite(pht)) return false;
  for (int q = 0; q < nfilter; ++q)
    if (!(tht < filt[2 * q] || pht - filt[2 * q + 1] < margin)) return false;
  const bool switching = gphi < 0 && alpha * pow(-gphi, S_PHI) > DELTA_SW * pow(theta, S_THETA);
  if (switching && theta <= theta_min) {
    *ftype = 1;
    return pht - phi <= ETA_PHI * alpha * gphi + margin;
  }
  return tht <= (1 - GAMMA_THETA) * theta || pht - phi <= -GAMMA_PHI * theta + margin;
}

// ------------------------------------------------------------------ reductions into R[]
enum {
  R_MAX_GL, R_MAX_ZV, R_MAX_G, R_MAX_HS, R_MAX_SV, R_MAX_XL, R_MAX_XU,  // max |.|
  R_SUM_Y, R_SUM_Z, R_SUM_V, R_SUM_ZL, R_SUM_ZU,                        // sums |.|
  R_TH_G, R_TH_H, R_LOG_S, R_LOG_XL, R_LOG_XU,                          // theta / phi parts
  R_GPHI_X, R_GPHI_S,                                                    // d phi
  R_AMAX, R_AZ,                                                          // step bounds (min)
  R_PD, R_QD, R_MAXGRAD,                                                 // set-up
  // complementarity products s v, (x - xl) zl, (xu - x) zu: min and max over each set.  For any
  // mu, max_i |c_i - mu| = max(cmax - mu, mu - cmin) exactly (rounding is monotone), so the
  // barrier test can try several mu without another pass over the vectors.
  R_SV_MIN, R_SV_MAX, R_CL_MIN, R_CL_MAX, R_CU_MIN, R_CU_MAX,
  R_CG_A, R_CG_B,  // batched HyKKT CG: r.r and p.S p
  // restoration phase (single-problem IPM): objective part of phi_R, maxima of the dual,
  // primal and complementarity residuals, sums of all multipliers and of the bound-type ones
  R_RS_OBJ, R_RS_DUAL, R_RS_PRIM, R_RS_COMP, R_RS_SUMD, R_RS_SUMC,
  // restoration trial points (batched IPM): theta and barrier logs of the original problem
  R_RS_TH0, R_RS_LOG0,
  // batched PCG after a stagnating refinement: r.z, r.r, p.K p (t.t at its start)
  R_PG_A, R_PG_B, R_PG_C,
  R_COUNT
};

__device__ __forceinline__ void amax_nonneg(double *a, double v) {
  atomicMax((unsigned long long *)a, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void amin_nonneg(double *a, double v) {
  atomicMin((unsigned long long *)a, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ double wmax(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double wmin(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// warp-level reduce then one atomic per warp (every lane of the warp must call); the values
// reduced by max / min are non-negative, so their bit patterns order like the numbers
__device__ __forceinline__ void red_max(double *R, int k, double v) {
  v = wmax(v);
  if ((threadIdx.x & 31) == 0) amax_nonneg(R + k, v);
}
__device__ __forceinline__ void red_min(double *R, int k, double v) {
  v = wmin(v);
  if ((threadIdx.x & 31) == 0) amin_nonneg(R + k, v);
}
__device__ __forceinline__ void red_sum(double *R, int k, double v) {
  v = wsum(v);
  if ((threadIdx.x & 31) == 0) atomicAdd(R + k, v);
}

struct Dims {
  int n, me0, mi0;  // model sizes: variables, equality rows g, inequality rows h
  int me, mi;       // IPM sizes: equality rows (HyKKT: me0, Lifted: 0), slack rows
  int lifted;
};

struct It {  // device pointers of the iterate and work vectors
  double *x, *s, *y, *z, *v, *zl, *zu;
  double *xl, *xu;
  double *grad, *jtl;  // grad f, J~^T lambda
  double *geq, *hin;   // IPM rows
};

// step recovery and update arguments
struct StepArgs {
  Dims D;
  It P;
  double mu, dw;
  const double *r2, *r4, *Ds, *jdx, *dx, *sigma;
  const double *dzH;  // HyKKT: dz over H rows (from hykkt_cg)
  double *dz, *ds, *dv, *dzl, *dzu;
};

// a starting value moved strictly inside the bounds of variable j (Ipopt's bound push with
// kappa_1 = kappa_2 = 1e-2)
__device__ __forceinline__ double push_at(double v, const double *xl, const double *xu, int j) {
  const bool hl = isfinite(xl[j]), hu = isfinite(xu[j]);
  double pl = hl ? KAPPA1 * fmax(1.0, fabs(xl[j])) : 0.0;
  double pu = hu ? KAPPA1 * fmax(1.0, fabs(xu[j])) : 0.0;
  if (hl && hu) {
    pl = fmin(pl, KAPPA1 * (xu[j] - xl[j]));
    pu = fmin(pu, KAPPA1 * (xu[j] - xl[j]));
  }
  if (hl) v = fmax(v, xl[j] + pl);
  if (hu) v = fmin(v, xu[j] - pu);
  return v;
}

// flat start (|V| = 1, theta = 0, generators share the load equally), pushed inside the bounds
__device__ __forceinline__ double x0_at(int nb, int ng, double psum, double qsum,
                                        const double *xl, const double *xu, int j) {
  double v;
  if (j < nb) v = 1.0;
  else if (j < 2 * nb) v = 0.0;
  else if (j < 2 * nb + ng) v = fmin(fmax(psum / ng, xl[j]), xu[j]);
  else v = fmin(fmax(qsum / ng, xl[j]), xu[j]);
  return push_at(v, xl, xu, j);
}

// IPM constraint values from the scaled model: HyKKT  g' = g~, h' = h~;
// Lifted  h' = [g~ - tau ; -g~ - tau ; h~]
__device__ __forceinline__ void ipm_rows_at(const Dims &D, double tau, const double *gs,
                                            const double *hs, double *geq, double *hin, int k) {
  if (D.lifted) {
    if (k < D.me0) {
      hin[k] = gs[k] - tau;
      hin[D.me0 + k] = -gs[k] - tau;
    }
    if (k < D.mi0) hin[2 * D.me0 + k] = hs[k];
  } else {
    if (k < D.me0) geq[k] = gs[k];
    if (k < D.mi0) hin[k] = hs[k];
  }
}

// multipliers of the model rows: lambda = [lambda_g ; lambda_h] (unscaled-row weights)
__device__ __forceinline__ void lambda_at(const Dims &D, const double *y, const double *z,
                                          double *lam, int k) {
  if (k < D.me0) lam[k] = D.lifted ? z[k] - z[D.me0 + k] : y[k];
  if (k < D.mi0) lam[D.me0 + k] = D.lifted ? z[2 * D.me0 + k] : z[k];
}

// optimality error parts (Ipopt E_mu) of element i: maxima and 1-norm sums
struct ErrParts {
  double gl, zv, ge, hs, sv, xl, xu;  // |.| for the maxima
  double sy, sz, svv, szl, szu;       // |.| for the sums
  double csv, ccl, ccu;               // complementarity products (-1 where absent)
};
__device__ __forceinline__ ErrParts errors_at(const Dims &D, const It &P, double sig, double mu,
                                              int i) {
  ErrParts E{};
  E.csv = E.ccl = E.ccu = -1.0;
  if (i < D.n) {
    double x = P.x[i];
    E.gl = fabs(sig * P.grad[i] + P.jtl[i] - P.zl[i] + P.zu[i]);
    if (isfinite(P.xl[i])) {
      E.ccl = (x - P.xl[i]) * P.zl[i];
      E.xl = fabs(E.ccl - mu);
    }
    if (isfinite(P.xu[i])) {
      E.ccu = (P.xu[i] - x) * P.zu[i];
      E.xu = fabs(E.ccu - mu);
    }
    E.szl = fabs(P.zl[i]);
    E.szu = fabs(P.zu[i]);
  }
  if (i < D.mi) {
    E.zv = fabs(P.z[i] - P.v[i]);
    E.hs = fabs(P.hin[i] + P.s[i]);
    E.csv = P.s[i] * P.v[i];
    E.sv = fabs(E.csv - mu);
    E.sz = fabs(P.z[i]);
    E.svv = fabs(P.v[i]);
  }
  if (i < D.me) {
    E.ge = fabs(P.geq[i]);
    E.sy = fabs(P.y[i]);
  }
  return E;
}

// theta and phi parts of element i at (x, s) with constraint rows geq/hin
struct MeritParts {
  double tg, th, ls, lxl, lxu;
};
__device__ __forceinline__ MeritParts merit_at(const Dims &D, const double *x, const double *s,
                                               const double *xl, const double *xu,
                                               const double *geq, const double *hin, int i) {
  MeritParts M{};
  if (i < D.me) M.tg = fabs(geq[i]);
  if (i < D.mi) {
    M.th = fabs(hin[i] + s[i]);
    M.ls = log(s[i]);
  }
  if (i < D.n) {
    if (isfinite(xl[i])) M.lxl = log(x[i] - xl[i]);
    if (isfinite(xu[i])) M.lxu = log(xu[i] - x[i]);
  }
  return M;
}

// Sum of logarithms taken as the logarithm of a product: each factor is split on its bits into
// a mantissa in [1, 2) and an exponent, the mantissas are multiplied (one FP64 multiply per
// factor, the product renormalized on its bits) and the exponents added as integers; value()
// returns e ln 2 + log(m) (ln 2 in two parts, the first with 21 significant bits so that e times
// it is exact).  One log per thread instead of one per factor: on this GPU a double log is a
// few dozen FP64 instructions at 64 cycles each per warp.  A factor that is not a positive
// normal number adds its log directly.
struct LogSum {
  double m = 1.0, direct = 0.0;
  long long e = 0;
  __device__ __forceinline__ void add(double v) {
    const long long b = __double_as_longlong(v);
    const long long ex = b >> 52;  // includes the sign bit: negative v gives ex < 0
    if (ex <= 0 || ex >= 0x7ff) {
      direct += log(v);
      return;
    }
    m *= __longlong_as_double((b & 0xfffffffffffffLL) | 0x3ff0000000000000LL);
    const long long bm = __double_as_longlong(m);
    e += ex - 1023 + ((bm >> 52) - 1023);
    m = __longlong_as_double((bm & 0xfffffffffffffLL) | 0x3ff0000000000000LL);
  }
  __device__ __forceinline__ double value() const {
    const double ln2_hi = 0x1.62e42p-1, ln2_lo = 0x1.fdf473de6af28p-22;
    const double fe = (double)e;
    return fe * ln2_hi + (fe * ln2_lo + log(m)) + direct;
  }
};

// Newton right-hand sides and diagonals:
//   sigma_x = zl/(x-xl) + zu/(xu-x); r1 = sig grad + J~^T lambda - mu/(x-xl) + mu/(xu-x)
//   r2 = z - mu/s; r4 = h' + s; Ds = v/s
// A denominator used twice is inverted once (an FP64 division is a chain of about ten FP64
// instructions here, a multiply one).
__device__ __forceinline__ void newton_rhs_at(const Dims &D, const It &P, double sig, double mu,
                                              double *sigma, double *r1, double *r2, double *r4,
                                              double *Ds, int i) {
  if (i < D.n) {
    double sx = 0.0, r = sig * P.grad[i] + P.jtl[i];
    if (isfinite(P.xl[i])) {
      const double il = 1.0 / (P.x[i] - P.xl[i]);
      sx += P.zl[i] * il;
      r -= mu * il;
    }
    if (isfinite(P.xu[i])) {
      const double iu = 1.0 / (P.xu[i] - P.x[i]);
      sx += P.zu[i] * iu;
      r += mu * iu;
    }
    sigma[i] = sx;
    r1[i] = r;
  }
  if (i < D.mi) {
    const double is = 1.0 / P.s[i];
    r2[i] = P.z[i] - mu * is;
    r4[i] = P.hin[i] + P.s[i];
    Ds[i] = P.v[i] * is;
  }
}

// weights d and right-hand side b of the augmented system over the model rows [G; H]
//   Lifted: G rows combine the relaxed pair (D1 = Ds_a + dw, D2 = Ds_b + dw):
//           d = D1 + D2, b = (-D1 r4a + r2a + D2 r4b - r2b) / d;  H rows d = Ds + dw, b = -r4 + r2/d
//   HyKKT:  G rows d = gamma, b = -r3;  H rows as above
__device__ __forceinline__ void aug_rhs_at(const Dims &D, double dw, double gamma,
                                           const double *r2, const double *r4, const double *Ds,
                                           const double *geq, double *d, double *b, int k) {
  if (k < D.me0) {
    if (D.lifted) {
      double d1 = Ds[k] + dw, d2 = Ds[D.me0 + k] + dw;
      d[k] = d1 + d2;
      b[k] = (-d1 * r4[k] + r2[k] + d2 * r4[D.me0 + k] - r2[D.me0 + k]) / (d1 + d2);
    } else {
      d[k] = gamma;
      b[k] = -geq[k];
    }
  }
  if (k < D.mi0) {
    int ip = D.lifted ? 2 * D.me0 + k : k;
    double dh = Ds[ip] + dw;
    d[D.me0 + k] = dh;
    b[D.me0 + k] = -r4[ip] + r2[ip] / dh;
  }
}

// recover dz over the IPM slack rows from J~ dx (jdx over model rows), then ds, dv, dzl, dzu
__device__ __forceinline__ void recover_at(const StepArgs &A, int i) {
  const Dims &D = A.D;
  if (i < D.mi) {
    double dz;
    if (D.lifted) {
      double dh = A.Ds[i] + A.dw;
      double hdx = i < D.me0 ? A.jdx[i] : (i < 2 * D.me0 ? -A.jdx[i - D.me0] : A.jdx[i - D.me0]);
      dz = -A.r2[i] + dh * (hdx + A.r4[i]);
    } else {
      dz = A.dzH[i];
    }
    A.dz[i] = dz;
    double ds = -(A.r2[i] + dz) / (A.Ds[i] + A.dw);
    A.ds[i] = ds;
    A.dv[i] = (A.mu - A.P.v[i] * ds) / A.P.s[i] - A.P.v[i];
  }
  if (i < D.n) {
    double dx = A.dx[i];
    // dzl = (mu - zl dx) / (x - xl) - zl, dzu = (mu + zu dx) / (xu - x) - zu: one division each
    if (isfinite(A.P.xl[i])) {
      const double dl = A.P.x[i] - A.P.xl[i];
      A.dzl[i] = fma(-A.P.zl[i], dx, A.mu) / dl - A.P.zl[i];
    } else {
      A.dzl[i] = 0.0;
    }
    if (isfinite(A.P.xu[i])) {
      const double du = A.P.xu[i] - A.P.x[i];
      A.dzu[i] = fma(A.P.zu[i], dx, A.mu) / du - A.P.zu[i];
    } else {
      A.dzu[i] = 0.0;
    }
  }
}

// fraction to the boundary (ratios) and the directional derivative of phi, element i.  A ratio
// tau u / |d| only matters below 1 (the step bounds start at 1): it is divided out only when
// tau u < |d|, which near convergence leaves most elements without a division.
struct FtbParts {
  double ap, az, gx, gs;
};
__device__ __forceinline__ FtbParts ftb_at(const StepArgs &A, double tau, double sig, int i) {
  const Dims &D = A.D;
  FtbParts F{1.0, 1.0, 0.0, 0.0};
  if (i < D.n) {
    const double x = A.P.x[i], dx = A.dx[i];
    F.gx = sig * A.P.grad[i] * dx;
    const bool hl = isfinite(A.P.xl[i]), hu = isfinite(A.P.xu[i]);
    const double dl = hl ? x - A.P.xl[i] : 1.0, du = hu ? A.P.xu[i] - x : 1.0;
    if (hl) {
      if (dx < 0 && tau * dl < -dx) F.ap = fmin(F.ap, -tau * dl / dx);
      const double dz = A.dzl[i];
      if (dz < 0 && tau * A.P.zl[i] < -dz) F.az = fmin(F.az, -tau * A.P.zl[i] / dz);
    }
    if (hu) {
      if (dx > 0 && tau * du < dx) F.ap = fmin(F.ap, tau * du / dx);
      const double dz = A.dzu[i];
      if (dz < 0 && tau * A.P.zu[i] < -dz) F.az = fmin(F.az, -tau * A.P.zu[i] / dz);
    }
    // mu dx (1/du - 1/dl) with one division when both bounds exist
    if (hl && hu) F.gx += A.mu * dx * ((dl - du) / (dl * du));
    else if (hl) F.gx -= A.mu * dx / dl;
    else if (hu) F.gx += A.mu * dx / du;
  }
  if (i < D.mi) {
    const double ds = A.ds[i], dv = A.dv[i];
    if (ds < 0 && tau * A.P.s[i] < -ds) F.ap = fmin(F.ap, -tau * A.P.s[i] / ds);
    if (dv < 0 && tau * A.P.v[i] < -dv) F.az = fmin(F.az, -tau * A.P.v[i] / dv);
    F.gs = -A.mu * ds / A.P.s[i];
  }
  return F;
}

__device__ __forceinline__ void trial_at(int n, int mi, double a, const double *x,
                                         const double *dx, const double *s, const double *ds,
                                         double *xt, double *st, int i) {
  if (i < n) xt[i] = x[i] + a * dx[i];
  if (i < mi) st[i] = s[i] + a * ds[i];
}

// accept the step: primal (x, s from the trial), y, z with alpha, bound duals with alpha_z, then
// the bound-multiplier safeguard kappa_Sigma
__device__ __forceinline__ void accept_at(const StepArgs &A, double alpha, double az,
                                          const double *xt, const double *st, const double *dy,
                                          int i) {
  const Dims &D = A.D;
  const double mu = A.mu;
  if (i < D.n) {
    double x = xt[i];
    A.P.x[i] = x;
    // the kappa_Sigma band [mu / (kappa c), kappa mu / c] from one division mu / c
    if (isfinite(A.P.xl[i])) {
      const double q = mu / (x - A.P.xl[i]);
      const double zl = A.P.zl[i] + az * A.dzl[i];
      A.P.zl[i] = fmin(fmax(zl, q * KAPPA_SIGMA_INV), KAPPA_SIGMA * q);
    } else {
      A.P.zl[i] = 0.0;
    }
    if (isfinite(A.P.xu[i])) {
      const double q = mu / (A.P.xu[i] - x);
      const double zu = A.P.zu[i] + az * A.dzu[i];
      A.P.zu[i] = fmin(fmax(zu, q * KAPPA_SIGMA_INV), KAPPA_SIGMA * q);
    } else {
      A.P.zu[i] = 0.0;
    }
  }
  if (i < D.mi) {
    const double s = st[i];
    A.P.s[i] = s;
    A.P.z[i] += alpha * A.dz[i];
    const double q = mu / s;
    const double v = A.P.v[i] + az * A.dv[i];
    A.P.v[i] = fmin(fmax(v, q * KAPPA_SIGMA_INV), KAPPA_SIGMA * q);
  }
  if (i < D.me) A.P.y[i] += alpha * dy[i];
}

__device__ __forceinline__ void init_duals_at(const Dims &D, const It &P, double *s, int i) {
  if (i < D.mi) {
    s[i] = fmax(-P.hin[i], KAPPA1);
    P.z[i] = 1.0;
    P.v[i] = 1.0;
  }
  if (i < D.me) P.y[i] = 0.0;
  if (i < D.n) {
    P.zl[i] = isfinite(P.xl[i]) ? 1.0 : 0.0;
    P.zu[i] = isfinite(P.xu[i]) ? 1.0 : 0.0;
  }
}

// scaled optimality error from the reduced parts (Ipopt's s_d, s_c with s_max = 100);
// comp_mu: the complementarity part, already reduced for the mu in use
__host__ __device__ __forceinline__ double kkt_error(const double *h, const Dims &D, int nl,
                                                     int nu, double comp_mu) {
  double sd = fmax(S_MAX, (h[R_SUM_Y] + h[R_SUM_Z] + h[R_SUM_V] + h[R_SUM_ZL] + h[R_SUM_ZU]) /
                              (double)max(D.me + 2 * D.mi + nl + nu, 1)) / S_MAX;
  double sc = fmax(S_MAX, (h[R_SUM_V] + h[R_SUM_ZL] + h[R_SUM_ZU]) /
                              (double)max(D.mi + nl + nu, 1)) / S_MAX;
  double dual = fmax(h[R_MAX_GL], h[R_MAX_ZV]) / sd;
  double prim = fmax(h[R_MAX_G], h[R_MAX_HS]);
  return fmax(fmax(dual, prim), comp_mu / sc);
}

}  // namespace cipm
