// Feasibility restoration phase of the single-problem IPM (Waechter & Biegler 2006, Sec. 3.3:
// the restoration phase of the filter line-search method cited in Sec. 2.2 of the paper).
//
// Restoration problem at the reference point xr, one pair (p, q) >= 0 per IPM row r:
//   min  rho sum(p + q) + zeta/2 sum_j dr2_j (x_j - xr_j)^2,   dr2 = min(1, 1/|xr|)^2
//   s.t. c_r - p_r + q_r = 0,   c_r = g_r (equality rows) or h'_r + s_r (slack rows),
//        bounds on x, s >= 0, p, q >= 0,
// solved by the same primal-dual filter IPM.  Its Newton system is condensed like the main
// one: p, q and their duals are eliminated row by row, which leaves every row of J with a
// (2,2) entry -E_r, E_r = 1/(Sigma_p + dw) + 1/(Sigma_q + dw) [+ 1/(D_s + dw) on slack rows],
// so K_R = W_R + Sigma_x + zeta D_R^2 + dw I + J^T diag(1/E) J has the pattern of the main
// condensed matrix (the same symbolic analysis and factor storage), and the refined condensed
// solve of the LiftedKKT form solves it for every KKT form.  W_R is the Hessian of the
// constraints' Lagrangian only (no objective term).
#pragma once
#include "ipm_core.cuh"

namespace cipm {

static constexpr double RHO_RESTO = 1000.0, KAPPA_RESTO = 0.9;

struct RArgs {
  Dims D;
  It P;                           // x, s, y (equality rows), z (slack rows), v, zl, zu, jtl
  double *p, *q, *zp, *zq;        // [R] per IPM row, R = D.me + D.mi
  const double *xr, *dr2;         // [n]
  double *sigma, *r1, *r2, *Ds;   // [n], [n], [mi], [mi]
  double *rc, *rp, *rq;           // [R] c - p + q, rho - lambda - mu/p, rho + lambda - mu/q
  double mu, zeta, dw;
  // step
  const double *dx, *jdx;         // [n], J~ dx over the model rows
  double *dy, *dz, *ds, *dv, *dzl, *dzu, *dp, *dq, *dzp, *dzq;
};

__device__ __forceinline__ double r_lam(const RArgs &A, int r) {
  return r < A.D.me ? A.P.y[r] : A.P.z[r - A.D.me];
}
__device__ __forceinline__ double r_c(const Dims &D, const double *geq, const double *hin,
                                      const double *s, int r) {
  return r < D.me ? geq[r] : hin[r - D.me] + s[r - D.me];
}

// right-hand sides and diagonals of the restoration Newton system
__device__ __forceinline__ void resto_rhs_at(const RArgs &A, int i) {
  const Dims &D = A.D;
  if (i < D.n) {
    const double x = A.P.x[i];
    double sx = A.zeta * A.dr2[i], r = A.zeta * A.dr2[i] * (x - A.xr[i]) + A.P.jtl[i];
    if (isfinite(A.P.xl[i])) {
      const double il = 1.0 / (x - A.P.xl[i]);
      sx += A.P.zl[i] * il;
      r -= A.mu * il;
    }
    if (isfinite(A.P.xu[i])) {
      const double iu = 1.0 / (A.P.xu[i] - x);
      sx += A.P.zu[i] * iu;
      r += A.mu * iu;
    }
    A.sigma[i] = sx;
    A.r1[i] = r;
  }
  if (i < D.mi) {
    A.r2[i] = A.P.z[i] - A.mu / A.P.s[i];
    A.Ds[i] = A.P.v[i] / A.P.s[i];
  }
  if (i < D.me + D.mi) {
    const double lam = r_lam(A, i), p = A.p[i], q = A.q[i];
    A.rc[i] = r_c(D, A.P.geq, A.P.hin, A.P.s, i) - p + q;
    A.rp[i] = RHO_RESTO - lam - A.mu / p;
    A.rq[i] = RHO_RESTO + lam - A.mu / q;
  }
}

// weight d_r = 1/E_r and right-hand side b_r of IPM row r
__device__ __forceinline__ void resto_row(const RArgs &A, int r, double *d, double *b) {
  const double sp = A.zp[r] / A.p[r] + A.dw, sq = A.zq[r] / A.q[r] + A.dw;
  double E = 1.0 / sp + 1.0 / sq;
  double bb = -A.rc[r] - A.rp[r] / sp + A.rq[r] / sq;
  if (r >= A.D.me) {
    const int k = r - A.D.me;
    const double dh = A.Ds[k] + A.dw;
    E += 1.0 / dh;
    bb += A.r2[k] / dh;
  }
  *d = 1.0 / E;
  *b = bb;
}

// weights and right-hand sides over the model rows [G; H] (LiftedKKT merges the relaxed pair,
// whose second row carries -G)
__device__ __forceinline__ void resto_aug_at(const RArgs &A, double *d, double *b, int k) {
  const Dims &D = A.D;
  if (k < D.me0) {
    if (D.lifted) {
      double d1, b1, d2, b2;
      resto_row(A, k, &d1, &b1);
      resto_row(A, D.me0 + k, &d2, &b2);
      d[k] = d1 + d2;
      b[k] = (d1 * b1 - d2 * b2) / (d1 + d2);
    } else {
      resto_row(A, k, d + k, b + k);
    }
  }
  if (k < D.mi0) {
    const int r = D.lifted ? 2 * D.me0 + k : D.me0 + k;
    resto_row(A, r, d + D.me0 + k, b + D.me0 + k);
  }
}

// step of every eliminated variable from dx (jdx = J~ dx over the model rows)
__device__ __forceinline__ void resto_recover_at(const RArgs &A, int i) {
  const Dims &D = A.D;
  if (i < D.me + D.mi) {
    double jv;
    if (D.lifted) {
      jv = i < D.me0 ? A.jdx[i] : (i < 2 * D.me0 ? -A.jdx[i - D.me0] : A.jdx[i - D.me0]);
    } else {
      jv = A.jdx[i];
    }
    double d, b;
    resto_row(A, i, &d, &b);
    const double dl = d * (jv - b);
    if (i < D.me) {
      A.dy[i] = dl;
    } else {
      const int k = i - D.me;
      A.dz[k] = dl;
      const double ds = -(A.r2[k] + dl) / (A.Ds[k] + A.dw);
      A.ds[k] = ds;
      A.dv[k] = (A.mu - A.P.v[k] * ds) / A.P.s[k] - A.P.v[k];
    }
    const double p = A.p[i], q = A.q[i];
    const double dp = (dl - A.rp[i]) / (A.zp[i] / p + A.dw);
    const double dq = (-dl - A.rq[i]) / (A.zq[i] / q + A.dw);
    A.dp[i] = dp;
    A.dq[i] = dq;
    A.dzp[i] = (A.mu - A.zp[i] * dp) / p - A.zp[i];
    A.dzq[i] = (A.mu - A.zq[i] * dq) / q - A.zq[i];
  }
  if (i < D.n) {
    const double dx = A.dx[i];
    if (isfinite(A.P.xl[i])) {
      const double dl = A.P.x[i] - A.P.xl[i];
      A.dzl[i] = (A.mu - A.P.zl[i] * dx) / dl - A.P.zl[i];
    } else {
      A.dzl[i] = 0.0;
    }
    if (isfinite(A.P.xu[i])) {
      const double du = A.P.xu[i] - A.P.x[i];
      A.dzu[i] = (A.mu + A.P.zu[i] * dx) / du - A.P.zu[i];
    } else {
      A.dzu[i] = 0.0;
    }
  }
}

// fraction to the boundary (primal: x bounds, s, p, q; dual: v, zl, zu, zp, zq) and the
// directional derivative of phi_R
__device__ __forceinline__ void resto_ftb_at(const RArgs &A, double tau, double *ap, double *az,
                                             double *g, int i) {
  const Dims &D = A.D;
  auto lim = [&](double val, double d, double *a) {
    if (d < 0 && tau * val < -d) *a = fmin(*a, -tau * val / d);
  };
  *ap = *az = 1.0;
  *g = 0.0;
  if (i < D.n) {
    const double x = A.P.x[i], dx = A.dx[i];
    *g += A.zeta * A.dr2[i] * (x - A.xr[i]) * dx;
    if (isfinite(A.P.xl[i])) {
      const double dl = x - A.P.xl[i];
      lim(dl, dx, ap);
      lim(A.P.zl[i], A.dzl[i], az);
      *g -= A.mu * dx / dl;
    }
    if (isfinite(A.P.xu[i])) {
      const double du = A.P.xu[i] - x;
      lim(du, -dx, ap);
      lim(A.P.zu[i], A.dzu[i], az);
      *g += A.mu * dx / du;
    }
  }
  if (i < D.mi) {
    lim(A.P.s[i], A.ds[i], ap);
    lim(A.P.v[i], A.dv[i], az);
    *g -= A.mu * A.ds[i] / A.P.s[i];
  }
  if (i < D.me + D.mi) {
    lim(A.p[i], A.dp[i], ap);
    lim(A.q[i], A.dq[i], ap);
    lim(A.zp[i], A.dzp[i], az);
    lim(A.zq[i], A.dzq[i], az);
    *g += RHO_RESTO * (A.dp[i] + A.dq[i]) - A.mu * (A.dp[i] / A.p[i] + A.dq[i] / A.q[i]);
  }
}

// theta_R, phi_R parts at the trial point (xt, st, pt, qt) with model rows geqt / hint:
// theta = sum |c - p + q|; obj = rho sum(p + q) + zeta/2 sum dr2 (x - xr)^2; logs of s, p, q
// and of the distances to the bounds
struct RMerit {
  double th, obj, ls, lxl, lxu;
};
__device__ __forceinline__ RMerit resto_merit_at(const RArgs &A, const double *xt,
                                                 const double *st, const double *pt,
                                                 const double *qt, const double *geqt,
                                                 const double *hint, int i) {
  const Dims &D = A.D;
  RMerit M{};
  if (i < D.n) {
    const double e = xt[i] - A.xr[i];
    M.obj = 0.5 * A.zeta * A.dr2[i] * e * e;
    if (isfinite(A.P.xl[i])) M.lxl = log(xt[i] - A.P.xl[i]);
    if (isfinite(A.P.xu[i])) M.lxu = log(A.P.xu[i] - xt[i]);
  }
  if (i < D.mi) M.ls = log(st[i]);
  if (i < D.me + D.mi) {
    M.th = fabs(r_c(D, geqt, hint, st, i) - pt[i] + qt[i]);
    M.obj += RHO_RESTO * (pt[i] + qt[i]);
    M.ls += log(pt[i]) + log(qt[i]);
  }
  return M;
}

// optimality error parts of the restoration problem at the current iterate (rows of the
// iterate: P.geq, P.hin at x): dual (x-gradient, z - v, p and q stationarity), primal
// (c - p + q), complementarity against mu, and the multiplier sums of Ipopt's s_d, s_c
struct RErr {
  double dual, prim, comp, sumd, sumc;
};
__device__ __forceinline__ RErr resto_errors_at(const RArgs &A, double mu, int i) {
  const Dims &D = A.D;
  RErr E{};
  if (i < D.n) {
    const double x = A.P.x[i];
    E.dual = fabs(A.zeta * A.dr2[i] * (x - A.xr[i]) + A.P.jtl[i] - A.P.zl[i] + A.P.zu[i]);
    if (isfinite(A.P.xl[i])) E.comp = fmax(E.comp, fabs((x - A.P.xl[i]) * A.P.zl[i] - mu));
    if (isfinite(A.P.xu[i])) E.comp = fmax(E.comp, fabs((A.P.xu[i] - x) * A.P.zu[i] - mu));
    E.sumc += fabs(A.P.zl[i]) + fabs(A.P.zu[i]);
  }
  if (i < D.mi) {
    E.dual = fmax(E.dual, fabs(A.P.z[i] - A.P.v[i]));
    E.comp = fmax(E.comp, fabs(A.P.s[i] * A.P.v[i] - mu));
    E.sumc += fabs(A.P.v[i]);
    E.sumd += fabs(A.P.z[i]);
  }
  if (i < D.me) E.sumd += fabs(A.P.y[i]);
  if (i < D.me + D.mi) {
    const double lam = r_lam(A, i);
    E.dual = fmax(E.dual, fmax(fabs(RHO_RESTO - lam - A.zp[i]), fabs(RHO_RESTO + lam - A.zq[i])));
    E.prim = fabs(r_c(D, A.P.geq, A.P.hin, A.P.s, i) - A.p[i] + A.q[i]);
    E.comp = fmax(E.comp, fmax(fabs(A.p[i] * A.zp[i] - mu), fabs(A.q[i] * A.zq[i] - mu)));
    E.sumc += fabs(A.zp[i]) + fabs(A.zq[i]);
  }
  E.sumd += E.sumc;
  return E;
}

// accept the step: primal with alpha (x, s, p, q from the trial), constraint multipliers with
// alpha, bound-type multipliers with alpha_z and the kappa_Sigma band
__device__ __forceinline__ void resto_accept_at(const RArgs &A, double alpha, double az,
                                                const double *xt, const double *st,
                                                const double *pt, const double *qt, int i) {
  const Dims &D = A.D;
  const double mu = A.mu;
  auto band = [&](double zval, double c) {
    const double qv = mu / c;
    return fmin(fmax(zval, qv * KAPPA_SIGMA_INV), KAPPA_SIGMA * qv);
  };
  if (i < D.n) {
    const double x = xt[i];
    A.P.x[i] = x;
    A.P.zl[i] = isfinite(A.P.xl[i]) ? band(A.P.zl[i] + az * A.dzl[i], x - A.P.xl[i]) : 0.0;
    A.P.zu[i] = isfinite(A.P.xu[i]) ? band(A.P.zu[i] + az * A.dzu[i], A.P.xu[i] - x) : 0.0;
  }
  if (i < D.mi) {
    A.P.s[i] = st[i];
    A.P.z[i] += alpha * A.dz[i];
    A.P.v[i] = band(A.P.v[i] + az * A.dv[i], st[i]);
  }
  if (i < D.me) A.P.y[i] += alpha * A.dy[i];
  if (i < D.me + D.mi) {
    A.p[i] = pt[i];
    A.q[i] = qt[i];
    A.zp[i] = band(A.zp[i] + az * A.dzp[i], pt[i]);
    A.zq[i] = band(A.zq[i] + az * A.dzq[i], qt[i]);
  }
}

// start of the restoration phase: p, q from the closed form of Eq. (33) of Waechter & Biegler
// (the minimizer of rho (p + q) - mu (log p + log q) on p - q = c, each root in the form that
// does not cancel), duals mu/p, mu/q; constraint multipliers zero; bound multipliers capped at
// rho; reference point and D_R^2
__device__ __forceinline__ void resto_start_at(const RArgs &A, double mu_r, double *xr,
                                               double *dr2, int i) {
  const Dims &D = A.D;
  if (i < D.n) {
    xr[i] = A.P.x[i];
    const double d = fmin(1.0, 1.0 / fmax(fabs(A.P.x[i]), 1e-300));
    dr2[i] = d * d;
    A.P.zl[i] = fmin(RHO_RESTO, A.P.zl[i]);
    A.P.zu[i] = fmin(RHO_RESTO, A.P.zu[i]);
  }
  if (i < D.mi) {
    A.P.v[i] = fmin(RHO_RESTO, A.P.v[i]);
    A.P.z[i] = 0.0;
  }
  if (i < D.me) A.P.y[i] = 0.0;
  if (i < D.me + D.mi) {
    const double c = r_c(D, A.P.geq, A.P.hin, A.P.s, i);
    const double rho = RHO_RESTO;
    const double sd = sqrt(mu_r * mu_r + (rho * c) * (rho * c));
    const double bq = mu_r - rho * c, bp = mu_r + rho * c;
    const double q = bq >= 0 ? (bq + sd) / (2.0 * rho) : -mu_r * c / (bq - sd);
    const double p = bp >= 0 ? (bp + sd) / (2.0 * rho) : mu_r * c / (bp - sd);
    A.p[i] = p;
    A.q[i] = q;
    A.zp[i] = mu_r / p;
    A.zq[i] = mu_r / q;
  }
}

// back to the main problem at element i: constraint multipliers from zero, bound-type
// multipliers above 1e3 reset to one (as Ipopt does after its restoration phase)
__device__ __forceinline__ void resto_finish_at(const Dims &D, const It &P, int i) {
  if (i < D.n) {
    if (P.zl[i] > 1e3) P.zl[i] = 1.0;
    if (P.zu[i] > 1e3) P.zu[i] = 1.0;
  }
  if (i < D.mi) {
    P.z[i] = 0.0;
    if (P.v[i] > 1e3) P.v[i] = 1.0;
  }
  if (i < D.me) P.y[i] = 0.0;
}

}  // namespace cipm
