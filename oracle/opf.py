"""Oracle AC-OPF model: objective, constraints and exact derivatives (FP64, numpy).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package.

The model is the nonlinear program of Eq. (1) for a polar-form AC optimal
power flow on a synthetic grid (layout in ``synth.grid``):
  f(x) = sum_g c2 (100 Pg)^2 + c1 (100 Pg)
  g(x) = [P balance; Q balance; theta_ref]           (equalities)
  h(x) = [|S_from|^2 - rate^2; |S_to|^2 - rate^2]    (inequalities, h <= 0)
Each branch is a pi-model (series y = 1/(r + j x), shunt j b/2 at each end,
unit tap).  Derivatives are written out analytically per branch end and
assembled by coordinate sums (scipy COO), which is the plain definition of the
sparse Jacobian and of the Lagrangian Hessian W = sigma_f grad^2 f +
sum y_i grad^2 g_i + sum z_j grad^2 h_j (Section 2.2, block W_k of (K_3)).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

BASE = 100.0


def _branch_admittances(grid):
    den = grid.r ** 2 + grid.x ** 2
    gs = grid.r / den
    bs = -grid.x / den
    # from end: G1 = gs, B1 = bs + b/2, G2 = -gs, B2 = -bs ; to end identical (unit tap)
    return gs, bs + grid.b / 2.0, -gs, -bs


def _end_flow(Va, Vb, tha, thb, G1, B1, G2, B2):
    """Power leaving bus a on the branch end at a, with derivatives in the
    local variable order (Va, Vb, tha, thb)."""
    c = np.cos(tha - thb)
    s = np.sin(tha - thb)
    A = G2 * c + B2 * s
    Bq = G2 * s - B2 * c
    P = G1 * Va ** 2 + Va * Vb * A
    Q = -B1 * Va ** 2 + Va * Vb * Bq
    k = len(Va)
    dP = np.empty((k, 4))
    dQ = np.empty((k, 4))
    dP[:, 0] = 2 * G1 * Va + Vb * A
    dP[:, 1] = Va * A
    dP[:, 2] = -Va * Vb * Bq
    dP[:, 3] = Va * Vb * Bq
    dQ[:, 0] = -2 * B1 * Va + Vb * Bq
    dQ[:, 1] = Va * Bq
    dQ[:, 2] = Va * Vb * A
    dQ[:, 3] = -Va * Vb * A
    hP = np.zeros((k, 4, 4))
    hQ = np.zeros((k, 4, 4))
    hP[:, 0, 0] = 2 * G1
    hP[:, 0, 1] = A
    hP[:, 0, 2] = -Vb * Bq
    hP[:, 0, 3] = Vb * Bq
    hP[:, 1, 2] = -Va * Bq
    hP[:, 1, 3] = Va * Bq
    hP[:, 2, 2] = -Va * Vb * A
    hP[:, 2, 3] = Va * Vb * A
    hP[:, 3, 3] = -Va * Vb * A
    hQ[:, 0, 0] = -2 * B1
    hQ[:, 0, 1] = Bq
    hQ[:, 0, 2] = Vb * A
    hQ[:, 0, 3] = -Vb * A
    hQ[:, 1, 2] = Va * A
    hQ[:, 1, 3] = -Va * A
    hQ[:, 2, 2] = -Va * Vb * Bq
    hQ[:, 2, 3] = Va * Vb * Bq
    hQ[:, 3, 3] = -Va * Vb * Bq
    for H in (hP, hQ):
        for a in range(4):
            for b in range(a + 1, 4):
                H[:, b, a] = H[:, a, b]
    return P, Q, dP, dQ, hP, hQ


class OPFModel:
    """Evaluates f, grad f, g, h, J = [G; H] and W for one synthetic grid."""

    def __init__(self, grid):
        self.grid = grid
        self.n, self.m_e, self.m_i = grid.n, grid.m_e, grid.m_i
        self.oV, self.oT, self.oP, self.oQ = grid.var_offsets()
        self.xl, self.xu = grid.bounds()

    def x0(self):
        """Flat start: |V| = 1, theta = 0, every generator carrying an equal share of
        the total load (clipped to its bounds)."""
        g = self.grid
        pg = np.clip(np.full(g.ng, g.pd.sum() / g.ng), g.pmin, g.pmax)
        qg = np.clip(np.full(g.ng, g.qd.sum() / g.ng), g.qmin, g.qmax)
        return np.concatenate([np.ones(g.nb), np.zeros(g.nb), pg, qg])

    # -- per-end local variable indices (Va, Vb, tha, thb) ------------------
    def _ends(self):
        g = self.grid
        f, t = g.f_bus.astype(np.int64), g.t_bus.astype(np.int64)
        idx_f = np.stack([self.oV + f, self.oV + t, self.oT + f, self.oT + t], 1)
        idx_t = np.stack([self.oV + t, self.oV + f, self.oT + t, self.oT + f], 1)
        return (f, idx_f), (t, idx_t)

    def _flows(self, x):
        g = self.grid
        G1, B1, G2, B2 = _branch_admittances(g)
        out = []
        for bus, idx in self._ends():
            Va, Vb, tha, thb = (x[idx[:, k]] for k in range(4))
            out.append((bus, idx) + _end_flow(Va, Vb, tha, thb, G1, B1, G2, B2))
        return out

    def objective(self, x):
        pg = x[self.oP:self.oP + self.grid.ng] * BASE
        return float(np.sum(self.grid.c2 * pg ** 2 + self.grid.c1 * pg))

    def grad(self, x):
        gr = np.zeros(self.n)
        pg = x[self.oP:self.oP + self.grid.ng] * BASE
        gr[self.oP:self.oP + self.grid.ng] = BASE * (2 * self.grid.c2 * pg + self.grid.c1)
        return gr

    def cons(self, x):
        g = self.grid
        ge = np.zeros(self.m_e)
        np.add.at(ge, g.gen_bus, x[self.oP:self.oP + g.ng])
        np.add.at(ge, g.nb + g.gen_bus, x[self.oQ:self.oQ + g.ng])
        ge[:g.nb] -= g.pd
        ge[g.nb:2 * g.nb] -= g.qd
        hi = np.zeros(self.m_i)
        for e, (bus, idx, P, Q, *_r) in enumerate(self._flows(x)):
            np.add.at(ge, bus, -P)
            np.add.at(ge, g.nb + bus, -Q)
            hi[e * g.nbr:(e + 1) * g.nbr] = P ** 2 + Q ** 2 - g.rate ** 2
        ge[2 * g.nb] = x[self.oT + g.ref_bus]
        return ge, hi

    def jacobian(self, x):
        """J = [G; H] as a CSR matrix (m_e + m_i) x n with duplicates summed."""
        g = self.grid
        rows, cols, vals = [], [], []
        gi = np.arange(g.ng)
        rows += [g.gen_bus, g.nb + g.gen_bus]
        cols += [self.oP + gi, self.oQ + gi]
        vals += [np.ones(g.ng), np.ones(g.ng)]
        for e, (bus, idx, P, Q, dP, dQ, _hP, _hQ) in enumerate(self._flows(x)):
            for k in range(4):
                rows += [bus, g.nb + bus]
                cols += [idx[:, k], idx[:, k]]
                vals += [-dP[:, k], -dQ[:, k]]
                hrow = self.m_e + e * g.nbr + np.arange(g.nbr)
                rows.append(hrow)
                cols.append(idx[:, k])
                vals.append(2 * P * dP[:, k] + 2 * Q * dQ[:, k])
        rows.append(np.array([2 * g.nb]))
        cols.append(np.array([self.oT + g.ref_bus]))
        vals.append(np.array([1.0]))
        J = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.m_e + self.m_i, self.n)).tocsr()
        J.sum_duplicates()
        return J

    def hessian(self, x, y, z, sigma_f=1.0):
        """Full symmetric W = sigma_f grad^2 f + sum y grad^2 g + sum z grad^2 h."""
        g = self.grid
        rows, cols, vals = [], [], []
        gi = np.arange(g.ng)
        rows.append(self.oP + gi)
        cols.append(self.oP + gi)
        vals.append(sigma_f * 2 * g.c2 * BASE * BASE)
        for e, (bus, idx, P, Q, dP, dQ, hP, hQ) in enumerate(self._flows(x)):
            yP = y[bus]
            yQ = y[g.nb + bus]
            zz = z[e * g.nbr:(e + 1) * g.nbr]
            for a in range(4):
                for b in range(4):
                    hh = 2 * (dP[:, a] * dP[:, b] + P * hP[:, a, b]
                              + dQ[:, a] * dQ[:, b] + Q * hQ[:, a, b])
                    v = -yP * hP[:, a, b] - yQ * hQ[:, a, b] + zz * hh
                    rows.append(idx[:, a])
                    cols.append(idx[:, b])
                    vals.append(v)
        W = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.n, self.n)).tocsr()
        W.sum_duplicates()
        return W


class FlowOPFModel:
    """The same AC-OPF with branch-flow variables (the formulation whose sizes the paper's
    instances have: n = 2 N_b + 2 N_g + 4 N_br, m_e = 2 N_b + 1 + 4 N_br):
      x = [V | theta | Pg | Qg | p_end (2 N_br) | q_end (2 N_br)], ends = from ends then to ends
      g = [P balance (with -p_end) | Q balance (with -q_end) | theta_ref |
           p_end - P_end(V, theta) | q_end - Q_end(V, theta)]
      h = [p_end^2 + q_end^2 - rate^2]  (one row per branch end, h <= 0)
    Flow variables are free.  Its feasible set projects onto the compact model's, so both have
    the same optimum."""

    def __init__(self, grid):
        self.grid = grid
        nb, nbr, ng = grid.nb, grid.nbr, grid.ng
        self.nc = 2 * nb + 2 * ng
        self.n = self.nc + 4 * nbr
        self.m_e = 2 * nb + 1 + 4 * nbr
        self.m_i = 2 * nbr
        self.base = OPFModel(grid)
        lo, hi = grid.bounds()
        self.xl = np.concatenate([lo, np.full(4 * nbr, -np.inf)])
        self.xu = np.concatenate([hi, np.full(4 * nbr, np.inf)])
        self.op = self.nc                # p_end block
        self.oq = self.nc + 2 * nbr      # q_end block
        self.rp = 2 * nb + 1             # p definition rows
        self.rq = 2 * nb + 1 + 2 * nbr   # q definition rows

    def x0(self):
        """Compact flat start; each flow variable at the flow the start voltages give."""
        xc = self.base.x0()
        P = np.concatenate([fl[2] for fl in self.base._flows(xc)])
        Q = np.concatenate([fl[3] for fl in self.base._flows(xc)])
        return np.concatenate([xc, P, Q])

    def objective(self, x):
        return self.base.objective(x[:self.nc])

    def grad(self, x):
        return np.concatenate([self.base.grad(x[:self.nc]), np.zeros(4 * self.grid.nbr)])

    def cons(self, x):
        g = self.grid
        nb, nbr = g.nb, g.nbr
        xc = x[:self.nc]
        p, q = x[self.op:self.op + 2 * nbr], x[self.oq:self.oq + 2 * nbr]
        ge = np.zeros(self.m_e)
        np.add.at(ge, g.gen_bus, xc[2 * nb:2 * nb + g.ng])
        np.add.at(ge, nb + g.gen_bus, xc[2 * nb + g.ng:])
        ge[:nb] -= g.pd
        ge[nb:2 * nb] -= g.qd
        buses = np.concatenate([g.f_bus, g.t_bus])
        np.add.at(ge, buses, -p)
        np.add.at(ge, nb + buses, -q)
        ge[2 * nb] = xc[nb + g.ref_bus]
        flows = self.base._flows(xc)
        P = np.concatenate([fl[2] for fl in flows])
        Q = np.concatenate([fl[3] for fl in flows])
        ge[self.rp:self.rp + 2 * nbr] = p - P
        ge[self.rq:self.rq + 2 * nbr] = q - Q
        hi = p ** 2 + q ** 2 - np.concatenate([g.rate, g.rate]) ** 2
        return ge, hi

    def jacobian(self, x):
        g = self.grid
        nb, nbr, ng = g.nb, g.nbr, g.ng
        rows, cols, vals = [], [], []
        gi = np.arange(ng)
        rows += [g.gen_bus, nb + g.gen_bus]
        cols += [2 * nb + gi, 2 * nb + ng + gi]
        vals += [np.ones(ng), np.ones(ng)]
        ends = np.arange(2 * nbr)
        buses = np.concatenate([g.f_bus, g.t_bus])
        pv, qv = self.op + ends, self.oq + ends
        rows += [buses, nb + buses, self.rp + ends, self.rq + ends]
        cols += [pv, qv, pv, qv]
        vals += [-np.ones(2 * nbr), -np.ones(2 * nbr), np.ones(2 * nbr), np.ones(2 * nbr)]
        flows = self.base._flows(x[:self.nc])
        for e, (bus, idx, P, Q, dP, dQ, _hP, _hQ) in enumerate(flows):
            sl = np.arange(e * nbr, (e + 1) * nbr)
            for k in range(4):
                rows += [self.rp + sl, self.rq + sl]
                cols += [idx[:, k], idx[:, k]]
                vals += [-dP[:, k], -dQ[:, k]]
        hrow = self.m_e + ends
        rows += [hrow, hrow, np.array([2 * nb])]
        cols += [pv, qv, np.array([nb + g.ref_bus])]
        vals += [2 * x[pv], 2 * x[qv], np.array([1.0])]
        J = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.m_e + self.m_i, self.n)).tocsr()
        J.sum_duplicates()
        return J

    def hessian(self, x, y, z, sigma_f=1.0):
        g = self.grid
        nb, nbr, ng = g.nb, g.nbr, g.ng
        rows, cols, vals = [], [], []
        gi = np.arange(ng)
        rows.append(2 * nb + gi)
        cols.append(2 * nb + gi)
        vals.append(sigma_f * 2 * g.c2 * BASE * BASE)
        flows = self.base._flows(x[:self.nc])
        for e, (bus, idx, P, Q, dP, dQ, hP, hQ) in enumerate(flows):
            sl = np.arange(e * nbr, (e + 1) * nbr)
            yp, yq = y[self.rp + sl], y[self.rq + sl]
            for a in range(4):
                for b in range(4):
                    rows.append(idx[:, a])
                    cols.append(idx[:, b])
                    vals.append(-yp * hP[:, a, b] - yq * hQ[:, a, b])
        ends = np.arange(2 * nbr)
        rows += [self.op + ends, self.oq + ends]
        cols += [self.op + ends, self.oq + ends]
        vals += [2 * z, 2 * z]
        W = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.n, self.n)).tocsr()
        W.sum_duplicates()
        return W
