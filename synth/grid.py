"""Seeded synthetic AC-OPF grids shaped like the paper's power-grid workloads.

The paper benchmarks on PGLIB-OPF instances (Section 6.2); those files are not
available here, so seeded synthetic grids stand in for them.  They keep the
shape that matters to the KKT solve: sparse, near-planar, average bus degree
about 2.6, and n = 2*N_bus + 2*N_gen primal variables in the compact polar
formulation.

Problem layout (shared convention, no arithmetic):
  x = [V (nb) | theta (nb) | Pg (ng) | Qg (ng)]             n   = 2nb + 2ng
  g = [P balance (nb) | Q balance (nb) | theta_ref]          m_e = 2nb + 1
  h = [|S_from|^2 - rate^2 (nbr) | |S_to|^2 - rate^2 (nbr)]  m_i = 2nbr
Per-unit quantities on a 100 MVA base; cost c2*(100 Pg)^2 + c1*(100 Pg).
"""
from __future__ import annotations

import dataclasses
import numpy as np

BASE_MVA = 100.0


@dataclasses.dataclass
class Grid:
    nb: int
    nbr: int
    ng: int
    f_bus: np.ndarray      # int32 [nbr]
    t_bus: np.ndarray      # int32 [nbr]
    r: np.ndarray          # float64 [nbr] series resistance
    x: np.ndarray          # float64 [nbr] series reactance
    b: np.ndarray          # float64 [nbr] total line charging
    rate: np.ndarray       # float64 [nbr] apparent-power limit (pu)
    pd: np.ndarray         # float64 [nb]
    qd: np.ndarray         # float64 [nb]
    gen_bus: np.ndarray    # int32 [ng], gen_bus[0] is the reference bus
    c2: np.ndarray         # float64 [ng]
    c1: np.ndarray         # float64 [ng]
    pmin: np.ndarray
    pmax: np.ndarray
    qmin: np.ndarray
    qmax: np.ndarray
    vmin: np.ndarray       # float64 [nb]
    vmax: np.ndarray       # float64 [nb]
    name: str = ""

    @property
    def ref_bus(self) -> int:
        return int(self.gen_bus[0])

    @property
    def n(self) -> int:
        return 2 * self.nb + 2 * self.ng

    @property
    def m_e(self) -> int:
        return 2 * self.nb + 1

    @property
    def m_i(self) -> int:
        return 2 * self.nbr

    def var_offsets(self):
        """Offsets of the V, theta, Pg, Qg blocks inside x."""
        return 0, self.nb, 2 * self.nb, 2 * self.nb + self.ng

    def bounds(self):
        """Lower/upper bounds on x (theta is free: +-inf)."""
        inf = np.inf
        lo = np.concatenate([self.vmin, np.full(self.nb, -inf), self.pmin, self.qmin])
        hi = np.concatenate([self.vmax, np.full(self.nb, inf), self.pmax, self.qmax])
        return lo, hi

    def arrays(self):
        return {k: getattr(self, k) for k in
                ("f_bus", "t_bus", "r", "x", "b", "rate", "pd", "qd", "gen_bus",
                 "c2", "c1", "pmin", "pmax", "qmin", "qmax", "vmin", "vmax")}


def _dc_rates(nb, f, t, x, pd, gen_bus, ref, factor, floor):
    """Branch ratings from a DC power flow of a proportional dispatch.

    The 'base flow' of the rating rule is read as the DC flow obtained when
    every generator supplies an equal share of the total load.  The rating is
    factor * |P_dc| * sqrt(1 + 0.3^2) (loads carry Q = 0.3 P), floored.  The floor
    matters on lines that carry almost no active power in the DC flow: their AC
    flow is mostly reactive (line charging, voltage differences), and a floor of
    0.1 pu made some grids infeasible (no dispatch and voltage profile met every
    rating), while 0.2 pu leaves all of the workload's grids feasible.
    """
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    inj = -pd.copy()
    np.add.at(inj, gen_bus, pd.sum() / len(gen_bus))
    bw = 1.0 / x
    rows = np.concatenate([f, t, f, t])
    cols = np.concatenate([f, t, t, f])
    vals = np.concatenate([bw, bw, -bw, -bw])
    B = sp.csr_matrix((vals, (rows, cols)), shape=(nb, nb)).tolil()
    keep = np.array([i for i in range(nb) if i != ref])
    Bred = B.tocsr()[keep][:, keep].tocsc()
    th = np.zeros(nb)
    th[keep] = spla.spsolve(Bred, inj[keep])
    pf = (th[f] - th[t]) * bw
    return np.maximum(factor * np.abs(pf) * np.sqrt(1.09), floor)


def _finish(rng, nb, f, t, ng, name, rate_factor=2.0, rate_floor=0.2, z_scale=1.0, load_scale=1.0):
    nbr = len(f)
    r = z_scale * rng.uniform(0.005, 0.05, nbr)
    x = r * rng.uniform(5.0, 10.0, nbr)
    b = rng.uniform(0.0, 0.05, nbr)
    pd = load_scale * rng.uniform(0.0, 0.5, nb)
    qd = 0.3 * pd
    gen_bus = rng.choice(nb, size=ng, replace=False).astype(np.int32)
    c2 = rng.uniform(0.01, 0.1, ng)
    c1 = rng.uniform(10.0, 40.0, ng)
    pmax = np.full(ng, 2.0 * pd.sum() / ng)
    pmin = np.zeros(ng)
    qmax = pmax.copy()
    qmin = -pmax
    rate = _dc_rates(nb, f, t, x, pd, gen_bus, int(gen_bus[0]), rate_factor, rate_floor)
    return Grid(nb=nb, nbr=nbr, ng=ng, f_bus=f.astype(np.int32), t_bus=t.astype(np.int32),
                r=r, x=x, b=b, rate=rate, pd=pd, qd=qd, gen_bus=gen_bus, c2=c2, c1=c1,
                pmin=pmin, pmax=pmax, qmin=qmin, qmax=qmax,
                vmin=np.full(nb, 0.94), vmax=np.full(nb, 1.06), name=name)


def ring_grid(nb: int = 30, n_chords: int = 11, ng: int = 6, seed: int = 1) -> Grid:
    """Ring over nb buses plus n_chords distinct random chords (no ring duplicates)."""
    rng = np.random.default_rng(seed)
    edges = {(i, (i + 1) % nb) if i < (i + 1) % nb else ((i + 1) % nb, i) for i in range(nb)}
    ring = sorted(edges)
    chords = []
    while len(chords) < n_chords:
        a, c = sorted(int(v) for v in rng.choice(nb, size=2, replace=False))
        if (a, c) in edges:
            continue
        edges.add((a, c))
        chords.append((a, c))
    allb = ring + chords
    f = np.array([e[0] for e in allb])
    t = np.array([e[1] for e in allb])
    return _finish(rng, nb, f, t, ng, f"ring{nb}")


def planar_grid(nb: int, ng: int, seed: int, branch_ratio: float = 1.3,
                z_scale: float = 0.2, load_scale: float = 0.2, rate_factor: float = 2.0,
                rate_floor: float = 0.2) -> Grid:
    """Random geometric planar graph: Delaunay triangulation of uniform points,
    its Euclidean minimum spanning tree, then the shortest remaining Delaunay
    edges until nbr = branch_ratio * nb.  Series impedances are the ring-grid
    draws times z_scale (r ~ z_scale U[0.005, 0.05], x = r U[5, 10]): with the
    unscaled draws the long, tree-like paths of these grids cannot carry the
    load within the voltage band.  Loads are load_scale U[0, 0.5] for the same
    reason (at full load a filter IPM without restoration does not converge)."""
    from scipy.spatial import Delaunay
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import minimum_spanning_tree
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 1.0, (nb, 2))
    tri = Delaunay(pts)
    s = tri.simplices
    e = np.concatenate([s[:, [0, 1]], s[:, [1, 2]], s[:, [0, 2]]])
    e.sort(axis=1)
    e = np.unique(e, axis=0)
    length = np.linalg.norm(pts[e[:, 0]] - pts[e[:, 1]], axis=1)
    W = coo_matrix((length, (e[:, 0], e[:, 1])), shape=(nb, nb)).tocsr()
    mst = minimum_spanning_tree(W).tocoo()
    in_tree = set(zip(np.minimum(mst.row, mst.col).tolist(), np.maximum(mst.row, mst.col).tolist()))
    order = np.lexsort((e[:, 1], e[:, 0], length))
    chosen = sorted(in_tree)
    target = int(round(branch_ratio * nb))
    for k in order:
        if len(chosen) >= target:
            break
        pair = (int(e[k, 0]), int(e[k, 1]))
        if pair in in_tree:
            continue
        in_tree.add(pair)
        chosen.append(pair)
    chosen = np.array(chosen)
    # shuffle branch order deterministically so the branch list carries no geometry
    perm = rng.permutation(len(chosen))
    chosen = chosen[perm]
    return _finish(rng, nb, chosen[:, 0], chosen[:, 1], ng, f"planar{nb}", z_scale=z_scale,
                   load_scale=load_scale, rate_factor=rate_factor, rate_floor=rate_floor)


def scale_loads(grid: Grid, seed: int, lo: float = 0.8, hi: float = 1.2) -> Grid:
    """Scenario: scale each bus load by U[lo, hi] (same pattern, new loads)."""
    rng = np.random.default_rng(seed)
    s = rng.uniform(lo, hi, grid.nb)
    return dataclasses.replace(grid, pd=grid.pd * s, qd=grid.qd * s,
                               name=f"{grid.name}-s{seed}")


def make_grid(nb: int, seed: int) -> Grid:
    """Planar grid with 20 % generator buses (the 10k / 80k / 1k-bus shapes)."""
    return planar_grid(nb, max(2, nb // 5), seed)


CONFIGS = {
    "ring30": dict(kind="ring", nb=30, seed=1),
    "planar1k": dict(kind="planar", nb=1000, seed=4),
    "planar10k": dict(kind="planar", nb=10000, seed=2),
    "planar80k": dict(kind="planar", nb=80000, seed=6),
}


def config_grid(name: str) -> Grid:
    c = CONFIGS[name]
    if c["kind"] == "ring":
        return ring_grid(c["nb"], seed=c["seed"])
    return make_grid(c["nb"], c["seed"])


def mixed_grid(seed: int, lo: int = 118, hi: int = 2000) -> Grid:
    """A grid of the mixed batch: N_b log-uniform in [lo, hi] drawn from the seed, then the
    planar generator with the same seed."""
    rng = np.random.default_rng(seed)
    nb = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
    return make_grid(nb, seed)


def recipe_grid(nb: int, seed: int) -> Grid:
    """Planar grid at the workload description's stated parameters, without this project's
    lightening: impedances and loads unscaled, ratings 1.2 x the base flow (the DC-flow reading)
    floored at 0.05 pu."""
    return planar_grid(nb, max(2, nb // 5), seed, z_scale=1.0, load_scale=1.0, rate_factor=1.2,
                       rate_floor=0.05)


def recipe_batch(n_scen: int = 32, n_mixed: int = 8):
    """The batched workload's shape at the stated parameters (recipe_grid): n_scen load scenarios
    of the 1,000-bus grid (seed 4; per-bus scaling U[0.8, 1.2], seeds 1000, ...) and n_mixed
    grids of 118-2000 buses (seeds 2000, ...)."""
    g = recipe_grid(1000, 4)
    mixed = []
    for k in range(n_mixed):
        rng = np.random.default_rng(2000 + k)
        nb = int(round(np.exp(rng.uniform(np.log(118), np.log(2000)))))
        mixed.append(recipe_grid(nb, 2000 + k))
    return [scale_loads(g, 1000 + k) for k in range(n_scen)] + mixed


def batch_grids(n_scen: int = 256, n_mixed: int = 64, base: str = "planar1k", part: int = 0):
    """The batched workload: n_scen load scenarios of the base grid (per-bus scaling U[0.8, 1.2],
    seeds 1000, 1001, ...) followed by n_mixed grids of 118-2000 buses (seeds 2000, 2001, ...).
    part > 0 draws another set of the same shape (scenario seeds from 1000 + 100000 part, mixed
    seeds from 2000 + 100000 part), e.g. one set per GPU."""
    g = config_grid(base)
    o = 100000 * part
    return ([scale_loads(g, o + 1000 + k) for k in range(n_scen)] +
            [mixed_grid(o + 2000 + k) for k in range(n_mixed)])


def kkt_point(grid: Grid, seed: int, log_range: float = 8.0):
    """A late-iteration-shaped KKT point: primal x inside the bounds, multipliers
    y, z ~ U[-1, 1], barrier diagonals Sigma_x and D_s log-uniform in
    [10^-log_range, 10^log_range], and standard-normal right-hand sides."""
    rng = np.random.default_rng(seed)
    nb, ng = grid.nb, grid.ng
    V = rng.uniform(0.95, 1.05, nb)
    th = rng.uniform(-0.2, 0.2, nb)
    th[grid.ref_bus] = 0.0
    pg = rng.uniform(grid.pmin, grid.pmax)
    qg = rng.uniform(grid.qmin, grid.qmax)
    x = np.concatenate([V, th, pg, qg])
    y = rng.uniform(-1.0, 1.0, grid.m_e)
    z = rng.uniform(-1.0, 1.0, grid.m_i)
    lo, hi = grid.bounds()
    sigma_x = 10.0 ** rng.uniform(-log_range, log_range, grid.n)
    sigma_x[~np.isfinite(lo) & ~np.isfinite(hi)] = 0.0
    d_s = 10.0 ** rng.uniform(-log_range, log_range, grid.m_i)
    d_g = 10.0 ** rng.uniform(-log_range, log_range, grid.m_e)
    r1 = rng.standard_normal(grid.n)
    r2 = rng.standard_normal(grid.m_i)
    r3 = rng.standard_normal(grid.m_e)
    r4 = rng.standard_normal(grid.m_i)
    return dict(x=x, y=y, z=z, sigma_x=sigma_x, d_s=d_s, d_g=d_g,
                r1=r1, r2=r2, r3=r3, r4=r4)
