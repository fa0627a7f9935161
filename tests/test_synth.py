"""The seeded input generators against the input recipe (host logic, no GPU): topology, sizes,
parameter ranges, reproducibility, and the shapes of the batched and warm-start workloads."""
import numpy as np
import pytest

from synth import config_grid, scale_loads, batch_grids
from synth.grid import mixed_grid, ring_grid, BASE_MVA


def _connected(nb, f, t):
    adj = [[] for _ in range(nb)]
    for a, c in zip(f.tolist(), t.tolist()):
        adj[a].append(c)
        adj[c].append(a)
    seen = np.zeros(nb, bool)
    stack = [0]
    seen[0] = True
    while stack:
        u = stack.pop()
        for v in adj[u]:
            if not seen[v]:
                seen[v] = True
                stack.append(v)
    return seen.all()


def _edges(g):
    return {(min(a, c), max(a, c)) for a, c in zip(g.f_bus.tolist(), g.t_bus.tolist())}


def test_ring30_topology():
    g = ring_grid()
    assert (g.nb, g.nbr, g.ng) == (30, 41, 6)
    e = _edges(g)
    assert len(e) == 41  # 30 ring edges and 11 distinct chords, no duplicates
    assert all((i, i + 1) in e for i in range(29)) and (0, 29) in e
    assert (g.f_bus != g.t_bus).all()
    assert _connected(g.nb, g.f_bus, g.t_bus)


@pytest.mark.parametrize("name", ["planar1k", "planar10k"])
def test_planar_grid_shape(name):
    g = config_grid(name)
    nb = g.nb
    assert g.nbr == int(round(1.3 * nb))
    assert len(_edges(g)) == g.nbr and (g.f_bus != g.t_bus).all()
    assert _connected(nb, g.f_bus, g.t_bus)
    assert abs(2 * g.nbr / nb - 2.6) < 1e-9          # average bus degree of the recipe
    assert g.ng == nb // 5 and len(set(g.gen_bus.tolist())) == g.ng
    assert g.ref_bus == g.gen_bus[0]
    assert (g.n, g.m_e, g.m_i) == (2 * nb + 2 * g.ng, 2 * nb + 1, 2 * g.nbr)


def test_parameter_ranges():
    for g, zs, ls in ((ring_grid(), 1.0, 1.0), (config_grid("planar1k"), 0.2, 0.2)):
        assert ((g.r >= 0.005 * zs) & (g.r <= 0.05 * zs)).all()
        ratio = g.x / g.r
        assert ((ratio >= 5.0) & (ratio <= 10.0)).all()
        assert ((g.b >= 0) & (g.b <= 0.05)).all()
        assert ((g.pd >= 0) & (g.pd <= 0.5 * ls)).all()
        assert np.allclose(g.qd, 0.3 * g.pd)
        assert np.allclose(g.pmax, 2.0 * g.pd.sum() / g.ng) and (g.pmin == 0).all()
        assert np.allclose(g.qmax, g.pmax) and np.allclose(g.qmin, -g.pmax)
        assert ((g.c2 >= 0.01) & (g.c2 <= 0.1)).all() and ((g.c1 >= 10) & (g.c1 <= 40)).all()
        assert (g.vmin == 0.94).all() and (g.vmax == 1.06).all()
        assert (g.rate >= 0.2).all()
    assert BASE_MVA == 100.0


def test_generators_are_reproducible():
    a, b = config_grid("planar1k"), config_grid("planar1k")
    for k, v in a.arrays().items():
        assert np.array_equal(v, b.arrays()[k]), k
    s1, s2 = scale_loads(a, 1003), scale_loads(a, 1003)
    assert np.array_equal(s1.pd, s2.pd)
    assert not np.array_equal(scale_loads(a, 1004).pd, s1.pd)


def test_load_scenarios_keep_the_pattern():
    g = config_grid("planar1k")
    s = scale_loads(g, 1000)
    assert np.array_equal(s.f_bus, g.f_bus) and np.array_equal(s.gen_bus, g.gen_bus)
    f = s.pd[g.pd > 0] / g.pd[g.pd > 0]
    assert ((f >= 0.8) & (f <= 1.2)).all()
    assert np.allclose(s.qd, 0.3 * s.pd)


def test_batch_and_mixed_workload_shapes():
    sizes = [mixed_grid(2000 + k).nb for k in range(64)]
    assert min(sizes) >= 118 and max(sizes) <= 2000
    assert len(set(sizes)) > 32  # unevenly sized grids
    grids = batch_grids(4, 2)
    assert len(grids) == 6
    assert all(g.nb == 1000 for g in grids[:4]) and [g.nb for g in grids[4:]] == sizes[:2]
    other = batch_grids(4, 2, part=1)  # another GPU's set: other seeds
    assert not np.array_equal(other[0].pd, grids[0].pd)


def test_recipe_grid_has_the_stated_parameters():
    """recipe_grid draws the planar topology with unscaled impedances and loads and ratings of
    1.2 x the DC base flow floored at 0.05 pu; the default grid of the same seed is the lightened
    one (x 0.2 impedances and loads, 2.0 x ratings floored at 0.2 pu)."""
    from synth import recipe_grid, recipe_batch, make_grid
    a, b = recipe_grid(300, 11), make_grid(300, 11)
    assert np.array_equal(a.f_bus, b.f_bus) and np.array_equal(a.t_bus, b.t_bus)
    assert np.allclose(a.r, 5 * b.r) and np.allclose(a.x, 5 * b.x)
    assert np.allclose(a.pd, 5 * b.pd) and np.allclose(a.qd, 0.3 * a.pd)
    assert a.r.min() >= 0.005 and a.r.max() <= 0.05
    assert a.rate.min() >= 0.05 - 1e-15 and b.rate.min() >= 0.2 - 1e-15
    gs = recipe_batch(3, 2)
    assert len(gs) == 5 and all(g.nb == 1000 for g in gs[:3]) and 118 <= gs[3].nb <= 2000
