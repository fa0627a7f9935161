"""Shared test fixtures: seeded KKT problems evaluated by the oracle (test side only)."""
import functools

import numpy as np
import scipy.sparse as sp

from synth import config_grid, kkt_point
from oracle.opf import OPFModel
from oracle import kkt as K


@functools.lru_cache(maxsize=None)
def kkt_case(name, seed=3, log_range=8.0, form="lifted", gamma=1e6):
    """J, W(lower), sigma_x, row weights d, rhs (a, b), delta_w (oracle inertia search)."""
    g = config_grid(name)
    m = OPFModel(g)
    p = kkt_point(g, seed, log_range)
    J = m.jacobian(p["x"]).tocsr()
    J.sort_indices()
    Wf = m.hessian(p["x"], p["y"], p["z"])
    Wl = K.lower(Wf)
    Wl.sort_indices()
    sigma = p["sigma_x"]
    if form == "lifted":
        d = np.concatenate([p["d_g"], p["d_s"]])
        me = 0
    else:
        d = np.concatenate([np.full(g.m_e, gamma), p["d_s"]])
        me = g.m_e
    solver = K.CondensedSolver(Wf, J)
    dw, F, _ = K.inertia_schedule(lambda dw: K.condensed_matrix(Wf, sigma, J, d, dw), solver)
    a = p["r1"]
    b = np.concatenate([p["r3"], p["r4"]])
    return dict(grid=g, J=J, Wl=Wl, Wf=Wf, sigma=sigma, d=d, me=me, dw=dw, a=a, b=b,
                solver=solver, F=F, gamma=gamma)
