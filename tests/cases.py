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


def kkt_backward_error(opf, e):
    """Oracle backward error of an exported KKT solve (IpmState.export_kkt, Batch.export_kkt):
    the augmented system (K_2) with the slack block eliminated, rebuilt by the oracle's
    definition (oracle/kkt.py) from the exported values and the model's patterns."""
    Jp, Ji = opf.J_rowptr.cpu().numpy(), opf.J_colind.cpu().numpy()
    Wp, Wi = opf.W_rowptr.cpu().numpy(), opf.W_colind.cpu().numpy()
    n, m = opf.n, opf.m_e + opf.m_i
    J = sp.csr_matrix((e["J_val"], Ji, Jp), shape=(m, n))
    Wl = sp.csr_matrix((e["W_val"], Wi, Wp), shape=(n, n))
    me = e["m_e"]   # rows kept as equalities (HyKKT): no -1/d block, d_row holds gamma there
    A = K.aug_matrix(K.full_from_lower(Wl), e["sigma"], J, e["d_row"][me:], me, e["delta_w"])
    sol = np.concatenate([e["dx"], e["dyz"]])
    return K.backward_error(A, sol, np.concatenate([e["a"], e["b"]]))


def kkt_oracle_eta(opf, e):
    """Backward error that the oracle's own solve reaches on an exported condensed-form KKT
    system (m_e = 0): condensed factor, Richardson refinement and the preconditioned CG after
    stagnation (oracle/kkt.py lifted_solve), measured like kkt_backward_error."""
    assert e["m_e"] == 0
    Jp, Ji = opf.J_rowptr.cpu().numpy(), opf.J_colind.cpu().numpy()
    Wp, Wi = opf.W_rowptr.cpu().numpy(), opf.W_colind.cpu().numpy()
    n, m = opf.n, opf.m_e + opf.m_i
    J = sp.csr_matrix((e["J_val"], Ji, Jp), shape=(m, n))
    Wf = K.full_from_lower(sp.csr_matrix((e["W_val"], Wi, Wp), shape=(n, n)))
    d = e["d_row"]
    F = K.CondensedSolver(Wf, J).factor(K.condensed_matrix(Wf, e["sigma"], J, d, e["delta_w"]))
    if not F.ok:
        return float("inf")
    A = K.aug_matrix(Wf, e["sigma"], J, d, 0, e["delta_w"])
    x, z, _ = K.lifted_solve(F, A, J, d, e["a"], e["b"])
    return K.backward_error(A, np.concatenate([x, z]), np.concatenate([e["a"], e["b"]]))
