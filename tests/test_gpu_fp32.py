"""FP32 condensation/factorization with FP64 refinement (precision row) against the oracle.

Bar: the factor is backward stable in single precision for the (shifted) FP32 matrix; every
KKT solve still reaches the FP64 bar of <= 1e-10 augmented backward error (computed by the
oracle on the GPU's solution); full IPM solves end at the oracle's objective within 1e-6.
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import config_grid
from oracle.opf import OPFModel
from oracle import kkt as K
from oracle import ipm as oipm
from tests.cases import kkt_case
from tests.test_gpu_parity import gpu_sym, dev, panels_to_lower, run_condense
import paper_2405_14236_gb300 as cp


@pytest.mark.parametrize("name", ["planar1k", "planar10k"])
def test_fp32_factor_is_single_precision_backward_stable(name):
    c = kkt_case(name)
    S = gpu_sym(c["J"], c["Wl"])
    N = cp.Numeric(S, precision=32)
    run_condense(c, S, N)
    torch.cuda.synchronize()
    K32 = panels_to_lower(S, N.export())
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    cp.ipm_factor(S, N, info)
    torch.cuda.synchronize()
    assert int(info.item()) == -1
    L = panels_to_lower(S, N.export())
    Kp = (K32 + sp.tril(K32, -1).T).tocsc()
    R = (L @ L.T - Kp).tocoo()
    absL = abs(L)
    bnd = np.asarray((absL @ absL.T).tocsc()[R.row, R.col]).ravel()
    k = int(np.diff(L.indptr).max()) + 1
    assert np.all(np.abs(R.data) <= 2 * k * np.finfo(np.float32).eps * bnd + 1e-30)


def fp32_factor(c, S, N, Wv, Jv, sig, d):
    """Inertia search in FP32: delta_w from the FP64 value upward until the FP32 factor exists."""
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    dw = c["dw"]
    for _ in range(30):
        cp.ipm_condense(S, N, Wv, sig, Jv, d, dw)
        cp.ipm_factor(S, N, info)
        if int(info.item()) == -1:
            return dw, info
        dw = max(1e-4, 100.0 * dw)
    raise AssertionError("no FP32 factor")


def fp32_lifted_solve(c):
    S = gpu_sym(c["J"], c["Wl"])
    N = cp.Numeric(S, precision=32)
    Wv, Jv = run_condense(c, S, N)
    sig, d = dev(c["sigma"], torch.float64), dev(c["d"], torch.float64)
    # the condensation inputs must stay alive for the FP64 products of the refinement
    dw, info = fp32_factor(c, S, N, Wv, Jv, sig, d)
    n, m = S.n, S.m
    dx = torch.zeros(n, dtype=torch.float64, device="cuda")
    dz = torch.zeros(m, dtype=torch.float64, device="cuda")
    eta = torch.zeros(1, dtype=torch.float64, device="cuda")
    steps = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = cp.ipm_aug_solve(S, N, Wv, sig, Jv, d, dw, dev(c["a"], torch.float64),
                          dev(c["b"], torch.float64), dx, dz, eta, steps)
    torch.cuda.synchronize()
    A = K.aug_matrix(c["Wf"], c["sigma"], c["J"], c["d"], 0, dw)
    sol = np.concatenate([dx.cpu().numpy(), dz.cpu().numpy()])
    return rc, K.backward_error(A, sol, np.concatenate([c["a"], c["b"]])), N


@pytest.mark.parametrize("name,log_range", [("ring30", 8.0), ("planar1k", 8.0), ("planar10k", 4.0)])
def test_fp32_lifted_solve_reaches_fp64_backward_error(name, log_range):
    """Sigma_x and D log-uniform over 10^-log_range .. 10^log_range; at 10,000 buses over eight
    decades (the shape of the middle iterations), where the FP32 factor still preconditions K."""
    rc, eta, N = fp32_lifted_solve(kkt_case(name, log_range=log_range))
    assert rc == cp.IPM_OK
    assert eta <= 1e-10
    prec, its = cp.ipm_num_info(N)
    assert prec == 32 and its >= 1


def test_fp32_lifted_reports_not_pd_when_ill_conditioned():
    """At 10,000 buses with Sigma_x and D spread over sixteen decades (late iterations)
    cond(K) 2^-24 >> 1: the FP32 factor no longer preconditions K to FP64 accuracy and the solve
    returns IPM_ERR_NOT_PD (the IPM then regularizes or moves to the FP64 factor) instead of an
    inaccurate step."""
    rc, eta, N = fp32_lifted_solve(kkt_case("planar10k", log_range=8.0))
    assert rc == cp.IPM_ERR_NOT_PD


def fp32_hykkt_solve(c):
    S = gpu_sym(c["J"], c["Wl"])
    N = cp.Numeric(S, precision=32)
    Wv, Jv = run_condense(c, S, N)
    sig, d = dev(c["sigma"], torch.float64), dev(c["d"], torch.float64)
    dw, info = fp32_factor(c, S, N, Wv, Jv, sig, d)
    me = c["me"]
    dx = torch.zeros(S.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(me, dtype=torch.float64, device="cuda")
    dz = torch.zeros(S.m - me, dtype=torch.float64, device="cuda")
    rc, its, rel = cp.hykkt_cg(S, N, me, Jv, d, c["gamma"], dev(c["a"], torch.float64),
                               dev(c["b"], torch.float64), dx, dy, dz)
    dh = c["d"][me:]
    A = K.aug_matrix(c["Wf"], c["sigma"], c["J"], dh, me, dw)
    sol = np.concatenate([dx.cpu().numpy(), dy.cpu().numpy(), dz.cpu().numpy()])
    return rc, K.backward_error(A, sol, np.concatenate([c["a"], c["b"]]))


@pytest.mark.parametrize("name,gamma", [("planar1k", 1e4), ("planar1k", 1e6), ("planar10k", 1e6)])
def test_fp32_hykkt_reaches_fp64_accuracy(name, gamma):
    """HyKKT with the FP32 factor of K_gamma: FP64-accurate inner solves, the Schur CG, and
    refinement on the augmented system reach the FP64 bar (Sigma_x, D over four decades)."""
    rc, eta = fp32_hykkt_solve(kkt_case(name, form="hykkt", gamma=gamma, log_range=2.0))
    assert rc == cp.IPM_OK
    assert eta <= 1e-10


def test_fp32_hykkt_reports_not_pd_when_ill_conditioned():
    """The condition number of K_gamma grows with gamma and with the spread of D (Theorem 4.1):
    with D over sixteen decades the FP32 factor does not precondition K_gamma to FP64 accuracy,
    and the solve says so (IPM_ERR_NOT_PD) rather than returning an inaccurate step."""
    rc, eta = fp32_hykkt_solve(kkt_case("planar1k", form="hykkt", gamma=1e6, log_range=8.0))
    assert rc == cp.IPM_ERR_NOT_PD


@pytest.mark.parametrize("kkt", ["lifted", "hykkt"])
def test_fp32_ipm_matches_oracle(kkt):
    """FP32 factor while its FP64-refined solves converge, then FP64 for good; same optimum."""
    g = config_grid("planar1k")
    ref = oipm.solve(OPFModel(g), oipm.Options(kkt=kkt, gamma=1e6))
    res = cp.ipm_solve_opf(cp.Opf(g), max_iter=2 * ref.iters + 20, kkt=kkt, gamma=1e6,
                           precision=32)
    assert res["status"] == 1, res["history"][-1]
    assert abs(res["obj"] - ref.obj) <= 1e-6 * abs(ref.obj)
    used = [h["precision"] for h in res["history"] if h["precision"]]
    # precision only escalates (FP32 while its refined solves converge, then FP64)
    assert all(a <= b for a, b in zip(used, used[1:]))
    if kkt == "lifted":
        assert used[0] == 32
    # HyKKT with gamma = 1e6: kappa(K_gamma) = Theta(max(1/s_min, gamma)) (Theorem 4.1) already
    # exceeds what an FP32 factor preconditions to FP64 accuracy, so it may switch at once
