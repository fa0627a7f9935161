"""The 80,000-bus configuration (192,000 variables, 368,001 model rows) against the oracle:
symbolic analysis bit for bit, the LiftedKKT solve to the 1e-10 backward error, and the large
HyKKT case (gamma = 1e7) with an FP64 factor and with an FP32 factor preconditioning the FP64
Schur-complement CG (the FP32 handle reaches the FP64 bar or reports a nonzero status; it never
returns an inaccurate step as success)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import kkt as K
from oracle.sparse import Symbolic as OSym, condensed_pattern
from tests.cases import kkt_case
from tests.test_gpu_parity import gpu_sym, dev, run_condense
import paper_2405_14236_gb300 as cp


def test_symbolic_bit_exact_80k():
    c = kkt_case("planar80k")
    S = gpu_sym(c["J"], c["Wl"])
    g = S.export()
    o = OSym(condensed_pattern(K.full_from_lower(c["Wl"]), c["J"]))
    for key, ref in (("perm", o.perm), ("parent", o.parent), ("sptr", o.sptr),
                     ("colptr", o.colptr), ("rowind", o.rowind)):
        np.testing.assert_array_equal(g[key], ref)


def test_lifted_solve_80k():
    c = kkt_case("planar80k")
    S = gpu_sym(c["J"], c["Wl"])
    N = cp.Numeric(S)
    Wv, Jv = run_condense(c, S, N)
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    cp.ipm_factor(S, N, info)
    assert int(info.item()) == -1
    dx = torch.zeros(S.n, dtype=torch.float64, device="cuda")
    dz = torch.zeros(S.m, dtype=torch.float64, device="cuda")
    eta = torch.zeros(1, dtype=torch.float64, device="cuda")
    steps = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = cp.ipm_aug_solve(S, N, Wv, dev(c["sigma"], torch.float64), Jv, dev(c["d"], torch.float64),
                          c["dw"], dev(c["a"], torch.float64), dev(c["b"], torch.float64), dx, dz,
                          eta, steps)
    assert rc == cp.IPM_OK
    A = K.aug_matrix(c["Wf"], c["sigma"], c["J"], c["d"], 0, c["dw"])
    sol = np.concatenate([dx.cpu().numpy(), dz.cpu().numpy()])
    assert K.backward_error(A, sol, np.concatenate([c["a"], c["b"]])) <= 1e-10


def hykkt_80k(precision, log_range):
    c = kkt_case("planar80k", form="hykkt", gamma=1e7, log_range=log_range)
    S = gpu_sym(c["J"], c["Wl"])
    N = cp.Numeric(S, precision=precision)
    Wv, Jv = run_condense(c, S, N)
    sig, d = dev(c["sigma"], torch.float64), dev(c["d"], torch.float64)
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    dw = c["dw"]
    for _ in range(30):  # the FP32 factor of the shifted matrix may need a larger delta_w
        cp.ipm_condense(S, N, Wv, sig, Jv, d, dw)
        cp.ipm_factor(S, N, info)
        if int(info.item()) == -1:
            break
        dw = max(1e-4, 100.0 * dw)
    assert int(info.item()) == -1
    me = c["me"]
    dx = torch.zeros(S.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(me, dtype=torch.float64, device="cuda")
    dz = torch.zeros(S.m - me, dtype=torch.float64, device="cuda")
    rc, its, rel = cp.hykkt_cg(S, N, me, Jv, d, c["gamma"], dev(c["a"], torch.float64),
                               dev(c["b"], torch.float64), dx, dy, dz)
    A = K.aug_matrix(c["Wf"], c["sigma"], c["J"], c["d"][me:], me, dw)
    sol = np.concatenate([dx.cpu().numpy(), dy.cpu().numpy(), dz.cpu().numpy()])
    return rc, K.backward_error(A, sol, np.concatenate([c["a"], c["b"]]))


@pytest.mark.parametrize("precision,log_range", [(64, 8.0), (32, 2.0)])
def test_hykkt_gamma_1e7_80k(precision, log_range):
    """HyKKT with gamma = 1e7 at 80,000 buses: the FP64 factor at a late-iteration point
    (Sigma_x, D over sixteen decades), the FP32 factor with FP64 refinement at an early one
    (four decades); both reach the FP64 bar."""
    rc, eta = hykkt_80k(precision, log_range)
    assert rc == cp.IPM_OK
    assert eta <= 1e-10


def test_hykkt_gamma_1e7_80k_fp32_reports_not_pd_late():
    """At the late-iteration point the FP32 factor of K_gamma cannot precondition it to FP64
    accuracy: IPM_ERR_NOT_PD, and the IPM moves to the FP64 factor."""
    rc, eta = hykkt_80k(32, 8.0)
    assert rc == cp.IPM_ERR_NOT_PD
