"""ipm_solve_noalloc (the allocation-free solve) against ipm_solve, through the C ABI.

Some callers cannot allocate device memory when they call into the library (a runtime that
owns all device memory from start-up, a fixed memory budget, a loop that must stay out of the
allocator).  ipm_solve_noalloc serves them with a static device scratch array; it must give
the same answer as ipm_solve, on consecutive calls that reuse that array.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.cases import kkt_case
from oracle import kkt as K
import paper_2405_14236_gb300 as cp


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("name", ["planar1k", "planar10k"])
def test_noalloc_solve_matches_ipm_solve_twice(name):
    c = kkt_case(name)
    J, Wl = c["J"], c["Wl"]
    S = cp.Symbolic(J.shape[1], J.shape[0], dev(J.indptr, torch.int32), dev(J.indices, torch.int32),
                    dev(Wl.indptr, torch.int32), dev(Wl.indices, torch.int32))
    N = cp.Numeric(S)
    cp.ipm_condense(S, N, dev(Wl.data), dev(c["sigma"]), dev(J.data), dev(c["d"]), c["dw"])
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    cp.ipm_factor(S, N, info)
    torch.cuda.synchronize()
    assert int(info.item()) == -1
    rng = np.random.default_rng(5)
    for call in range(2):
        b = dev(rng.standard_normal(S.n))
        x_ref = torch.zeros(S.n, dtype=torch.float64, device="cuda")
        cp.ipm_solve(S, N, b, x_ref)
        x = torch.full((S.n,), float("nan"), dtype=torch.float64, device="cuda")
        st = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        cp.ipm_solve_noalloc(S, N, b, x, st)
        torch.cuda.synchronize()
        assert int(st.item()) == cp.IPM_OK
        xr, xn = x_ref.cpu().numpy(), x.cpu().numpy()
        assert np.all(np.isfinite(xn))
        # same kernels; only the order of the atomic sums may differ
        assert np.abs(xn - xr).max() <= 1e-10 * np.abs(xr).max()
        # and it solves K x = b (normwise backward error, as for ipm_solve)
        Kf = K.condensed_matrix(c["Wf"], c["sigma"], J, c["d"], c["dw"])
        bb = b.cpu().numpy()
        eta = np.abs(Kf @ xn - bb).max() / (abs(Kf).sum(axis=1).max() * np.abs(xn).max()
                                             + np.abs(bb).max())
        assert eta < 1e-13


def test_noalloc_rejects_bad_arguments():
    c = kkt_case("ring30")
    J, Wl = c["J"], c["Wl"]
    S = cp.Symbolic(J.shape[1], J.shape[0], dev(J.indptr, torch.int32), dev(J.indices, torch.int32),
                    dev(Wl.indptr, torch.int32), dev(Wl.indices, torch.int32))
    N = cp.Numeric(S)
    x = torch.zeros(S.n, dtype=torch.float64, device="cuda")
    with pytest.raises(cp.CondipmError):
        cp.lib()  # loaded
        rc = cp.lib().ipm_solve_noalloc(S.h, N.h, None, cp._ptr(x), None, None)
        cp._check(rc, "ipm_solve_noalloc")


def test_noalloc_without_status_buffer_returns_the_status():
    """d_status = NULL: the call waits for the solve and returns its status itself, so a timed-out
    wait cannot go unseen."""
    c = kkt_case("planar1k")
    J, Wl = c["J"], c["Wl"]
    S = cp.Symbolic(J.shape[1], J.shape[0], dev(J.indptr, torch.int32), dev(J.indices, torch.int32),
                    dev(Wl.indptr, torch.int32), dev(Wl.indices, torch.int32))
    N = cp.Numeric(S)
    cp.ipm_condense(S, N, dev(Wl.data), dev(c["sigma"]), dev(J.data), dev(c["d"]), c["dw"])
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    cp.ipm_factor(S, N, info)
    b = dev(np.random.default_rng(9).standard_normal(S.n))
    x_ref = torch.zeros(S.n, dtype=torch.float64, device="cuda")
    cp.ipm_solve(S, N, b, x_ref)
    x = torch.full((S.n,), float("nan"), dtype=torch.float64, device="cuda")
    rc = cp.lib().ipm_solve_noalloc(S.h, N.h, cp._ptr(b), cp._ptr(x), None, None)
    assert rc == cp.IPM_OK
    xr, xn = x_ref.cpu().numpy(), x.cpu().numpy()
    assert np.abs(xn - xr).max() <= 1e-10 * np.abs(xr).max()


def test_noalloc_rejects_n_above_its_limit():
    """n = 302,500 > 262,144 (the static scratch limit): IPM_ERR_BAD_ARG with a message, before
    any work.  The pattern is a 550 x 550 lattice (W lower: the west and north neighbours)."""
    side = 550
    n = side * side
    k = np.arange(n)
    cols = [k - side, k - 1, k]
    ok = [k >= side, (k % side) > 0, np.ones(n, bool)]
    rows_c = [c[o] for c, o in zip(cols, ok)]
    rows_r = [k[o] for o in ok]
    r = np.concatenate(rows_r)
    cc = np.concatenate(rows_c)
    order = np.lexsort((cc, r))
    r, cc = r[order], cc[order]
    W_rowptr = np.zeros(n + 1, np.int64)
    np.add.at(W_rowptr, r + 1, 1)
    W_rowptr = np.cumsum(W_rowptr).astype(np.int32)
    J_rowptr = np.array([0, 1], np.int32)
    J_colind = np.array([0], np.int32)
    S = cp.Symbolic(n, 1, dev(J_rowptr, torch.int32), dev(J_colind, torch.int32),
                    dev(W_rowptr, torch.int32), dev(cc.astype(np.int32), torch.int32))
    assert S.n == n > 262144
    N = cp.Numeric(S)
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc = cp.lib().ipm_solve_noalloc(S.h, N.h, cp._ptr(b), cp._ptr(x), None, None)
    assert rc == cp.IPM_ERR_BAD_ARG
    assert b"262144" in cp.lib().ipm_last_error_message()
