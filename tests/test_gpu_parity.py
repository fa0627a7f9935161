"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bar: symbolic output bit-exact; condensed matrix equal up to summation order; factor and
solves backward-stable; augmented-KKT backward error <= 1e-10 (computed by the oracle on the
GPU's solution).
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.sparse import Symbolic as OSym, condensed_pattern, Cholesky
from oracle import kkt as K
from oracle.opf import FlowOPFModel
from synth import config_grid
from tests.cases import kkt_case

import paper_2405_14236_gb300 as cp


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def gpu_sym(J, Wl, relax=(8, 5)):
    n = J.shape[1]
    return cp.Symbolic(n, J.shape[0], dev(J.indptr, torch.int32), dev(J.indices, torch.int32),
                       dev(Wl.indptr, torch.int32), dev(Wl.indices, torch.int32), relax=relax)


def panels_to_lower(sym, Lx):
    """Dense-coordinate COO of the lower panels (permuted positions)."""
    srow_ptr, srow, lptr = sym.export_panels()
    ex = sym.export()
    sptr = ex["sptr"]
    rows, cols, vals = [], [], []
    for s in range(sym.nsuper):
        f, l = sptr[s], sptr[s + 1]
        w = l - f
        rr = srow[srow_ptr[s]:srow_ptr[s + 1]]
        ld = len(rr)
        P = Lx[lptr[s]:lptr[s] + ld * w].reshape(w, ld).T
        for c in range(w):
            rows.append(rr[c:])
            cols.append(np.full(ld - c, f + c))
            vals.append(P[c:, c])
    n = sym.n
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def random_pattern_case(n, m, density, seed):
    rng = np.random.default_rng(seed)
    J = sp.random(m, n, density=density, random_state=seed, format="csr")
    J.data[:] = rng.standard_normal(J.nnz)
    Wl = sp.tril(sp.random(n, n, density=density / 2, random_state=seed + 1) + sp.identity(n),
                 format="csr")
    J.sort_indices()
    Wl.sort_indices()
    return J, Wl


SYM_CASES = ["ring30", "planar1k", "planar10k", "rand60", "rand500", "denserow", "disconnected",
             "planar1k-flow", "planar10k-flow"]


def flow_pattern(name):
    """J and lower W of the branch-flow formulation (oracle model) at its start point: the
    pattern of the paper-shaped instances, with 4 N_br free flow variables and their rows."""
    g = config_grid(name)
    m = FlowOPFModel(g)
    x = m.x0()
    J = m.jacobian(x).tocsr()
    J.sort_indices()
    Wl = K.lower(m.hessian(x, np.ones(m.m_e), np.ones(m.m_i)))
    Wl.sort_indices()
    return J, Wl


def sym_case(name):
    if name.endswith("-flow"):
        return flow_pattern(name[:-len("-flow")])
    if name.startswith("rand"):
        n = int(name[4:])
        return random_pattern_case(n, n // 2, 4.0 / n, n)
    if name == "denserow":
        J, Wl = random_pattern_case(200, 80, 0.02, 5)
        J = sp.vstack([J, sp.csr_matrix(np.ones((1, 200)))]).tocsr()
        return J, Wl
    if name == "disconnected":
        # block-diagonal J and W: three independent blocks of different sizes
        blocks = [random_pattern_case(k, k // 2, 3.0 / k, k) for k in (40, 150, 7)]
        J = sp.block_diag([b[0] for b in blocks], format="csr")
        Wl = sp.block_diag([b[1] for b in blocks], format="csr")
        J.sort_indices()
        Wl.sort_indices()
        return J, Wl
    c = kkt_case(name)
    return c["J"], c["Wl"]


@pytest.mark.parametrize("name", SYM_CASES)
def test_symbolic_bit_exact(name):
    J, Wl = sym_case(name)
    S = gpu_sym(J, Wl)
    g = S.export()
    o = OSym(condensed_pattern(K.full_from_lower(Wl), J))
    np.testing.assert_array_equal(g["perm"], o.perm)
    np.testing.assert_array_equal(g["parent"], o.parent)
    np.testing.assert_array_equal(g["sptr"], o.sptr)
    np.testing.assert_array_equal(g["colptr"], o.colptr)
    np.testing.assert_array_equal(g["rowind"], o.rowind)


def test_symbolic_is_deterministic():
    """The analysis runs on the GPU with atomics in its graph phases; its output must not depend
    on their order: four analyses of the 76,000-column flow-form pattern agree bit for bit."""
    J, Wl = sym_case("planar10k-flow")
    first = gpu_sym(J, Wl).export()
    for _ in range(3):
        again = gpu_sym(J, Wl).export()
        for k in first:
            np.testing.assert_array_equal(again[k], first[k], err_msg=k)


@pytest.mark.parametrize("relax", [(1, 0), (4, 10), (16, 3), (64, 1)])
@pytest.mark.parametrize("name", ["planar1k", "planar10k"])
def test_supernode_partition_bit_exact_for_each_relaxation(name, relax):
    """The supernode partition for other relaxation parameters (the candidates of the
    supernode-shape tuning), bit for bit against the oracle's."""
    J, Wl = sym_case(name)
    S = gpu_sym(J, Wl, relax=relax)
    o = OSym(condensed_pattern(K.full_from_lower(Wl), J), relax=relax)
    np.testing.assert_array_equal(S.export()["sptr"], o.sptr)
    assert S.nsuper == o.nsuper


def run_condense(c, S, N):
    Wv = dev(c["Wl"].data, torch.float64)
    Jv = dev(c["J"].data, torch.float64)
    cp.ipm_condense(S, N, Wv, dev(c["sigma"], torch.float64), Jv, dev(c["d"], torch.float64),
                    c["dw"])
    return Wv, Jv


@pytest.mark.parametrize("name", ["ring30", "planar1k", "planar10k"])
def test_condense_matches_oracle(name):
    c = kkt_case(name)
    S = gpu_sym(c["J"], c["Wl"])
    N = cp.Numeric(S)
    run_condense(c, S, N)
    torch.cuda.synchronize()
    Kg = panels_to_lower(S, N.export())
    perm = S.export()["perm"]
    Ko = K.condensed_matrix(c["Wf"], c["sigma"], c["J"], c["d"], c["dw"])
    Ko = sp.tril(sp.csc_matrix(Ko)[perm][:, perm].tocsc()).tocsc()
    scale = K.condensed_matrix(abs(c["Wf"]), np.abs(c["sigma"]), abs(c["J"]), np.abs(c["d"]),
                               abs(c["dw"]))
    scale = sp.tril(sp.csc_matrix(scale)[perm][:, perm].tocsc()).tocsc()
    diff = (Kg - Ko).tocoo()
    sc = np.asarray(scale[diff.row, diff.col]).ravel()
    # entries missing from the panels would show up here as -K_ij
    assert np.all(np.abs(diff.data) <= 1e-14 * sc + 1e-300)


@pytest.mark.parametrize("name", ["ring30", "planar1k", "planar10k"])
def test_factor_backward_stable_and_solve(name):
    c = kkt_case(name)
    S = gpu_sym(c["J"], c["Wl"])
    N = cp.Numeric(S)
    run_condense(c, S, N)
    torch.cuda.synchronize()
    Kg = panels_to_lower(S, N.export())
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    cp.ipm_factor(S, N, info)
    torch.cuda.synchronize()
    assert int(info.item()) == -1
    L = panels_to_lower(S, N.export())
    Kp = (Kg + sp.tril(Kg, -1).T).tocsc()
    R = (L @ L.T - Kp).tocoo()
    # Assumption 4.2: backward-stable Cholesky of the matrix it was given,
    # |P K P^T - L L^T| <= gamma_k |L| |L|^T entrywise with k the longest column of L
    absL = abs(L)
    bound = (absL @ absL.T).tocsc()
    bnd = np.asarray(bound[R.row, R.col]).ravel()
    k = int(np.diff(L.indptr).max()) + 1
    assert np.all(np.abs(R.data) <= 2 * k * np.finfo(float).eps * bnd + 1e-300)
    # the oracle factor of the same permuted matrix agrees entrywise (same ordering)
    Lo = c["F"].to_csc()
    rel = abs(L - Lo).max() / abs(Lo).max()
    assert rel < 1e-8
    # solve: normwise backward error of K x = b
    rng = np.random.default_rng(0)
    b = rng.standard_normal(S.n)
    x = torch.zeros(S.n, dtype=torch.float64, device="cuda")
    cp.ipm_solve(S, N, dev(b, torch.float64), x)
    xs = x.cpu().numpy()
    Kf = K.condensed_matrix(c["Wf"], c["sigma"], c["J"], c["d"], c["dw"])
    eta = np.abs(Kf @ xs - b).max() / (abs(Kf).sum(axis=1).max() * np.abs(xs).max() + np.abs(b).max())
    assert eta < 1e-13
    # several right-hand sides in one call (columns of an n x 3 column-major block, solved in
    # place): each equals its own single solve up to the order of the solves' atomic sums
    B3 = rng.standard_normal((3, S.n))
    X3 = dev(B3, torch.float64)
    cp.ipm_solve(S, N, X3, X3)
    for k in range(3):
        xk = torch.zeros(S.n, dtype=torch.float64, device="cuda")
        cp.ipm_solve(S, N, dev(B3[k], torch.float64), xk)
        assert float((X3[k] - xk).abs().max()) <= 1e-12 * float(xk.abs().max())
        e = np.abs(Kf @ X3[k].cpu().numpy() - B3[k]).max() / (
            abs(Kf).sum(axis=1).max() * np.abs(X3[k].cpu().numpy()).max() + np.abs(B3[k]).max())
        assert e < 1e-13


@pytest.mark.parametrize("name", ["ring30", "planar1k", "planar10k"])
def test_lifted_aug_solve_backward_error(name):
    c = kkt_case(name)
    S = gpu_sym(c["J"], c["Wl"])
    N = cp.Numeric(S)
    Wv, Jv = run_condense(c, S, N)
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    cp.ipm_factor(S, N, info)
    n, m = S.n, S.m
    dx = torch.zeros(n, dtype=torch.float64, device="cuda")
    dz = torch.zeros(m, dtype=torch.float64, device="cuda")
    eta = torch.zeros(1, dtype=torch.float64, device="cuda")
    steps = torch.zeros(1, dtype=torch.int32, device="cuda")
    cp.ipm_aug_solve(S, N, Wv, dev(c["sigma"], torch.float64), Jv, dev(c["d"], torch.float64),
                     c["dw"], dev(c["a"], torch.float64), dev(c["b"], torch.float64), dx, dz, eta,
                     steps)
    A = K.aug_matrix(c["Wf"], c["sigma"], c["J"], c["d"], 0, c["dw"])
    sol = np.concatenate([dx.cpu().numpy(), dz.cpu().numpy()])
    eta_oracle = K.backward_error(A, sol, np.concatenate([c["a"], c["b"]]))
    assert eta_oracle <= 1e-10
    assert abs(eta.item() - eta_oracle) <= 1e-3 * eta_oracle + 1e-300
    ox, oz, _ = K.lifted_solve(c["F"], A, c["J"], c["d"], c["a"], c["b"])
    assert np.abs(dx.cpu().numpy() - ox).max() <= 1e-6 * np.abs(ox).max()


@pytest.mark.parametrize("name", ["ring30", "planar1k", "planar10k"])
def test_hykkt_cg_matches_oracle(name):
    c = kkt_case(name, form="hykkt", gamma=1e6)
    S = gpu_sym(c["J"], c["Wl"])
    N = cp.Numeric(S)
    Wv, Jv = run_condense(c, S, N)
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    cp.ipm_factor(S, N, info)
    n, m, me = S.n, S.m, c["me"]
    dx = torch.zeros(n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(me, dtype=torch.float64, device="cuda")
    dz = torch.zeros(m - me, dtype=torch.float64, device="cuda")
    d = dev(c["d"], torch.float64)
    rc, its, rel = cp.hykkt_cg(S, N, me, Jv, d, c["gamma"], dev(c["a"], torch.float64),
                               dev(c["b"], torch.float64), dx, dy, dz)
    assert rc == cp.IPM_OK
    dh = c["d"][me:]
    ox, oy, oz, oits, orel = K.hykkt_solve(c["F"], c["Wf"], c["sigma"], c["J"], dh, me, c["dw"],
                                           c["gamma"], c["a"], c["b"])
    # both refine on the augmented system until eta <= 1e-10; whether a refinement solve is
    # needed is decided near that bar, so the totals agree up to whole extra HyKKT solves
    assert any(abs(its - k * oits) <= max(2, k * oits // 10) for k in (1, 2, 3, 4)), (its, oits)
    A = K.aug_matrix(c["Wf"], c["sigma"], c["J"], dh, me, c["dw"])
    sol = np.concatenate([dx.cpu().numpy(), dy.cpu().numpy(), dz.cpu().numpy()])
    rhs = np.concatenate([c["a"], c["b"]])
    assert K.backward_error(A, sol, rhs) <= 1e-10
    osol = np.concatenate([ox, oy, oz])
    assert K.backward_error(A, sol, rhs) <= 10 * K.backward_error(A, osol, rhs) + 1e-16


def test_factor_reports_first_failing_pivot():
    c = kkt_case("planar1k")
    S = gpu_sym(c["J"], c["Wl"])
    N = cp.Numeric(S)
    # delta_w = 0 with a strongly negative shift on a few variables: not positive definite
    sigma = c["sigma"].copy()
    sigma[[5, 700, 1500]] = -1e9
    cp.ipm_condense(S, N, dev(c["Wl"].data, torch.float64), dev(sigma, torch.float64),
                    dev(c["J"].data, torch.float64), dev(c["d"], torch.float64), 0.0)
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    cp.ipm_factor(S, N, info)
    F = Cholesky(K.condensed_matrix(c["Wf"], sigma, c["J"], c["d"], 0.0), c["solver"].sym)
    assert not F.ok
    assert int(info.item()) == F.fail


def test_wait_timeout_reports_status_without_fault():
    """A dependency that nothing satisfies ends in IPM_ERR_TIMEOUT, not a hang or a fault;
    a fresh analysis of the same pattern factors normally afterwards."""
    c = kkt_case("ring30")
    S = gpu_sym(c["J"], c["Wl"])
    N = cp.Numeric(S)
    run_condense(c, S, N)
    cp.ipm_set_spin_limit(20000)
    try:
        cp.ipm_debug_add_dependency(S, S.nsuper - 1, 1)
        info = torch.zeros(1, dtype=torch.int32, device="cuda")
        cp.ipm_factor(S, N, info)
        torch.cuda.synchronize()
        assert int(info.item()) == -2
        assert cp.ipm_num_status(N) == cp.IPM_ERR_TIMEOUT
    finally:
        cp.ipm_set_spin_limit(1 << 23)
    S2 = gpu_sym(c["J"], c["Wl"])
    N2 = cp.Numeric(S2)
    run_condense(c, S2, N2)
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    cp.ipm_factor(S2, N2, info)
    torch.cuda.synchronize()
    assert int(info.item()) == -1 and cp.ipm_num_status(N2) == 0
