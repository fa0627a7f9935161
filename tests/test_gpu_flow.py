"""The flow-variable AC-OPF formulation on the GPU (ipm_opf_create_flow) against the oracle's
FlowOPFModel: identical sparsity patterns and model values, single-problem IPM solves in both
KKT forms, and a batch mixing both formulations.  The flow form reaches the compact form's
optimum (same problem, branch flows named as variables)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import config_grid, scale_loads
from oracle.opf import OPFModel, FlowOPFModel
from oracle import kkt as K
from oracle import ipm as oipm
import paper_2405_14236_gb300 as cp


@pytest.mark.parametrize("name", ["ring30", "planar1k"])
def test_flow_eval_matches_oracle(name):
    g = config_grid(name)
    m = FlowOPFModel(g)
    rng = np.random.default_rng(5)
    x = m.x0() + rng.normal(0, 0.02, m.n)
    y, z = rng.uniform(-1, 1, m.m_e), rng.uniform(-1, 1, m.m_i)
    opf = cp.Opf(g, form="flow")
    assert (opf.n, opf.m_e, opf.m_i) == (m.n, m.m_e, m.m_i)
    J = m.jacobian(x)
    Wl = K.lower(m.hessian(x, y, z, 0.37))
    J.sort_indices()
    Wl.sort_indices()
    np.testing.assert_array_equal(opf.J_rowptr.cpu().numpy(), J.indptr)
    np.testing.assert_array_equal(opf.J_colind.cpu().numpy(), J.indices)
    np.testing.assert_array_equal(opf.W_rowptr.cpu().numpy(), Wl.indptr)
    np.testing.assert_array_equal(opf.W_colind.cpu().numpy(), Wl.indices)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    # outputs start as NaN: every entry must be written by the evaluation (the IPM's buffers
    # are not cleared between evaluations, and reused device memory holds stale values)
    zz = lambda k: torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
    f, grad, gg, hh, Jv, Wv = zz(1), zz(m.n), zz(m.m_e), zz(m.m_i), zz(opf.nnzJ), zz(opf.nnzW)
    opf.eval(t(x), t(y), t(z), 0.37, f, grad, gg, hh, Jv, Wv)
    torch.cuda.synchronize()
    og, oh = m.cons(x)
    rel = lambda a, b: np.abs(a - b).max() / max(1.0, np.abs(b).max())
    assert abs(f.item() - m.objective(x)) <= 1e-12 * abs(m.objective(x))
    assert rel(grad.cpu().numpy(), m.grad(x)) < 1e-13
    assert rel(gg.cpu().numpy(), og) < 1e-12
    assert rel(hh.cpu().numpy(), oh) < 1e-12
    assert rel(Jv.cpu().numpy(), J.data) < 1e-12
    assert rel(Wv.cpu().numpy(), Wl.data) < 1e-12


@pytest.mark.parametrize("name,kkt", [("ring30", "hykkt"), ("ring30", "lifted"),
                                      ("planar1k", "hykkt"), ("planar1k", "lifted"),
                                      ("planar1k", "regularized")])
def test_flow_ipm_matches_oracle(name, kkt):
    g = config_grid(name)
    ref = oipm.solve(FlowOPFModel(g), oipm.Options(kkt=kkt, gamma=1e6))
    assert ref.status == "converged"
    res = cp.ipm_solve_opf(cp.Opf(g, form="flow"), kkt=kkt, gamma=1e6)
    assert res["status"] == 1, res["history"][-1]
    assert abs(res["obj"] - ref.obj) <= 1e-6 * abs(ref.obj)
    assert abs(res["iters"] - ref.iters) <= max(3, ref.iters // 5)
    if kkt == "hykkt":
        compact = oipm.solve(OPFModel(g), oipm.Options(kkt="hykkt", gamma=1e6))
        assert abs(res["obj"] - compact.obj) <= 1e-6 * abs(compact.obj)


@pytest.mark.parametrize("kkt", ["hykkt", "lifted"])
def test_flow_ipm_repeats_on_reused_memory(kkt):
    """Solves of the same 1,000-bus flow-form problem one after another, each with new handles
    whose device memory is what the previous solve freed: every solve reaches the same optimum
    in nearly the same number of iterations (a buffer read before it is written would make the
    result depend on the previous solve's leftovers)."""
    g = config_grid("planar1k")
    runs = []
    for _ in range(4):
        res = cp.ipm_solve_opf(cp.Opf(g, form="flow"), kkt=kkt, gamma=1e6)
        assert res["status"] == 1, res["history"][-1]
        runs.append((res["obj"], res["iters"]))
        del res
    objs = np.array([r[0] for r in runs])
    its = np.array([r[1] for r in runs])
    assert np.abs(objs - objs[0]).max() <= 1e-8 * abs(objs[0]), objs
    assert its.max() - its.min() <= 3, its


def test_batch_mixes_both_formulations():
    base = config_grid("planar1k")
    grids = [scale_loads(base, 1000 + k) for k in range(2)]
    opfs = [cp.Opf(grids[0]), cp.Opf(grids[0], form="flow"), cp.Opf(grids[1], form="flow")]
    B = cp.Batch(opfs, kkt="regularized", gamma=1e6)
    assert B.info()["patterns"] == 2
    B.run(max_iter=300)
    r = B.results()
    assert (r["status"] == 1).all(), r["status"]
    o = oipm.Options(kkt="regularized", gamma=1e6)
    refs = [oipm.solve(OPFModel(grids[0]), o), oipm.solve(FlowOPFModel(grids[0]), o),
            oipm.solve(FlowOPFModel(grids[1]), o)]
    for i, ref in enumerate(refs):
        assert abs(r["obj"][i] - ref.obj) <= 1e-6 * abs(ref.obj), i
