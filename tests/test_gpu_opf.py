"""GPU AC-OPF model evaluation against the oracle model (same point, same multipliers)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import config_grid, kkt_point
from oracle.opf import OPFModel
from oracle import kkt as K
import paper_2405_14236_gb300 as cp


@pytest.mark.parametrize("name", ["ring30", "planar1k", "planar10k"])
def test_opf_eval_matches_oracle(name):
    g = config_grid(name)
    m = OPFModel(g)
    p = kkt_point(g, 11)
    opf = cp.Opf(g)
    assert (opf.n, opf.m_e, opf.m_i) == (g.n, g.m_e, g.m_i)
    J = m.jacobian(p["x"])
    Wl = K.lower(m.hessian(p["x"], p["y"], p["z"], 0.37))
    J.sort_indices()
    Wl.sort_indices()
    # identical sparsity patterns (bit-exact)
    np.testing.assert_array_equal(opf.J_rowptr.cpu().numpy(), J.indptr)
    np.testing.assert_array_equal(opf.J_colind.cpu().numpy(), J.indices)
    np.testing.assert_array_equal(opf.W_rowptr.cpu().numpy(), Wl.indptr)
    np.testing.assert_array_equal(opf.W_colind.cpu().numpy(), Wl.indices)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    # outputs start as NaN: every entry must be written by the evaluation
    z = lambda k: torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
    f, grad, gg, hh, Jv, Wv = z(1), z(g.n), z(g.m_e), z(g.m_i), z(opf.nnzJ), z(opf.nnzW)
    opf.eval(t(p["x"]), t(p["y"]), t(p["z"]), 0.37, f, grad, gg, hh, Jv, Wv)
    torch.cuda.synchronize()
    og, oh = m.cons(p["x"])
    rel = lambda a, b: np.abs(a - b).max() / max(1.0, np.abs(b).max())
    assert abs(f.item() - m.objective(p["x"])) <= 1e-12 * abs(m.objective(p["x"]))
    assert rel(grad.cpu().numpy(), m.grad(p["x"])) < 1e-13
    assert rel(gg.cpu().numpy(), og) < 1e-12
    assert rel(hh.cpu().numpy(), oh) < 1e-12
    assert rel(Jv.cpu().numpy(), J.data) < 1e-12
    assert rel(Wv.cpu().numpy(), Wl.data) < 1e-12
