"""The entry points on a non-blocking stream (torch.cuda.Stream(): no implicit ordering with the
legacy default stream, on which the library's synchronous host copies run).  Model creation,
symbolic analysis, IPM-state and batch creation order their work after the caller's stream and
finish before they return; the iterations run on the caller's stream.  The solves must give what
they give on the default stream: HyKKT and the dual-regularized form take the same path every
run, so the iteration counts and objectives agree to rounding."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import config_grid, scale_loads, mixed_grid
import paper_2405_14236_gb300 as cp


@pytest.mark.parametrize("form,kkt", [("compact", "hykkt"), ("flow", "regularized")])
def test_single_problem_on_a_nonblocking_stream(form, kkt):
    g = config_grid("planar1k")
    ref = cp.ipm_solve_opf(cp.Opf(g, form=form), kkt=kkt, gamma=1e6)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        res = cp.ipm_solve_opf(cp.Opf(g, form=form), kkt=kkt, gamma=1e6)
        # a checkpoint taken and loaded on the same stream continues to the same point
        st = res["state"]
        buf = st.save()
        st.load(buf)
        x_again = st.x()
    torch.cuda.synchronize()
    assert ref["status"] == 1 and res["status"] == 1, res["history"][-1]
    assert res["iters"] == ref["iters"]
    assert abs(res["obj"] - ref["obj"]) <= 1e-9 * abs(ref["obj"])
    np.testing.assert_array_equal(x_again, res["x"])


def test_batch_on_a_nonblocking_stream():
    base = config_grid("planar1k")
    grids = [scale_loads(base, 1000 + k) for k in range(3)] + [mixed_grid(2003)]
    ref_B = cp.Batch([cp.Opf(g) for g in grids], kkt="regularized", gamma=1e6)
    ref_B.run(max_iter=200)
    ref = ref_B.results()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        B = cp.Batch([cp.Opf(g) for g in grids], kkt="regularized", gamma=1e6)
        out = []
        for rnd in range(2):
            if rnd:
                B.reset()
            B.run(max_iter=200)
            out.append(B.results())
        x = B.x_all()
    torch.cuda.synchronize()
    for r in out:
        assert (r["status"] == 1).all(), r["status"]
        np.testing.assert_array_equal(r["iters"], ref["iters"])
        np.testing.assert_allclose(r["obj"], ref["obj"], rtol=1e-9)
    assert np.isfinite(x).all()
