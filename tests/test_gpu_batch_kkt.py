"""Per-solve parity of the batched KKT kernels: the all-instance condensation (k_b_condense), the
per-instance factorization (k_b_fact_inst) and triangular solves (k_b_solve_inst), with the
refinement (LiftedKKT) or the Schur-complement CG (HyKKT) on top.

Every instance is held right after the KKT solve of chosen iterations (ipm_batch_pause_at) and
exports the system it solved and its solution (ipm_batch_export_kkt); the oracle rebuilds the
augmented matrix (K_2) with the slack block eliminated from those values and computes the
normwise backward error eta of the GPU's solution (bar: 1e-10, Sec. 3.2 with Sec. 2.2's
iterative refinement).  The batch mixes load scenarios of the 1,000-bus grid with grids of
118-2,000 buses; the biggest run on 8-block thread-block clusters, and a second run takes the
shape the autotuner picks.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import config_grid, scale_loads, mixed_grid
from tests.cases import kkt_backward_error, kkt_oracle_eta
import paper_2405_14236_gb300 as cp

HOLD_AT = (0, 8, 20, 35)


def workload():
    base = config_grid("planar1k")
    return ([scale_loads(base, 1000 + k) for k in range(10)] +
            [mixed_grid(s) for s in (2025, 2016, 2036, 2003, 2010, 2011)])


def held_solves(B, opfs):
    """Runs the batch with holds after the KKT solves of the iterations in HOLD_AT; returns the
    oracle eta of every held solve as (iteration, instance, eta, eta of the oracle's own solve of
    that system where eta > 1e-10, else 0)."""
    out = []
    for k in HOLD_AT:
        B.pause_at(k)
        B.run(max_iter=300)
        r = B.results()
        for i in range(len(opfs)):
            if r["status"][i] != 0:
                continue   # converged (or stopped) before iteration k
            assert r["iters"][i] == k, (i, r["iters"][i], k)
            e = B.export_kkt(i)
            eta = kkt_backward_error(opfs[i], e)
            # LiftedKKT: where cond(K_tau) leaves the refinement stagnating above 1e-10 (Sec.
            # 3.2), the oracle's own solve of the same system is the bar (within 10x)
            eo = kkt_oracle_eta(opfs[i], e) if eta > 1e-10 and e["m_e"] == 0 else 0.0
            out.append((k, i, eta, eo))
        B.resume()
    B.pause_at(-1)
    B.run(max_iter=300)
    return out


def check_bar(etas, kkt):
    """HyKKT and the dual-regularized form: every held solve at eta <= 1e-10.  LiftedKKT: at least
    90 % at 1e-10, the rest within 10x of what the oracle's own solve of the same system reaches
    (the same bar as the single-problem LiftedKKT solves at 10,000 and 80,000 buses)."""
    if kkt != "lifted":
        worst = max(etas, key=lambda t: t[2])
        assert worst[2] <= 1e-10, worst
        return
    assert np.mean([t[2] <= 1e-10 for t in etas]) >= 0.9, sorted(t[2] for t in etas)[-5:]
    for k, i, eta, eo in etas:
        assert eta <= 1e-10 or eta <= 10 * eo, (k, i, eta, eo)


@pytest.mark.parametrize("kkt", ["lifted", "hykkt", "regularized"])
def test_batched_kkt_solves_on_clusters(kkt):
    grids = workload()
    opfs = [cp.Opf(g) for g in grids]
    B = cp.Batch(opfs, kkt=kkt, gamma=1e6)
    nbig = B.set_shape(8, 6, 5, 0)   # 8-block clusters above 1.2x the median supernode count
    assert nbig >= 3
    etas = held_solves(B, opfs)
    held_first = sum(1 for t in etas if t[0] == 0)
    assert held_first == len(grids)
    check_bar(etas, kkt)
    # the solves resume after the holds and end as the unheld batch does (convergence of the
    # whole batch against the oracle is tested in test_gpu_batch.py)
    r = B.results()
    assert np.isin(r["status"], [1, 5]).all() and (r["status"] == 1).mean() >= 0.8, r["status"]


@pytest.mark.parametrize("kkt", ["lifted", "regularized"])
def test_batched_kkt_solves_autotuned_shape(kkt):
    grids = workload()
    opfs = [cp.Opf(g) for g in grids]
    B = cp.Batch(opfs, kkt=kkt, gamma=1e6)
    t = B.autotune(sweeps=2)
    assert 0 <= t["best"] < len(t["candidates"])
    etas = held_solves(B, opfs)
    assert len(etas) >= len(grids)
    check_bar(etas, kkt)


def test_export_requires_a_held_instance():
    B = cp.Batch([cp.Opf(config_grid("ring30"))])
    with pytest.raises(cp.CondipmError):
        B.export_kkt(0)
