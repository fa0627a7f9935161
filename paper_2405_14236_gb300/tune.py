"""Tuning of the supernode partition (the shape of the supernodal panels) for a batch.

The relaxed-supernode rule (ipm_symbolic_relaxed) trades explicit zeros in the panels (more
arithmetic) for fewer, wider supernodes (fewer levels of the supernodal elimination tree, fewer
barriers in the level-by-level batched kernels).  Which trade is faster depends on the patterns
and on the GPU, so the batch is built with each candidate rule and a few sweeps of it are timed
from the starting point; the fastest rule wins.  Host-side orchestration only: every analysis,
factorization and solve runs in the library.
"""
from __future__ import annotations

import time

# (relax_w, relax_den): (1, 0) = fundamental supernodes; (8, 5) = the library's default
CANDIDATES = ((1, 0), (4, 10), (8, 5), (16, 3))


def supernode_shapes(opfs, candidates=CANDIDATES, sweeps=8, max_iter=300, **batch_opts):
    """Times `sweeps` sweeps of the batch over `opfs` for each candidate partition rule.

    Returns (best, records): best = the (relax_w, relax_den) with the least time per sweep;
    records = per candidate {relax, ms_per_sweep, create_s, nsuper, nlevels (of the first
    pattern)}.  Each candidate's batch is destroyed before the next is built."""
    import torch
    import paper_2405_14236_gb300 as cp
    stream = torch.cuda.current_stream()
    recs = []
    for relax in candidates:
        t0 = time.perf_counter()
        B = cp.Batch(opfs, relax=relax, **batch_opts)
        torch.cuda.synchronize()
        create_s = time.perf_counter() - t0
        B.run(max_iter=max_iter, max_sweeps=1)  # captures the sweep graph
        B.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        B.run(max_iter=max_iter, max_sweeps=sweeps)
        e1.record(stream)
        e1.synchronize()
        done = max(1, B.results()["sweeps"])
        recs.append({"relax": list(relax), "ms_per_sweep": e0.elapsed_time(e1) / done,
                     "create_s": create_s})
        del B
        torch.cuda.synchronize()
    best = min(recs, key=lambda r: r["ms_per_sweep"])
    return tuple(best["relax"]), recs
