"""Learned warm start of the batched interior-point method.

A network maps the loads of a scenario (2 N_load inputs: P and Q per bus) to an interior
primal-dual point of that scenario's OPF (x, log s, log v, log zl, log zu).  It is trained on
points that the batched IPM itself produces at a loose tolerance (central-path points near the
solution), and at solve time its prediction replaces the cold start of every instance (mu0 =
s^T v / m_i of the predicted point; an instance with a non-finite prediction keeps its cold
start).  Every arithmetic step runs in the library's kernels (batched IPM, MLP products on the
tensor cores, normalization); this module only orders the calls and shuffles indices.
"""
from __future__ import annotations

import numpy as np

from . import Batch, MLP, Opf, col_stats, gather_rows, normalize

HIDDEN = (512, 512, 512)


def input_rows(grids):
    """Loads of each scenario as one float32 row: [P_d (nb) | Q_d (nb)]."""
    return np.stack([np.concatenate([g.pd, g.qd]) for g in grids]).astype(np.float32)


def collect(grids, tol=1e-3, tau=1e-6, chunk=320, max_iter=300, kkt="lifted", gamma=1e6):
    """Solves every scenario (same grid, different loads) with the batched IPM in the KKT form
    ``kkt`` to ``tol`` (the LiftedKKT relaxation tau kept at the value of the full solves) and
    returns the state rows (float32 CUDA matrix) and the converged mask (numpy bool).  One batch
    of ``chunk`` instances is reused: loads are replaced, the batch is reset and run."""
    import torch
    n = len(grids)
    chunk = min(chunk, n)
    opfs = [Opf(g) for g in grids[:chunk]]
    B = Batch(opfs, tol=tol, tau=tau, kkt=kkt, gamma=gamma)
    rows = None
    ok = np.zeros(n, bool)
    for c0 in range(0, n, chunk):
        part = grids[c0:c0 + chunk]
        for o, g in zip(opfs, part):
            o.set_loads(np.ascontiguousarray(g.pd, np.float64), np.ascontiguousarray(g.qd, np.float64))
        for o, g in zip(opfs[len(part):], grids[:chunk - len(part)]):  # unused slots: any loads
            o.set_loads(np.ascontiguousarray(g.pd, np.float64), np.ascontiguousarray(g.qd, np.float64))
        B.reset()
        B.run(max_iter=max_iter)
        st = B.state_rows()
        if rows is None:
            rows = torch.empty(n, st.shape[1], dtype=torch.float32, device="cuda")
        rows[c0:c0 + len(part)] = st[:len(part)]
        ok[c0:c0 + len(part)] = B.results()["status"][:len(part)] == 1
    return rows, ok


def init_params(dims, seed):
    """Glorot-uniform weights, zero biases, in the flat layout of MLP.set_params."""
    rng = np.random.default_rng(seed)
    out = []
    for k, n in zip(dims[:-1], dims[1:]):
        a = np.sqrt(6.0 / (k + n))
        out += [rng.uniform(-a, a, k * n), np.zeros(n)]
    return np.concatenate(out).astype(np.float32)


class WarmStart:
    """The trained network with the normalization of its inputs and outputs."""

    def __init__(self, net, xmean, xstd, tmean, tstd):
        self.net, self.xmean, self.xstd, self.tmean, self.tstd = net, xmean, xstd, tmean, tstd

    def predict(self, X_host):
        """Normalized predictions (float32 CUDA) for host input rows."""
        import torch
        X = torch.as_tensor(X_host, device="cuda").contiguous()
        normalize(X, self.xmean, self.xstd)
        out = torch.empty(X.shape[0], self.tmean.shape[0], dtype=torch.float32, device="cuda")
        for r0 in range(0, X.shape[0], self.net.max_batch):
            r1 = min(X.shape[0], r0 + self.net.max_batch)
            self.net.forward(X[r0:r1], out[r0:r1])
        return out

    def start(self, batch, X_host):
        """Warm start of every instance of ``batch`` (after its reset) from its load rows."""
        pred = self.predict(X_host)
        return batch.warm_start(pred, self.tmean, self.tstd)


def train(X_host, T, steps=2000, batch=256, lr=1e-3, seed=0, hidden=HIDDEN, log_every=0):
    """Trains the network on input rows X_host (numpy) and target rows T (float32 CUDA; it is
    normalized in place) with Adam on the mean squared error; returns (WarmStart, losses)."""
    import torch
    X = torch.as_tensor(X_host, device="cuda").contiguous()
    xmean, xstd = col_stats(X)
    normalize(X, xmean, xstd)
    tmean, tstd = col_stats(T)
    normalize(T, tmean, tstd)
    dims = [X.shape[1], *hidden, T.shape[1]]
    net = MLP(dims, batch)
    net.set_params(init_params(dims, seed))
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    xb = torch.empty(batch, X.shape[1], dtype=torch.float32, device="cuda")
    tb = torch.empty(batch, T.shape[1], dtype=torch.float32, device="cuda")
    losses = []
    perm, pos = rng.permutation(n), 0
    for step in range(steps):
        if pos + batch > n:
            perm, pos = rng.permutation(n), 0
        bs = min(batch, n)
        idx = torch.as_tensor(perm[pos:pos + bs].astype(np.int32), device="cuda")
        pos += bs
        gather_rows(idx, X, xb[:bs])
        gather_rows(idx, T, tb[:bs])
        net.forward(xb[:bs])
        loss = net.loss_backward(tb[:bs])
        # step decay: the last quarter of the steps at a tenth of the rate
        net.adam(lr if step < 0.75 * steps else 0.1 * lr)
        if log_every and (step % log_every == 0 or step == steps - 1):
            losses.append((step, float(loss.item())))
    if not losses:
        losses.append((steps - 1, float(net.loss_backward(tb[:bs]).item())))
    return WarmStart(net, xmean, xstd, tmean, tstd), losses
