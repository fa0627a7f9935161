"""The warm-start network on the GPU (mlp_* kernels: BF16 tensor-core products, FP32
accumulation) against the CPU oracle (oracle/mlp.py) with the same BF16 rounding points.

Bar: outputs and loss within 1e-3 relative (norm-wise) of the oracle, and every layer's
gradient within 1e-3 for the shallow network and 5e-3 for the five-layer one: the pre-rounding
values differ by FP32 (tensor-core) accumulation against FP64, a value near a BF16 rounding
boundary then rounds to the neighbouring BF16 number (2^-8 relative), and the backward pass
carries such differences through every layer.  Against the unrounded FP64 definition the bar is
5e-2 (the effect of BF16 storage itself).  Sizes are not multiples of the 64 x 64 product tiles,
so ragged tiles are covered."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlp as O
import paper_2405_14236_gb300 as cp


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("dims,B", [([40, 64, 72, 30], 37), ([2000, 512, 512, 512, 300], 96)])
def test_forward_backward_match_oracle(dims, B):
    rng = np.random.default_rng(3)
    net = cp.MLP(dims, max_batch=128)
    p = np.concatenate([np.concatenate([rng.normal(0, 1 / np.sqrt(k), k * n), rng.normal(0, 0.1, n)])
                        for k, n in zip(dims[:-1], dims[1:])]).astype(np.float32)
    net.set_params(p)
    X = rng.normal(size=(B, dims[0])).astype(np.float32)
    T = rng.normal(size=(B, dims[-1])).astype(np.float32)
    Xd = torch.as_tensor(X, device="cuda")
    Td = torch.as_tensor(T, device="cuda")
    Y = torch.empty(B, dims[-1], dtype=torch.float32, device="cuda")
    net.forward(Xd, Y)
    loss = float(net.loss_backward(Td).item())
    g = net.get_grads()
    Yo, lo, go = O.forward_backward(dims, p.astype(np.float64), X, T, bf16=True)
    _, _, gx = O.forward_backward(dims, p.astype(np.float64), X, T, bf16=False)
    assert rel(Y.cpu().numpy(), Yo) <= 1e-3
    assert abs(loss - lo) <= 1e-3 * lo
    bar = 1e-3 if len(dims) <= 4 else 5e-3
    o, errs = 0, []
    for k, n in zip(dims[:-1], dims[1:]):
        errs.append(("W", k, n, rel(g[o:o + k * n], go[o:o + k * n]), rel(g[o:o + k * n], gx[o:o + k * n])))
        o += k * n
        errs.append(("b", n, n, rel(g[o:o + n], go[o:o + n]), rel(g[o:o + n], gx[o:o + n])))
        o += n
    assert all(e[3] <= bar for e in errs), errs
    assert all(e[4] <= 5e-2 for e in errs), errs


def test_adam_step_matches_oracle():
    rng = np.random.default_rng(4)
    dims = [20, 33, 10]
    net = cp.MLP(dims, max_batch=16)
    p = rng.normal(0, 0.3, net.nparams).astype(np.float32)
    net.set_params(p)
    X = torch.as_tensor(rng.normal(size=(16, 20)).astype(np.float32), device="cuda")
    T = torch.as_tensor(rng.normal(size=(16, 10)).astype(np.float32), device="cuda")
    m = v = np.zeros(net.nparams)
    q = p.astype(np.float64)
    for t in range(1, 4):
        net.forward(X)
        net.loss_backward(T)
        g = net.get_grads().astype(np.float64)
        net.adam(1e-2)
        q, m, v = O.adam_step(q, g, m, v, t, lr=1e-2)
        assert rel(net.get_params(), q) <= 1e-5


def test_training_reduces_loss():
    rng = np.random.default_rng(5)
    X = rng.normal(size=(512, 16)).astype(np.float32)
    A = rng.normal(size=(16, 8))
    T = np.tanh(X @ A).astype(np.float32)
    from paper_2405_14236_gb300.warm import train
    _, losses = train(X, torch.as_tensor(T, device="cuda"), steps=300, batch=64, lr=3e-3,
                      hidden=(64, 64), log_every=50)
    assert losses[-1][1] < 0.1 * losses[0][1]
