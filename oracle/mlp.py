"""CPU oracle of the warm-start network: a multilayer perceptron with GELU hidden layers, a
linear output layer, mean-squared-error loss and Adam, in FP64 numpy.

Test infrastructure only (the tests, the smoke check and the benchmark's CPU baseline use it; the
CUDA path never calls it).

Definitions (the learned warm start has no counterpart in the paper; the network shape comes
from the workload description: 2 N_load inputs, three hidden layers of 512, GELU):
  Z_l = A_l W_l + b_l,  A_{l+1} = gelu(Z_l) for l < L-1,  Y = Z_{L-1}
  gelu(z) = z Phi(z), Phi the standard normal distribution function
  loss = mean over all B x d_L entries of (Y - T)^2
Backward pass by the chain rule; Adam (Kingma & Ba 2015) with bias correction.

``bf16=True`` rounds at the points where the GPU kernels hold BF16 values (network input,
hidden activations, weights as read by the products, output gradients fed to the products), so
that the remaining difference to the GPU is the FP32 accumulation order.  ``bf16=False`` is the
plain FP64 definition (pinned by finite differences in the tests).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def unflatten(dims, flat):
    """Per layer (W_l [d_l x d_{l+1}], b_l [d_{l+1}]) from the flat layout W_0, b_0, W_1, ..."""
    out, o = [], 0
    for l in range(len(dims) - 1):
        k, n = dims[l], dims[l + 1]
        W = np.asarray(flat[o:o + k * n], dtype=np.float64).reshape(k, n)
        o += k * n
        b = np.asarray(flat[o:o + n], dtype=np.float64)
        o += n
        out.append((W, b))
    return out


def flatten(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def forward_backward(dims, flat, X, T, bf16=False):
    """Returns (Y, loss, flat gradient) for parameters ``flat`` on inputs X [B x d_0] and
    targets T [B x d_L]."""
    layers = unflatten(dims, flat)
    L = len(layers)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    A = [r(X)]
    Z = []
    for l, (W, b) in enumerate(layers):
        z = A[l] @ r(W) + b
        Z.append(z)
        if l < L - 1:
            A.append(r(gelu(z)))
    Y = Z[-1]
    cnt = Y.size
    loss = float(np.sum((Y - np.asarray(T, dtype=np.float64)) ** 2) / cnt)
    dZ = 2.0 * (Y - T) / cnt
    grads = [None] * L
    for l in range(L - 1, -1, -1):
        W, b = layers[l]
        gW = A[l].T @ r(dZ)
        gb = dZ.sum(axis=0)
        grads[l] = (gW, gb)
        if l > 0:
            dA = r(dZ) @ r(W).T
            dZ = dA * gelu_grad(Z[l - 1])
    return Y, loss, flatten(grads)


def adam_step(flat, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step; returns new (flat, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v
