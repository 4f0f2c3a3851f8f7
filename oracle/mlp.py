"""FP64 reference of the emulator's network (test infrastructure only).

Plain numpy: the 16-256-256-256-392 multilayer perceptron with GELU (tanh
form: 0.5 x (1 + tanh(sqrt(2 / pi) (x + 0.044715 x^3)))), the mean over rows of the summed cross-entropies of its three
129-way heads, and the gradients of that loss by the chain rule.  The tests
pin these gradients to central finite differences and compare the CUDA
kernels' gradients with them.
"""
from __future__ import annotations

import math

import numpy as np

HEADS, BINS = 3, 129

_C = math.sqrt(2.0 / math.pi)
_A = 0.044715


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(_C * (x + _A * x ** 3)))


def gelu_grad(x):
    t = np.tanh(_C * (x + _A * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * _C * (1.0 + 3.0 * _A * x * x)


def forward(Ws, bs, X):
    """Ws[l]: (out, in) weights, bs[l]: (out,) biases, X: (B, in).  Returns
    logits and the per-layer (input, pre-activation) pairs."""
    h = X
    cache = []
    for li, (Wl, bl) in enumerate(zip(Ws, bs)):
        pre = h @ Wl.T + bl
        cache.append((h, pre))
        h = gelu(pre) if li < len(Ws) - 1 else pre
    return h, cache


def loss_and_grads(Ws, bs, X, targets, return_cache=False):
    """Mean over rows of the summed head cross-entropies, and dW, db.  With
    ``return_cache`` also the forward cache (per layer: input, pre-activation)
    and the gradient of the loss with respect to each layer's pre-activation
    (the tests derive their tolerances from these)."""
    logits, cache = forward(Ws, bs, X)
    B = X.shape[0]
    d = np.zeros_like(logits)
    loss = 0.0
    for h in range(HEADS):
        lg = logits[:, h * BINS:(h + 1) * BINS]
        mx = lg.max(axis=1, keepdims=True)
        lz = mx[:, 0] + np.log(np.exp(lg - mx).sum(axis=1))
        t = targets[:, h]
        loss += (lz - lg[np.arange(B), t]).sum()
        p = np.exp(lg - lz[:, None])
        p[np.arange(B), t] -= 1.0
        d[:, h * BINS:(h + 1) * BINS] = p / B
    dWs, dbs = [None] * len(Ws), [None] * len(Ws)
    deltas = [None] * len(Ws)
    delta = d
    for li in range(len(Ws) - 1, -1, -1):
        hin, pre = cache[li]
        deltas[li] = delta
        dWs[li] = delta.T @ hin
        dbs[li] = delta.sum(axis=0)
        if li > 0:
            _, pre_prev = cache[li - 1]
            delta = (delta @ Ws[li]) * gelu_grad(pre_prev)
    if return_cache:
        return loss / B, dWs, dbs, cache, deltas
    return loss / B, dWs, dbs
