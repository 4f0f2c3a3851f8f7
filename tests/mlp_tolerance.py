"""Per-element tolerances for comparing the emulator network's tensor-core
kernels with the FP64 oracle network (``oracle/mlp.py``).  Test
infrastructure: these functions compute no expected value, only how far the
GPU's result may sit from the oracle's.

The GPU path differs from the FP64 network by rounding only: BF16 storage of
activations and gradients (unit roundoff 2^-8), E4M3 storage of activations in
the FP8 path (unit roundoff 2^-4 for normal values, half the subnormal step
2^-10 times the layer's scale below them), FP32 accumulation in the
tensor cores (2^-24 per addition; 2^-13 is assumed for E4M3 products, a
conservative figure), and the hardware tanh in GELU and its derivative
(relative error taken as 2^-10, twice the documented ~2^-11).  Each rounding
error is bounded by half a unit in the last place and treated as an
independent zero-mean error with variance (bound)^2 / 3 (uniform); the
variances are carried through the layers to first order:

  forward   Var dz_l = sum_k W_lk^2 Var dh_(l-1),k + accumulation,
            Var dh_l = gelu'(z_l)^2 Var dz_l + (GELU evaluation)^2 / 3
                       + (storage rounding)^2 / 3;
  loss      Var dp   = p^2 (Var dz + sum_j p_j^2 Var dz_j) for the softmax p
                       of a head, Var d_L = Var dp / B^2 + (BF16 storage)^2 / 3;
  backward  Var dW_l = Var d_l^T h^2 + d_l^2^T Var dh (+ accumulation),
            Var db_l = sum_b Var d_l,
            Var dpost = Var d_l W_l^2,
            Var d_(l-1) = gelu'(z)^2 Var dpost + dpost^2 (gelu''(z)^2 Var dz
                          + (tanh error through gelu')^2 / 3) + (BF16)^2 / 3.

A result element passes if |GPU - oracle| <= K_SIGMA sqrt(Var) + a floor of
1e-30; the worst-case (all errors of one sign) bound is far looser and, for
E4M3, larger than the values themselves, which is why the independent-error
form is used.  The tests also check that the measured errors are of the
predicted size (their root mean square within a factor of the predicted
one), so that the tolerance is neither vacuous nor violated on average.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import mlp

U16 = 2.0 ** -8       # BF16 unit roundoff (8 significant bits, nearest)
U8 = 2.0 ** -4        # E4M3 unit roundoff (4 significant bits, nearest)
E4M3_HALF_SUB = 2.0 ** -10  # half the E4M3 subnormal step (2^-9)
U32 = 2.0 ** -24      # FP32 unit roundoff
ET = 2.0 ** -10       # hardware tanh, relative error (documented ~2^-11)
UACC_F8 = 2.0 ** -13  # E4M3 tensor-core accumulation (conservative)
K_SIGMA = 8.0

_C = math.sqrt(2.0 / math.pi)
_A = 0.044715


def _gelu_dd(x):
    # second derivative of the tanh-form GELU (central difference of the
    # oracle's first derivative; only a tolerance depends on it)
    h = 1e-5
    return (mlp.gelu_grad(x + h) - mlp.gelu_grad(x - h)) / (2 * h)


def _acc_var(u, K, h_abs, W_abs, b_abs=0.0):
    return (u * u / 3.0) * K * (h_abs @ W_abs.T + b_abs) ** 2


def forward_variances(Ws, bs, X, store="bf16", scales=None):
    """Variances of the GPU's deviation from the FP64 network, per element:
    (Var of each layer's pre-activation, Var of each hidden activation as
    stored).  store = "bf16" (BF16 path) or "e4m3" (layer 1 BF16 operands,
    layers 2-4 E4M3 operands; ``scales`` = the three activation scales)."""
    _, cache = mlp.forward(Ws, bs, X)
    L = len(Ws)
    Vz, Vh = [], []
    vh = np.zeros_like(X)
    for li in range(L):
        W, b = Ws[li], bs[li]
        h_in, z = cache[li]
        uacc = UACC_F8 if (store == "e4m3" and li > 0) else U32
        vz = vh @ (W * W).T + _acc_var(uacc, W.shape[1], np.abs(h_in), np.abs(W), np.abs(b))
        vz = vz + (U32 * np.abs(z)) ** 2 / 3.0  # scale and bias in FP32
        Vz.append(vz)
        if li < L - 1:
            g1 = mlp.gelu_grad(z)
            h = mlp.gelu(z)
            v = g1 * g1 * vz + (0.5 * np.abs(z) * ET) ** 2 / 3.0
            if store == "bf16":
                v = v + (U16 * np.abs(h)) ** 2 / 3.0
            else:
                s = scales[li]
                half_ulp = np.maximum(U8 * np.abs(h), E4M3_HALF_SUB * s)
                v = v + half_ulp ** 2 / 3.0
            Vh.append(v)
            vh = v
    return Vz, Vh


def gradient_variances(Ws, bs, X, targets):
    """Variances of the GPU's deviation from the FP64 gradients (dW, db per
    layer) for the BF16 training path; also returns the oracle's loss, dW
    and db."""
    loss, dWs, dbs, cache, deltas = mlp.loss_and_grads(Ws, bs, X, targets, return_cache=True)
    Vz, Vh = forward_variances(Ws, bs, X, "bf16")
    B = X.shape[0]
    L = len(Ws)
    logits = cache[-1][1]
    vz = Vz[-1]
    vp = np.zeros_like(logits)
    for h in range(mlp.HEADS):
        sl = slice(h * mlp.BINS, (h + 1) * mlp.BINS)
        lg = logits[:, sl]
        p = np.exp(lg - lg.max(axis=1, keepdims=True))
        p /= p.sum(axis=1, keepdims=True)
        cross = (p * p * vz[:, sl]).sum(axis=1, keepdims=True)
        vp[:, sl] = p * p * (vz[:, sl] + cross) + (4 * U32 * p) ** 2 / 3.0
    d = deltas[-1]
    vd = vp / (B * B) + (U16 * np.abs(d)) ** 2 / 3.0
    VdW, Vdb = [None] * L, [None] * L
    for li in range(L - 1, -1, -1):
        h_in = cache[li][0]
        vh_in = Vh[li - 1] if li > 0 else np.zeros_like(h_in)
        d = deltas[li]
        VdW[li] = (vd.T @ (h_in * h_in) + (d * d).T @ vh_in
                   + (U32 * U32 / 3.0) * B * (np.abs(d).T @ np.abs(h_in)) ** 2)
        Vdb[li] = vd.sum(axis=0) + (U32 * U32 / 3.0) * B * np.abs(d).sum(axis=0) ** 2
        if li > 0:
            W = Ws[li]
            dpost = d @ W
            vpost = vd @ (W * W) + (U32 * U32 / 3.0) * W.shape[0] * (np.abs(d) @ np.abs(W)) ** 2
            z = cache[li - 1][1]
            g1 = mlp.gelu_grad(z)
            t = np.tanh(_C * (z + _A * z ** 3))
            dg_dt = 0.5 - z * t * _C * (1.0 + 3.0 * _A * z * z)
            vg = _gelu_dd(z) ** 2 * Vz[li - 1] + (dg_dt * ET * np.abs(t)) ** 2 / 3.0
            vd = (g1 * g1 * vpost + dpost * dpost * vg
                  + (U16 * np.abs(deltas[li - 1])) ** 2 / 3.0)
    return (loss, dWs, dbs), VdW, Vdb


def check(got, ref, var, what, k=K_SIGMA, rms_lo=0.02, rms_hi=2.0):
    """Element-wise |got - ref| <= k sqrt(var), and the root mean square of
    the errors within [rms_lo, rms_hi] times that of sqrt(var)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    sd = np.sqrt(np.asarray(var, dtype=np.float64))
    err = np.abs(got - ref)
    bad = err > k * sd + 1e-30
    assert not bad.any(), (f"{what}: {int(bad.sum())} of {bad.size} elements beyond "
                           f"{k} sigma; worst ratio {float((err / (sd + 1e-300)).max()):.2f}")
    ratio = math.sqrt(float((err ** 2).mean())) / math.sqrt(float((sd ** 2).mean()))
    assert rms_lo <= ratio <= rms_hi, f"{what}: rms error / rms sigma = {ratio:.3g}"
    return ratio
