"""Learned one-day emulator for SISe3 nodes (an extension of the method; the
paper has no emulator).

For a node inside the emulator's range, a small MLP predicts the
distribution of each age class's one-day increment of I from the node's
counts, phi and the six rate parameters; sampling it replaces that node's
direct SSA for the day.  Within a day phi is constant, so under the SSA the
three age classes are independent birth-death chains: three independent
129-bin heads (increments -64 .. 64) describe the joint law exactly, and
moving S opposite to I keeps every age class's size, as the SSA does.

Training data are one-day SSA outcomes generated by this library's own
kernels; the network is trained by this library's own tensor-core forward
and backward kernels and Adam kernel (all through the C ABI).  This module
only allocates tensors and sequences those calls.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import binding
from . import workloads as W

NIN, HID, NOUT, NUSED, BINS, HALF = 16, 256, 392, 387, 129, 64
DIMS = [(HID, NIN), (HID, HID), (HID, HID), (NOUT, HID)]  # (out, in) per layer


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _s():
    return binding._stream_handle(None)


def _check(rc):
    if rc:
        raise binding.SimInfError(rc)


class Emulator:
    """Weights (FP32 master copies, BF16 copies used by the kernels, FP32
    biases) and Adam state of the 16-256-256-256-392 MLP."""

    def __init__(self, device="cuda", seed=0):
        import torch
        self.torch = torch
        self.device = device
        g = torch.Generator(device="cpu").manual_seed(seed)
        self.W32, self.b32, self.W16 = [], [], []
        for li, (o, i) in enumerate(DIMS):
            std = math.sqrt(2.0 / i) * (0.25 if li == 3 else 1.0)
            w = torch.randn(o, i, generator=g) * std
            if li == 3:
                w[NUSED:] = 0.0  # padding outputs stay zero
            self.W32.append(w.float().to(device).contiguous())
            self.b32.append(torch.zeros(o, dtype=torch.float32, device=device))
            self.W16.append(self.W32[-1].to(torch.bfloat16).contiguous())
        self.mW = [torch.zeros_like(w) for w in self.W32]
        self.vW = [torch.zeros_like(w) for w in self.W32]
        self.mb = [torch.zeros_like(b) for b in self.b32]
        self.vb = [torch.zeros_like(b) for b in self.b32]
        self.step = 0

    # -- forward -------------------------------------------------------------
    def forward(self, feat16, keep=False):
        """Logits (B x 392 FP32); with keep=True also the activations and
        pre-activations the backward pass needs."""
        x = feat16
        acts, pres = [feat16], []
        for li in range(3):
            pre, post = binding.gemm_bf16(x, self.W16[li], bias=self.b32[li], act=1,
                                          out32=keep, out16=True)
            pres.append(pre)
            acts.append(post)
            x = post
        logits, _ = binding.gemm_bf16(x, self.W16[3], bias=self.b32[3], act=0,
                                      out32=True, out16=False)
        return logits, acts, pres

    # -- FP8 inference ---------------------------------------------------------
    def quantize_fp8(self, calib_feat16, margin=1.0):
        """E4M3 copies of the weights of layers 2-4 (one scale per output row,
        max |w| / 448) and static scales of their input activations (max
        |activation| of the BF16 network over the calibration features, times
        margin, / 448).  Layer 1 keeps BF16 operands (its inputs are the
        features) and writes its output in E4M3."""
        self.W8, self.wscale = [], []
        for li in (1, 2, 3):
            w8, sc = binding.quant_fp8_rows(self.W32[li])
            self.W8.append(w8)
            self.wscale.append(sc)
        _, acts, _ = self.forward(calib_feat16)
        f32 = np.float32
        self.act_scale = [float(f32(max(binding.absmax_bf16(a), 1e-30) * margin) / f32(448.0))
                          for a in acts[1:4]]

    def _inv(self, li):
        # the same single-precision reciprocal the engine takes
        return float(np.float32(1.0) / np.float32(self.act_scale[li]))

    def forward_fp8(self, feat16):
        """Logits (B x 392 FP32) of the E4M3 network: the same kernels and
        arguments the engine uses when FP8 inference is switched on."""
        x8 = binding.gemm_bf16_to_fp8(feat16, self.W16[0], self._inv(0), bias=self.b32[0],
                                      act=1)
        for li in (1, 2):
            _, _, x8 = binding.gemm_fp8(x8, self.act_scale[li - 1], self.W8[li - 1],
                                        self.wscale[li - 1], bias=self.b32[li], act=1,
                                        out32=False, out8_inv_scale=self._inv(li))
        logits, _, _ = binding.gemm_fp8(x8, self.act_scale[2], self.W8[2], self.wscale[2],
                                        bias=self.b32[3], act=0, out32=True)
        return logits

    # -- backward ------------------------------------------------------------
    def gradients(self, feat16, targets):
        """Mean cross-entropy and its gradients (dW per layer FP32 out x in,
        db per layer), all on the GPU."""
        torch = self.torch
        L = binding.lib()
        B = feat16.shape[0]
        logits, acts, pres = self.forward(feat16, keep=True)
        dlog = torch.empty((B, NOUT), dtype=torch.bfloat16, device=self.device)
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        _check(L.sg_mlp_ce_loss(_p(logits), NOUT, _p(targets), B, _p(dlog), NOUT, _p(loss),
                                _s()))
        dW, db = [None] * 4, [None] * 4
        delta = dlog
        for li in (3, 2, 1, 0):
            o, i = DIMS[li]
            dT = torch.empty((o, B), dtype=torch.bfloat16, device=self.device)
            aT = torch.empty((i, B), dtype=torch.bfloat16, device=self.device)
            _check(L.sg_transpose_bf16(_p(delta), B, o, _p(dT), _s()))
            _check(L.sg_transpose_bf16(_p(acts[li]), B, i, _p(aT), _s()))
            dW[li], _ = binding.gemm_bf16(dT, aT, out32=True)
            db[li] = torch.empty(o, dtype=torch.float32, device=self.device)
            _check(L.sg_colsum_bf16(_p(delta), B, o, _p(db[li]), _s()))
            if li > 0:
                WT = torch.empty((i, o), dtype=torch.bfloat16, device=self.device)
                _check(L.sg_transpose_bf16(_p(self.W16[li]), o, i, _p(WT), _s()))
                dpost, _ = binding.gemm_bf16(delta, WT, out32=True)
                nxt = torch.empty((B, i), dtype=torch.bfloat16, device=self.device)
                _check(L.sg_gelu_backward(_p(dpost), _p(pres[li - 1]), B * i, _p(nxt), _s()))
                delta = nxt
        return float(loss.item()) / B, dW, db

    def adam(self, dW, db, lr, b1=0.9, b2=0.999, eps=1e-8):
        L = binding.lib()
        self.step += 1
        for li in range(4):
            _check(L.sg_adam_step(_p(self.W32[li]), _p(dW[li]), _p(self.mW[li]),
                                  _p(self.vW[li]), self.W32[li].numel(), lr, b1, b2, eps,
                                  self.step, _p(self.W16[li]), _s()))
            _check(L.sg_adam_step(_p(self.b32[li]), _p(db[li]), _p(self.mb[li]),
                                  _p(self.vb[li]), self.b32[li].numel(), lr, b1, b2, eps,
                                  self.step, None, _s()))

    def train(self, feat16, targets, steps, batch=4096, lr=2e-3, lr_min=1e-4, seed=0,
              log_every=0):
        """Mini-batch Adam with a cosine learning-rate decay; returns the
        loss history."""
        torch = self.torch
        n = feat16.shape[0]
        g = torch.Generator(device="cpu").manual_seed(seed)
        hist = []
        for s in range(steps):
            idx = torch.randint(0, n, (batch,), generator=g).to(self.device)
            f = feat16.index_select(0, idx).contiguous()
            t = targets.index_select(0, idx).contiguous()
            loss, dW, db = self.gradients(f, t)
            rate = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * s / max(1, steps)))
            self.adam(dW, db, rate)
            hist.append(loss)
            if log_every and s % log_every == 0:
                print(f"step {s} loss {loss:.4f} lr {rate:.2e}", flush=True)
        return hist

    def state_dict(self):
        return {"W32": [w.cpu() for w in self.W32], "b32": [b.cpu() for b in self.b32]}


# ---------------------------------------------------------------------------
# Training data: one-day SSA outcomes of random SISe3 nodes.
# ---------------------------------------------------------------------------

def random_states(rng, n, max_herd=2000):
    """SISe3 node states inside the emulator's range: log-normal herds
    (median 60, sigma 1.2, clamp 1..max_herd) split 0.2 / 0.2 / 0.6 by age,
    a per-node infected fraction (0 for 30% of nodes, else uniform up to
    0.7) and phi near its equilibrium 10 I / N, clipped to [0, 6]."""
    herd = np.clip(np.rint(np.exp(np.log(60) + 1.2 * rng.standard_normal(n))), 1,
                   max_herd).astype(np.int64)
    ages = W.split_ages(herd)
    frac = np.where(rng.random(n) < 0.3, 0.0, rng.uniform(0, 0.7, n))
    I = np.minimum(ages, np.rint(ages * frac[:, None]
                                 * rng.uniform(0.7, 1.3, (n, 3))).astype(np.int64))
    S = ages - I
    u0 = np.stack([S[:, 0], I[:, 0], S[:, 1], I[:, 1], S[:, 2], I[:, 2]], 1).astype(np.int32)
    tot = np.maximum(1, herd)
    phi = np.clip(10.0 * I.sum(1) / tot * rng.uniform(0.5, 1.5, n)
                  + 0.3 * rng.random(n), 0.0, 6.0)
    return u0, phi


def random_params(rng):
    """Rate parameters jittered +-50% around upsilon 0.0173, gamma 0.1."""
    ups = 0.0173 * rng.uniform(0.5, 1.5, 3)
    gam = 0.1 * rng.uniform(0.5, 1.5, 3)
    # alpha = 0 and no decay: phi stays as given through the day
    return W.sise3_gdata(upsilons=ups, gammas=gam, alpha=0.0, betas=(0.0,) * 4)


def ssa_one_day(u0, phi, gdata, seed, n_rep=1):
    """Run the SSA for one day on the GPU; returns (U device tensor
    (n_rep, 2, n, 6), workload)."""
    import torch
    n = u0.shape[0]
    w = W.plain_model(W.SISE3, u0, np.array([0, 1]), gdata, seed=seed, n_rep=n_rep,
                      v0=phi[:, None])
    m = binding.Model(w)
    try:
        u0d = torch.as_tensor(np.ascontiguousarray(w.u0), device="cuda")
        v0d = torch.as_tensor(np.ascontiguousarray(w.v0), device="cuda")
        U = torch.empty((n_rep, 2, n, 6), dtype=torch.int32, device="cuda")
        V = torch.empty((n_rep, 2, n, 1), dtype=torch.float64, device="cuda")
        m.run(w.tspan, seed, n_rep, u0d, v0d, U, V)
    finally:
        m.close()
    return U, w


def features(u, phi, gdata, max_herd=2000, phi_lo=0.0, phi_hi=6.0, min_rate=0.0):
    """Emulator features (BF16, n x 16) and range flags from device state."""
    import torch
    n = u.shape[0]
    feat = torch.empty((n, NIN), dtype=torch.bfloat16, device="cuda")
    flag = torch.empty(n, dtype=torch.int32, device="cuda")
    g = np.ascontiguousarray(gdata, dtype=np.float64)
    _check(binding.lib().sg_emu_features(_p(u), _p(phi), n,
                                          ctypes.c_void_p(g.ctypes.data), int(max_herd),
                                          float(phi_lo), float(phi_hi), float(min_rate),
                                          _p(feat), _p(flag), _s()))
    return feat, flag


def total_rate(u0, phi, gdata):
    """A node's total transition rate per day (numpy): sum over age classes
    of upsilon_a phi S_a + gamma_a I_a."""
    g = np.asarray(gdata, dtype=np.float64)
    S, I = u0[:, 0::2].astype(np.float64), u0[:, 1::2].astype(np.float64)
    return (g[None, 0:3] * phi[:, None] * S + g[None, 3:6] * I).sum(axis=1)


def sample_increments(logits, u, flag, seed, day, n_nodes=None):
    """Sampled one-day increments (units x 4: dI_1..dI_3, used) of the
    flagged units from the logits, with the engine's random stream for
    `day` (unit i = replicate * n_nodes + node)."""
    import torch
    units = u.shape[0]
    delta = torch.empty((units, 4), dtype=torch.int32, device="cuda")
    _check(binding.lib().sg_emu_sample(_p(logits), int(logits.shape[1]), _p(u), _p(flag),
                                        int(units), int(n_nodes or units),
                                        ctypes.c_uint64(int(seed)), int(day), _p(delta), _s()))
    return delta


def make_dataset(n_nodes, n_batches, seed=0, max_herd=2000):
    """(features BF16, target bins int32) of n_nodes x n_batches one-day SSA
    outcomes, each batch with its own jittered rate parameters."""
    import torch
    rng = np.random.default_rng(seed)
    feats, tgts = [], []
    for b in range(n_batches):
        u0, phi = random_states(rng, n_nodes, max_herd)
        g = random_params(rng)
        U, w = ssa_one_day(u0, phi, g, seed=10_000 + 7919 * seed + b)
        ub = U[0, 0].contiguous()
        ua = U[0, 1].contiguous()
        phid = torch.as_tensor(phi, device="cuda")
        f, _ = features(ub, phid, g, max_herd)
        t = torch.empty((n_nodes, 3), dtype=torch.int32, device="cuda")
        _check(binding.lib().sg_emu_targets(_p(ub), _p(ua), n_nodes, _p(t), _s()))
        feats.append(f)
        tgts.append(t)
    return torch.cat(feats), torch.cat(tgts)


def trajectory_states(U, V, gdata, n, seed=0, max_herd=2000, phi_hi=6.0, min_rate=0.0):
    """n node-day start states (u int32 (n, 6), phi (n,)) drawn uniformly,
    with replacement, from the in-range node-days of an SSA trajectory
    (device U (1, M, N, 6) int32 and V (1, M, N, 1) float64 of one run): the
    states the emulator meets on that workload.  None if none is in range."""
    import torch
    u = U[0, :-1].reshape(-1, 6)
    phi = V[0, :-1].reshape(-1)
    g = torch.as_tensor(np.asarray(gdata, np.float64), device=U.device)
    a0 = (g[0:3] * phi[:, None] * u[:, 0::2].double() + g[3:6] * u[:, 1::2].double()).sum(1)
    ok = (u.sum(1) <= max_herd) & (phi >= 0) & (phi <= phi_hi) & (a0 >= min_rate)
    idx = torch.nonzero(ok).flatten()
    if idx.numel() == 0:
        return None
    gen = torch.Generator(device=U.device).manual_seed(seed)
    pick = idx[torch.randint(0, idx.numel(), (n,), device=U.device, generator=gen)]
    return u[pick].cpu().numpy().astype(np.int32), phi[pick].cpu().numpy()


def make_dataset_from_states(u_pool, phi_pool, gdata, n_nodes, n_batches, seed=0,
                             max_herd=2000):
    """(features, target bins) of one-day SSA outcomes from given start
    states (consecutive slices of the pools, n_nodes per batch) under the
    workload's own rate parameters."""
    import torch
    feats, tgts = [], []
    for b in range(n_batches):
        u0 = np.ascontiguousarray(u_pool[b * n_nodes:(b + 1) * n_nodes])
        phi = np.ascontiguousarray(phi_pool[b * n_nodes:(b + 1) * n_nodes])
        U, w = ssa_one_day(u0, phi, gdata, seed=20_000 + 7919 * seed + b)
        ub, ua = U[0, 0].contiguous(), U[0, 1].contiguous()
        f, _ = features(ub, torch.as_tensor(phi, device="cuda"), gdata, max_herd)
        t = torch.empty((len(u0), 3), dtype=torch.int32, device="cuda")
        _check(binding.lib().sg_emu_targets(_p(ub), _p(ua), len(u0), _p(t), _s()))
        feats.append(f)
        tgts.append(t)
    return torch.cat(feats), torch.cat(tgts)


# ---------------------------------------------------------------------------
# Error against SSA ensembles: Wasserstein-1 and Kolmogorov-Smirnov.
# ---------------------------------------------------------------------------

def emulator_pmf(emu, u0, phi, gdata, fp8=False):
    """The emulator's law of each age class's increment (n x 3 x 129), with
    the mass beyond -I_a .. S_a moved to those bounds as the sampler does
    (fp8: the E4M3 network)."""
    import torch
    ud = torch.as_tensor(u0, device="cuda")
    f, _ = features(ud, torch.as_tensor(phi, device="cuda"), gdata)
    logits = emu.forward_fp8(f) if fp8 else emu.forward(f)[0]
    lg = logits[:, :NUSED].double().cpu().numpy().reshape(-1, 3, BINS)
    lg = lg - lg.max(axis=2, keepdims=True)
    p = np.exp(lg)
    p /= p.sum(axis=2, keepdims=True)
    d = np.arange(BINS) - HALF
    for a in range(3):
        lo, hi = -u0[:, 2 * a + 1], u0[:, 2 * a]
        for k in range(p.shape[0]):
            below = d < lo[k]
            above = d > hi[k]
            if below.any():
                p[k, a, np.searchsorted(d, lo[k])] += p[k, a, below].sum()
                p[k, a, below] = 0
            if above.any():
                p[k, a, np.searchsorted(d, hi[k])] += p[k, a, above].sum()
                p[k, a, above] = 0
    return p


def compare_with_ssa(emu, n_probes=1000, n_rep=1000, seed=5, max_herd=2000, fp8=False,
                     min_rate=0.0):
    """W1 and KS between the emulator's law and 1,000-replicate SSA ensembles
    at n_probes random in-range states (total rate >= min_rate), per age
    class's I (S moves by the same amount, so its distances are the same).
    Returns a dict of mean and max over probes."""
    rng = np.random.default_rng(seed)
    g = random_params(rng)
    us, ps, have = [], [], 0
    while have < n_probes:
        u, p = random_states(rng, 4 * n_probes, max_herd)
        keep = total_rate(u, p, g) >= min_rate
        us.append(u[keep])
        ps.append(p[keep])
        have += int(keep.sum())
    u0 = np.concatenate(us)[:n_probes]
    phi = np.concatenate(ps)[:n_probes]
    res = compare_at_states(emu, u0, phi, g, n_rep=n_rep, seed=seed, fp8=fp8)
    res["min_rate"] = float(min_rate)
    return res


def compare_at_states(emu, u0, phi, g, n_rep=1000, seed=5, fp8=False):
    """W1 and KS between the emulator's law and n_rep-replicate SSA
    ensembles at the given start states (rate parameters g), per age
    class's I."""
    n_probes = len(u0)
    U, w = ssa_one_day(u0, phi, g, seed=777 + seed, n_rep=n_rep)
    Ua = U[:, 1].cpu().numpy()  # (n_rep, n, 6)
    p = emulator_pmf(emu, u0, phi, g, fp8=fp8)
    d = np.arange(BINS) - HALF
    w1 = np.zeros((n_probes, 3))
    ks = np.zeros((n_probes, 3))
    for a in range(3):
        inc = Ua[:, :, 2 * a + 1] - u0[None, :, 2 * a + 1]  # (n_rep, n)
        inc = np.clip(inc, -HALF, HALF)
        for k in range(n_probes):
            emp = np.bincount(inc[:, k] + HALF, minlength=BINS) / n_rep
            cdf_e, cdf_m = np.cumsum(emp), np.cumsum(p[k, a])
            w1[k, a] = np.abs(cdf_e - cdf_m).sum()  # bins are one individual wide
            ks[k, a] = np.abs(cdf_e - cdf_m).max()
    return {"w1_mean": float(w1.mean()), "w1_max": float(w1.max()),
            "w1_per_age": w1.mean(0).tolist(), "ks_mean": float(ks.mean()),
            "ks_max": float(ks.max()), "probes": n_probes, "replicates": n_rep,
            "increments": d.tolist()[:1] + d.tolist()[-1:]}
