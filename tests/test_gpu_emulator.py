"""The learned one-day emulator: logits of the BF16 and E4M3 networks and the
gradients of the tensor-core training path against the FP64 oracle network,
element by element (tolerances from tests/mlp_tolerance.py), the optimiser,
the sampler, training on SSA-generated data to the W1 <= 0.5 target, and the
engine's use of the emulator with SSA fallback."""
import numpy as np
import pytest

from paper_1605_01421_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_01421_gb300 import binding, emulator
    binding.build()
    return torch, binding, emulator


def _net_inputs(torch, emulator, emu, n, seed):
    """Features of random in-range SISe3 states (the emulator's own inputs)
    and random biases (the initial ones are zero), so that every term of
    each layer is exercised."""
    rng = np.random.default_rng(seed)
    u0, phi = emulator.random_states(rng, n)
    g = emulator.random_params(rng)
    f, flag = emulator.features(torch.as_tensor(u0, device="cuda"),
                                torch.as_tensor(phi, device="cuda"), g)
    for li, b in enumerate(emu.b32):
        b.copy_(torch.as_tensor(rng.normal(0, 0.2, b.numel()), dtype=torch.float32))
    return f, rng


def _oracle_weights(emu):
    return ([w.double().cpu().numpy() for w in emu.W16],
            [b.double().cpu().numpy() for b in emu.b32])


def test_bf16_logits_match_fp64_oracle_per_element(env):
    # the BF16 network (four tcgen05 GEMMs with bias and GELU epilogues) vs
    # the FP64 network on the same BF16 weights and inputs, every logit
    # within its propagated rounding tolerance
    torch, binding, emulator = env
    from oracle import mlp
    import mlp_tolerance as tol
    emu = emulator.Emulator(seed=1)
    f, _ = _net_inputs(torch, emulator, emu, 3000, 41)  # 23 full tiles + a ragged one
    logits = emu.forward(f)[0].double().cpu().numpy()
    Ws, bs = _oracle_weights(emu)
    X = f.double().cpu().numpy()
    ref, _ = mlp.forward(Ws, bs, X)
    Vz, _ = tol.forward_variances(Ws, bs, X, "bf16")
    tol.check(logits[:, :mlp.HEADS * mlp.BINS], ref[:, :mlp.HEADS * mlp.BINS],
              Vz[-1][:, :mlp.HEADS * mlp.BINS], "BF16 logits")


def test_fp8_logits_match_fp64_oracle_per_element(env):
    # the E4M3 network (layer 1 BF16 operands, E4M3 output; layers 2-4 E4M3
    # operands with per-row weight scales and static activation scales) vs
    # the FP64 network on the dequantised weights, every logit within its
    # propagated rounding tolerance (E4M3 storage of the activations
    # dominates).  The engine's persistent chain samples from exactly these
    # logits (tested bit for bit below).
    torch, binding, emulator = env
    from oracle import mlp
    import mlp_tolerance as tol
    emu = emulator.Emulator(seed=2)
    f, _ = _net_inputs(torch, emulator, emu, 3000, 42)
    emu.quantize_fp8(f)
    logits = emu.forward_fp8(f).double().cpu().numpy()
    Ws = [emu.W16[0].double().cpu().numpy()]
    for li in range(3):
        w8 = emu.W8[li].cpu().view(torch.float8_e4m3fn).double()
        Ws.append((w8 * emu.wscale[li].cpu().double()[:, None]).numpy())
    bs = [b.double().cpu().numpy() for b in emu.b32]
    X = f.double().cpu().numpy()
    ref, _ = mlp.forward(Ws, bs, X)
    Vz, _ = tol.forward_variances(Ws, bs, X, "e4m3", emu.act_scale)
    n = mlp.HEADS * mlp.BINS
    tol.check(logits[:, :n], ref[:, :n], Vz[-1][:, :n], "E4M3 logits")


def test_gradients_match_fp64_oracle_per_element(env):
    # loss, dW and db of the training path (BF16 storage, FP32 accumulation:
    # loss kernel, transposes, GEMMs, GELU backward, column sums) vs the FP64
    # oracle's backpropagation, element by element within the propagated
    # rounding tolerance
    torch, binding, emulator = env
    import mlp_tolerance as tol
    emu = emulator.Emulator(seed=1)
    f, rng = _net_inputs(torch, emulator, emu, 512, 43)
    t = torch.as_tensor(rng.integers(40, 90, (512, 3)), dtype=torch.int32).cuda()
    loss, dW, db = emu.gradients(f, t)
    Ws, bs = _oracle_weights(emu)
    (ref_loss, rdW, rdb), VdW, Vdb = tol.gradient_variances(Ws, bs, f.double().cpu().numpy(),
                                                            t.cpu().numpy())
    # the loss (about 3 ln 129 per row, a mean over 512 rows of sums of
    # logits whose errors are ~1e-3 each) is expected within ~1e-4
    # relative; 1e-3 leaves room for the FP32 exponentials and logarithms
    assert abs(loss - ref_loss) <= 1e-3 * abs(ref_loss), (loss, ref_loss)
    for li in range(4):
        tol.check(dW[li].double().cpu().numpy(), rdW[li], VdW[li], f"dW layer {li + 1}")
        tol.check(db[li].double().cpu().numpy(), rdb[li], Vdb[li], f"db layer {li + 1}")


def test_adam_step_matches_definition(env):
    torch, binding, emulator = env
    import ctypes
    L = binding.lib()
    n = 1000
    g = torch.Generator().manual_seed(0)
    p = torch.randn(n, generator=g).cuda()
    gr = torch.randn(n, generator=g).cuda()
    m = torch.randn(n, generator=g).cuda() * 0.1
    v = torch.rand(n, generator=g).cuda() * 0.1
    p0, m0, v0 = p.clone(), m.clone(), v.clone()
    p16 = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    rc = L.sg_adam_step(ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(gr.data_ptr()),
                        ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(v.data_ptr()), n, 1e-2,
                        0.9, 0.999, 1e-8, 3, ctypes.c_void_p(p16.data_ptr()),
                        binding._stream_handle(None))
    assert rc == 0
    m1 = 0.9 * m0 + 0.1 * gr
    v1 = 0.999 * v0 + 0.001 * gr * gr
    p1 = p0 - 1e-2 * (m1 / (1 - 0.9 ** 3)) / (torch.sqrt(v1 / (1 - 0.999 ** 3)) + 1e-8)
    assert torch.allclose(p, p1, rtol=1e-5, atol=1e-6)
    assert torch.allclose(p16.float(), p1, rtol=1e-2, atol=1e-2)


def test_sampler_law_and_clamping(env):
    torch, binding, emulator = env
    import ctypes
    stats = pytest.importorskip("scipy.stats")
    L = binding.lib()
    units = 20000
    rng = np.random.default_rng(3)
    row = rng.normal(0, 1.5, 392).astype(np.float32)
    logits = torch.as_tensor(np.tile(row, (units, 1))).cuda()
    u = np.tile(np.array([[100, 100, 3, 2, 100, 100]], np.int32), (units, 1))
    ud = torch.as_tensor(u).cuda()
    flag = torch.ones(units, dtype=torch.int32, device="cuda")
    flag[::7] = 0
    delta = torch.full((units, 4), -99, dtype=torch.int32, device="cuda")
    rc = L.sg_emu_sample(ctypes.c_void_p(logits.data_ptr()), 392, ctypes.c_void_p(ud.data_ptr()),
                         ctypes.c_void_p(flag.data_ptr()), units, units, 11, 5,
                         ctypes.c_void_p(delta.data_ptr()), binding._stream_handle(None))
    assert rc == 0
    dl = delta.cpu().numpy()
    used = dl[:, 3] == 1
    assert np.array_equal(used, flag.cpu().numpy() == 1)
    # head 0: increments within [-100, 100] are not clamped: chi-square
    # against the softmax law of the row
    r64 = row[:129].astype(np.float64)
    p = np.exp(r64 - r64.max())
    p /= p.sum()
    obs = np.bincount(dl[used, 0] + 64, minlength=129).astype(float)
    keep = p * used.sum() >= 5
    exp = p * used.sum()
    obs_k = np.r_[obs[keep], obs[~keep].sum()]
    exp_k = np.r_[exp[keep], exp[~keep].sum()]
    exp_k *= obs_k.sum() / exp_k.sum()
    assert stats.chisquare(obs_k, exp_k).pvalue > 1e-3
    # head 1: S = 3, I = 2 bounds the increment to -2 .. 3
    assert dl[used, 1].min() >= -2 and dl[used, 1].max() <= 3


def test_engine_without_emulated_nodes_equals_ssa(env, orc):
    # with no node in range every node falls back to the SSA: bit-exact
    torch, binding, emulator = env
    w = W.config_sise3(n_nodes=600, days=40, gen_seed=14)
    emu = emulator.Emulator(seed=0)
    code, U0, V0, R0, err = orc.run(w)
    m = binding.Model(w)
    m.set_emulator(emu, max_herd=-1)
    u0, v0 = (torch.as_tensor(np.ascontiguousarray(a), device="cuda") for a in (w.u0, w.v0))
    M = len(w.tspan)
    U = torch.empty((1, M, w.n_nodes, 6), dtype=torch.int32, device="cuda")
    V = torch.empty((1, M, w.n_nodes, 1), dtype=torch.float64, device="cuda")
    rc, st, er = m.run(w.tspan, w.seed, 1, u0, v0, U, V)
    assert np.array_equal(U.cpu().numpy(), U0)
    assert np.array_equal(V.cpu().numpy().view(np.uint64), V0.view(np.uint64))


def test_training_and_emulated_run(env):
    torch, binding, emulator = env
    feat, tgt = emulator.make_dataset(500_000, 8, seed=1)
    emu = emulator.Emulator(seed=0)
    hist = emu.train(feat, tgt, steps=2500, batch=8192, lr=2e-3)
    assert np.mean(hist[-50:]) < 0.7 * np.mean(hist[:10])
    # the target: W1 <= 0.5 individuals per compartment per node-day against
    # SSA ensembles
    res = emulator.compare_with_ssa(emu, n_probes=200, n_rep=1000, seed=9)
    assert res["w1_mean"] <= 0.5, res
    # the engine with the emulator: populations per age class stay exact
    w = W.config_sise3(n_nodes=3000, days=60, gen_seed=15, events_per_node_day=0)
    m = binding.Model(w)
    m.set_emulator(emu, max_herd=2000)
    u0, v0 = (torch.as_tensor(np.ascontiguousarray(a), device="cuda") for a in (w.u0, w.v0))
    M = len(w.tspan)
    U = torch.empty((1, M, w.n_nodes, 6), dtype=torch.int32, device="cuda")
    V = torch.empty((1, M, w.n_nodes, 1), dtype=torch.float64, device="cuda")
    rc, st, er = m.run(w.tspan, w.seed, 1, u0, v0, U, V)
    Uc = U.cpu().numpy()[0]
    assert Uc.min() >= 0
    for a in range(3):
        tot = Uc[:, :, 2 * a] + Uc[:, :, 2 * a + 1]
        assert np.all(tot == tot[0:1])
    # the same run with E4M3 layers 2-4 (the persistent tensor-core chain)
    emu.quantize_fp8(feat[:65536].contiguous())
    m.set_emulator_fp8(emu)
    rc, st, er = m.run(w.tspan, w.seed, 1, u0, v0, U, V)
    U8 = U.cpu().numpy()[0]
    assert U8.min() >= 0 and not np.array_equal(U8, Uc)
    for a in range(3):
        tot = U8[:, :, 2 * a] + U8[:, :, 2 * a + 1]
        assert np.all(tot == tot[0:1])
    # the prevalence of the two runs stays close (both emulate the same law)
    p16 = (Uc[-1, :, 1::2].sum(1) > 0).mean()
    p8 = (U8[-1, :, 1::2].sum(1) > 0).mean()
    assert abs(p16 - p8) < 0.05, (p16, p8)


def test_engine_day_equals_sampled_network_bf16_and_fp8(env):
    # one day, every node inside the emulator's range: the engine's state
    # after the day is the start state moved by the sampler's increments for
    # the logits of the network computed on its own (BF16, then E4M3 layers
    # 2-4 with static activation scales), bit for bit
    torch, binding, emulator = env
    rng = np.random.default_rng(21)
    n, seed = 5000, 0x0123_4567_89AB
    u0, phi = emulator.random_states(rng, n)
    g = emulator.random_params(rng)
    emu = emulator.Emulator(seed=3)
    ud = torch.as_tensor(u0, device="cuda")
    f, flag = emulator.features(ud, torch.as_tensor(phi, device="cuda"), g)
    assert bool((flag == 1).all())
    emu.quantize_fp8(f)
    assert all(s > 0 for s in emu.act_scale)
    l16 = emu.forward(f)[0]
    l8 = emu.forward_fp8(f)
    rel = ((l8 - l16).norm() / l16.norm()).item()
    assert rel < 0.1, rel
    for fp8, logits in ((False, l16), (True, l8)):
        w = W.plain_model(W.SISE3, u0, np.array([0, 1]), g, seed=seed, v0=phi[:, None])
        m = binding.Model(w)
        m.set_emulator(emu, max_herd=2000)
        if fp8:
            m.set_emulator_fp8(emu)
        u0d, v0d = (torch.as_tensor(np.ascontiguousarray(a), device="cuda") for a in (w.u0, w.v0))
        U = torch.empty((1, 2, n, 6), dtype=torch.int32, device="cuda")
        V = torch.empty((1, 2, n, 1), dtype=torch.float64, device="cuda")
        rc, st, er = m.run(w.tspan, seed, 1, u0d, v0d, U, V)
        m.close()
        delta = emulator.sample_increments(logits, ud, flag, seed, 1)
        d = delta.cpu().numpy()
        want = u0.astype(np.int64).copy()
        for a in range(3):
            want[:, 2 * a] -= d[:, a]
            want[:, 2 * a + 1] += d[:, a]
        assert np.array_equal(U.cpu().numpy()[0, 1], want), fp8
    # switching FP8 off and on again through the API
    m = binding.Model(w)
    with pytest.raises(binding.SimInfError):
        m.set_emulator_fp8(emu)  # no emulator set yet
    m.set_emulator(emu, max_herd=2000)
    m.set_emulator_fp8(emu)
    m.set_emulator_fp8(emu, enable=False)
    m.close()


@pytest.mark.parametrize("min_rate", [0.0, 3.0])
def test_fp8_chain_ragged_replicates_and_fallback(env, orc, min_rate):
    # 1,237 nodes (a ragged last tile), two replicates, 4% of the herds above
    # the emulator's range and (min_rate 3) the nodes with fewer than three
    # expected transitions a day on the SSA: emulated nodes equal the sampled
    # E4M3 network bit for bit, the others equal the oracle's SSA
    torch, binding, emulator = env
    rng = np.random.default_rng(33)
    n, R, seed = 1237, 2, 0x5EED_0F_C4A1
    u0, phi = emulator.random_states(rng, n)
    g = emulator.random_params(rng)
    quiet = emulator.total_rate(u0, phi, g) < min_rate
    big = rng.random(n) < 0.04
    u0[big, 4] += 2500
    big |= quiet
    if min_rate > 0:
        assert 0.1 < quiet.mean() < 0.9
    emu = emulator.Emulator(seed=4)
    uu = torch.as_tensor(np.tile(u0, (R, 1)), device="cuda")
    ph = torch.as_tensor(np.tile(phi, R), device="cuda")
    f, flag = emulator.features(uu, ph, g, min_rate=min_rate)
    assert np.array_equal(flag.cpu().numpy() == 1, np.tile(~big, R))
    emu.quantize_fp8(f)
    logits = emu.forward_fp8(f)
    delta = emulator.sample_increments(logits, uu, flag, seed, 1, n_nodes=n).cpu().numpy()
    w = W.plain_model(W.SISE3, u0, np.array([0, 1]), g, seed=seed, v0=phi[:, None], n_rep=R)
    code, U0, V0, R0, err = orc.run(w)
    assert code == 0
    m = binding.Model(w)
    m.set_emulator(emu, max_herd=2000, min_rate=min_rate)
    m.set_emulator_fp8(emu)
    u0d, v0d = (torch.as_tensor(np.ascontiguousarray(a), device="cuda") for a in (w.u0, w.v0))
    U = torch.empty((R, 2, n, 6), dtype=torch.int32, device="cuda")
    V = torch.empty((R, 2, n, 1), dtype=torch.float64, device="cuda")
    rc, st, er = m.run(w.tspan, seed, R, u0d, v0d, U, V)
    m.close()
    Ug = U.cpu().numpy()
    for r in range(R):
        d = delta[r * n:(r + 1) * n]
        assert np.array_equal(d[:, 3] == 1, ~big)
        want = u0.astype(np.int64).copy()
        for a in range(3):
            want[:, 2 * a] -= d[:, a]
            want[:, 2 * a + 1] += d[:, a]
        assert np.array_equal(Ug[r, 1][~big], want[~big]), r
        assert np.array_equal(Ug[r, 1][big], U0[r, 1][big]), r
