"""Parity of the CUDA path with the CPU oracle: bit-exact integer
trajectories U, bit-exact FP64 continuous state V (both sides evaluate the
same IEEE operations in the same order, no contraction), identical reaction
counts and identical error codes, on the same seeded inputs.

Sizes span several thread blocks and a ragged tail; the SISe workload with
scheduled events is run at its full size (1,600 nodes x 365 days, ~200k
events), the size the benchmark times.
"""
import numpy as np
import pytest

from paper_1605_01421_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EXIT, ENTER, INTERNAL, EXTERNAL = 0, 1, 2, 3


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_01421_gb300 import binding
    binding.build()
    binding.lib()
    return binding


def _compare(orc, gpu, w, n_rep=None, seed=None):
    code, U0, V0, R0, err0 = orc.run(w, seed=seed, n_rep=n_rep)
    assert code == 0, err0
    U1, V1, st = gpu.simulate(w, seed=seed, n_rep=n_rep)
    # count diverging node-trajectories before asserting, for the report
    diff_nodes = np.any(U0 != U1, axis=(1, 3)).sum()
    assert diff_nodes == 0, f"{diff_nodes} node trajectories diverge"
    assert np.array_equal(U0, U1)
    assert np.array_equal(V0.view(np.uint64), V1.view(np.uint64))
    assert st["reactions"] == int(R0.sum())
    return U0, V0, R0, st


def test_philox_matches_oracle(orc, gpu):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = [0, 0, 0, 0]
    ctr[1] = [0xFFFFFFFF] * 4
    key = 0x299F31D0A4093822
    out = gpu.philox_batch(ctr.ravel(), key).reshape(-1, 4)
    for i in range(0, 4096, 37):
        assert list(out[i]) == orc.philox4x32_10(list(ctr[i]),
                                                 [key & 0xFFFFFFFF, key >> 32])


def test_log_is_bit_identical_to_oracle(orc, gpu):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.random(200_000), np.exp(rng.uniform(-740, 709, 50_000)),
                        [2.0 ** -53, 1.0 - 2.0 ** -53, 1.0, 2.0, 0.5, 5e-324,
                         1.4142135623730951, 0.7071067811865476]])
    y = gpu.log_batch(x)
    ref = np.array([orc.log(v) for v in x])
    assert np.array_equal(y.view(np.uint64), ref.view(np.uint64))


def test_u01_is_bit_identical_to_oracle(orc, gpu):
    rng = np.random.default_rng(2)
    w = rng.integers(0, 2 ** 32, size=20_000, dtype=np.uint64).astype(np.uint32)
    w[:4] = [0, 0, 0xFFFFFFFF, 0xFFFFFFFF]
    y = gpu.u01_batch(w)
    ref = np.array([orc.u01(w[2 * i], w[2 * i + 1]) for i in range(len(w) // 2)])
    assert np.array_equal(y, ref)
    assert y.min() > 0.0 and y.max() < 1.0


def test_sir_plain(orc, gpu):
    # SIR, 100 nodes of S=99 I=1 R=0, beta 0.16, gamma 0.077, tspan 1..100,
    # seed 42, no events
    _compare(orc, gpu, W.config_sir())


def test_sir_ragged_many_blocks(orc, gpu):
    w = W.plain_model(W.SIR, np.tile([[995, 5, 0]], (1037, 1)), np.arange(3, 61),
                      [0.3, 0.1], seed=7)
    _compare(orc, gpu, w)


def test_sis_and_sparse_tspan(orc, gpu):
    w = W.plain_model(W.SIS, np.tile([[40, 2]], (300, 1)), np.arange(1, 181, 7),
                      [0.01, 0.3], seed=11)
    _compare(orc, gpu, w)


def test_sise_full_size_with_events(orc, gpu):
    # 1,600 nodes x 365 days, ~200k events: the benchmark workload
    w = W.config_sise()
    assert w.n_events > 150_000
    U0, V0, R0, st = _compare(orc, gpu, w)
    assert st["events_applied"] == w.n_events


def test_sise3_with_all_event_types(orc, gpu):
    w = W.config_sise3(n_nodes=2500, days=200, gen_seed=33,
                       events_per_node_day=0.2)
    assert set(np.unique(w.events["event"])) == {0, 1, 2, 3}
    _compare(orc, gpu, w)


def test_shared_events_many_replicates(orc, gpu):
    w = W.config_sise3(n_nodes=400, days=90, gen_seed=5, n_rep=6)
    _compare(orc, gpu, w)


def test_replicate_specific_events(orc, gpu):
    w = W.config_sise3(n_nodes=300, days=80, gen_seed=6, n_rep=5,
                       per_rep_events=True, median=50, sigma=1.0, hi=5000)
    assert w.events["rep"] is not None
    _compare(orc, gpu, w)


def test_five_node_scenario_replicates(orc, gpu):
    from test_oracle_paper import five_node_scenario
    _compare(orc, gpu, five_node_scenario(1000, seed=123))


def test_single_time_point_and_events_outside_window(orc, gpu):
    rows = [(ENTER, -5, 0, 0, 2, 0.0, 0, -1), (ENTER, 3, 1, 0, 4, 0.0, 0, -1),
            (EXIT, 50, 0, 0, 1, 0.0, 0, -1)]
    w = W.plain_model(W.SIR, [[10, 2, 0], [0, 0, 0]], np.array([2, 5, 9]),
                      [0.2, 0.1], seed=3, events=W.make_events(rows))
    _compare(orc, gpu, w)
    w1 = W.plain_model(W.SIR, [[10, 2, 0]], np.array([4]), [0.2, 0.1])
    _compare(orc, gpu, w1)


def test_proportion_events_and_self_transfer(orc, gpu):
    rows = [(EXIT, 2, 0, 0, 0, 0.37, 2, -1), (EXTERNAL, 2, 1, 1, 3, 0.0, 2, -1),
            (EXTERNAL, 3, 1, 0, 0, 0.5, 2, -1), (ENTER, 3, 2, 0, 9, 0.0, 1, -1),
            (EXTERNAL, 3, 2, 1, 0, 1.0, 2, -1)]
    g = W.sise_gdata(upsilon=0.05, gamma=0.2)
    w = W.plain_model(W.SISE, [[30, 5], [10, 10], [0, 0]], np.arange(0, 8), g,
                      seed=19, events=W.make_events(rows),
                      v0=np.array([[0.5], [1.0], [0.0]]))
    _compare(orc, gpu, w)


def test_hub_waves_preserve_list_order(orc, gpu):
    # many transfers out of and into one hub on the same day: long wave chains
    rng = np.random.default_rng(4)
    rows = []
    for T in range(1, 6):
        for _ in range(300):
            a, b = rng.integers(1, 200, 2)
            if rng.random() < 0.5:
                rows.append((EXTERNAL, T, 0, int(a), 1, 0.0, 2, -1))
            else:
                rows.append((EXTERNAL, T, int(b), 0, 1, 0.0, 2, -1))
    u0 = np.tile([[400, 40]], (200, 1))
    u0[0] = [5000, 500]
    w = W.plain_model(W.SISE, u0, np.arange(0, 6), W.sise_gdata(), seed=8,
                      events=W.make_events(rows), v0=np.full((200, 1), 0.3))
    _compare(orc, gpu, w)


def test_event_underflow_reports_same_error(orc, gpu):
    rows = [(ENTER, 1, 0, 0, 2, 0.0, 0, -1), (EXIT, 2, 0, 0, 50, 0.0, 2, -1)]
    w = W.plain_model(W.SISE, [[5, 0], [5, 0]], np.arange(0, 5), W.sise_gdata(),
                      events=W.make_events(rows))
    code, U, V, R, err = orc.run(w)
    assert code == -2 and err["event"] == 1 and err["day"] == 2
    m = gpu.Model(w)
    import torch
    u0 = torch.as_tensor(w.u0, device="cuda")
    v0 = torch.as_tensor(w.v0, device="cuda")
    Ud = torch.empty((1, 5, 2, 2), dtype=torch.int32, device="cuda")
    Vd = torch.empty((1, 5, 2, 1), dtype=torch.float64, device="cuda")
    rc, st, er = m.run(w.tspan, w.seed, 1, u0, v0, Ud, Vd, check=False)
    assert rc == -2 and er["event"] == 1 and er["day"] == 2 and er["node"] == 0
    # the model stays usable after an error
    m.set_events(W.make_events(rows[:1]))
    rc, st, er = m.run(w.tspan, w.seed, 1, u0, v0, Ud, Vd, check=False)
    assert rc == 0


def test_negative_rate_reports_rate_error(orc, gpu):
    w = W.plain_model(W.SIR, [[5, 1, 0]], np.arange(0, 3), [-0.5, 0.1])
    code, *_ = orc.run(w)
    assert code == -4
    m = gpu.Model(w)
    import torch
    u0 = torch.as_tensor(w.u0, device="cuda")
    v0 = torch.zeros((1, 1, 0), dtype=torch.float64, device="cuda")
    Ud = torch.empty((1, 3, 1, 3), dtype=torch.int32, device="cuda")
    Vd = torch.empty((1, 3, 1, 0), dtype=torch.float64, device="cuda")
    rc, st, er = m.run(w.tspan, w.seed, 1, u0, v0, Ud, Vd, check=False)
    assert rc == -4


def test_invalid_event_table_is_rejected(gpu):
    w = W.plain_model(W.SIR, [[5, 1, 0]], np.arange(0, 3), [0.5, 0.1])
    m = gpu.Model(w)
    with pytest.raises(gpu.SimInfError) as e:
        m.set_events(W.make_events([(INTERNAL, 1, 0, 0, 1, 0.0, 0, -1)]))
    assert e.value.code == -1


def test_run_host_matches_run(orc, gpu):
    w = W.config_sise(n_nodes=500, days=60, gen_seed=9)
    U1, V1, st1 = gpu.simulate(w)
    m = gpu.Model(w)
    M = len(w.tspan)
    U = np.zeros((1, M, 500, 2), np.int32)
    V = np.zeros((1, M, 500, 1), np.float64)
    rc, st, er = m.run_host(w.tspan, w.seed, 1, np.ascontiguousarray(w.u0),
                            np.ascontiguousarray(w.v0), U, V)
    assert rc == 0
    assert np.array_equal(U, U1) and np.array_equal(V, V1)
    assert st["reactions"] == st1["reactions"]


def test_full_size_sise3_prefix(orc, gpu):
    # 37,000 nodes x 3,650 days with ~15M events on the GPU; the oracle runs
    # the first 60 days (the counter-based stream makes that prefix identical)
    w = W.config_sise3()
    U1, V1, st = gpu.simulate(w)
    assert st["node_days"] == 37_000 * 3650
    K = 60
    wp = W.Workload(**{**w.__dict__, "tspan": w.tspan[:K + 1]})
    code, U0, V0, R0, err = orc.run(wp)
    assert code == 0
    assert np.array_equal(U0[0], U1[0, :K + 1])
    assert np.array_equal(V0[0].view(np.uint64), V1[0, :K + 1].view(np.uint64))
    # properties at every time point of the full run
    assert U1.min() >= 0
    ev = w.events
    tot = U1[0].sum(axis=(1, 2)).astype(np.int64)
    d_enter = np.bincount(ev["time"][ev["event"] == ENTER],
                          weights=ev["n"][ev["event"] == ENTER], minlength=3651)
    d_exit = np.bincount(ev["time"][ev["event"] == EXIT],
                         weights=ev["n"][ev["event"] == EXIT], minlength=3651)
    assert np.array_equal(np.diff(tot), (d_enter - d_exit)[1:3651].astype(np.int64))


@pytest.mark.parametrize("tuning", [(1, 0), (16, 0), (32, 1), (64, 4), (128, 2), (128, 1 << 20)])
def test_work_split_never_changes_results(orc, gpu, tuning):
    # nodes per block and the thread-to-warp hand-off point change speed only
    w = W.config_sise(n_nodes=700, days=120, gen_seed=21)
    w.u0[0, :40, 1] = np.maximum(w.u0[0, :40, 1], w.u0[0, :40, 0] // 2)
    code, U0, V0, R0, err = orc.run(w)
    assert code == 0
    U1, V1, st = gpu.simulate(w, tuning=tuning)
    assert np.array_equal(U0, U1)
    assert np.array_equal(V0.view(np.uint64), V1.view(np.uint64))
    assert st["reactions"] == int(R0.sum())


def test_one_wave_larger_than_a_staging_chunk(orc, gpu):
    # 1,500 transfers between disjoint node pairs on one day form one wave,
    # larger than the 512 events the E2 kernel stages at a time
    n = 3000
    rows = [(EXTERNAL, 1, 2 * i, 2 * i + 1, 2, 0.0, 2, -1) for i in range(n // 2)]
    rows += [(EXTERNAL, 2, 2 * i + 1, 2 * i, 1, 0.0, 2, -1) for i in range(n // 2)]
    u0 = np.tile([[20, 3]], (n, 1))
    w = W.plain_model(W.SISE, u0, np.arange(0, 4), W.sise_gdata(), seed=13,
                      events=W.make_events(rows), v0=np.full((n, 1), 0.2))
    _compare(orc, gpu, w)


def _dev(w, n_rep=None):
    import torch
    n_rep = w.n_rep if n_rep is None else n_rep
    u0 = torch.as_tensor(np.ascontiguousarray(w.u0[:n_rep]), device="cuda")
    v0 = torch.as_tensor(np.ascontiguousarray(w.v0[:n_rep]), device="cuda")
    M = len(w.tspan)
    U = torch.empty((n_rep, M, w.n_nodes, w.n_comp), dtype=torch.int32, device="cuda")
    V = torch.empty((n_rep, M, w.n_nodes, w.n_v), dtype=torch.float64, device="cuda")
    return u0, v0, U, V


def test_graph_capture_and_replay(orc, gpu):
    # on a non-default stream the run is captured into a CUDA graph once and
    # replayed; a new seed forces a new capture
    import torch
    w = W.config_sise(n_nodes=400, days=50, gen_seed=31)
    code, U0, V0, R0, err = orc.run(w)
    code2, U2, V2, R2, err2 = orc.run(w, seed=7)
    m = gpu.Model(w)
    u0, v0, U, V = _dev(w)
    s = torch.cuda.Stream()
    for seed, (Ue, Ve, Re) in ((w.seed, (U0, V0, R0)), (w.seed, (U0, V0, R0)),
                               (7, (U2, V2, R2)), (w.seed, (U0, V0, R0))):
        U.fill_(-1)
        rc, st, er = m.run(w.tspan, seed, 1, u0, v0, U, V, stream=s)
        s.synchronize()
        assert np.array_equal(U.cpu().numpy(), Ue)
        assert np.array_equal(V.cpu().numpy().view(np.uint64), Ve.view(np.uint64))
        assert st["reactions"] == int(Re.sum())


def test_graph_recaptured_after_buffers_change(orc, gpu):
    import torch
    w = W.config_sise3(n_nodes=300, days=40, gen_seed=8, n_rep=3)
    code, U0, V0, R0, err = orc.run(w, n_rep=1)
    m = gpu.Model(w)
    s = torch.cuda.Stream()
    u0, v0, U, V = _dev(w, 1)
    m.run(w.tspan, w.seed, 1, u0, v0, U, V, stream=s)
    # a run with more replicates on the default stream reallocates the
    # model's working buffers
    u3, v3, U3, V3 = _dev(w, 3)
    m.run(w.tspan, w.seed, 3, u3, v3, U3, V3)
    U.fill_(-1)
    m.run(w.tspan, w.seed, 1, u0, v0, U, V, stream=s)
    s.synchronize()
    assert np.array_equal(U.cpu().numpy(), U0)
    assert np.array_equal(U3.cpu().numpy()[:1], U0)


def test_sise_sp_coupled_post_step(orc, gpu):
    # SISe_sp (spatial coupling of phi between farms within 2,500 m) with the
    # SISe event stream, 1,600 farms x 365 days
    w = W.config_sise_sp()
    assert len(w.neighbors[1]) > 1600
    _compare(orc, gpu, w)


def test_sise_sp_replicates_and_sparse_tspan(orc, gpu):
    w = W.config_sise_sp(n_nodes=500, days=90, gen_seed=44)
    w = W.Workload(**{**w.__dict__, "tspan": np.array([0, 1, 7, 30, 31, 90], np.int32),
                      "n_rep": 3, "u0": np.repeat(w.u0, 3, axis=0),
                      "v0": np.repeat(w.v0, 3, axis=0)})
    _compare(orc, gpu, w)


@pytest.mark.parametrize("mode", ["persistent", "fused", "separate"])
@pytest.mark.parametrize("tuning", [(1, 2), (48, 1), (128, 0)])
def test_external_transfers_every_schedule(orc, gpu, mode, tuning):
    # the day's external transfers run inside one persistent launch between
    # grid barriers, at the end of each day kernel (last block of each
    # replicate) or in their own kernel; with one node per block every
    # replicate spans hundreds of blocks, with 48 a block spans a replicate
    # boundary
    w = W.config_sise3(n_nodes=350, days=60, gen_seed=41, n_rep=3, per_rep_events=True,
                       median=50, sigma=1.0, hi=5000)
    code, U0, V0, R0, err = orc.run(w)
    assert code == 0
    m = gpu.Model(w)
    m.set_persistent(mode == "persistent")
    m.set_fused_events(mode == "fused")
    m.set_tuning(*tuning)
    u0, v0, U, V = _dev(w)
    rc, st, er = m.run(w.tspan, w.seed, w.n_rep, u0, v0, U, V)
    assert np.array_equal(U.cpu().numpy(), U0)
    assert np.array_equal(V.cpu().numpy().view(np.uint64), V0.view(np.uint64))
    assert st["reactions"] == int(R0.sum())
    m.close()


def test_persistent_and_split_runs_agree_on_the_benchmark_workload(orc, gpu):
    # 1,600 SISe nodes x 365 days, ~200k events: one persistent launch and
    # the split schedule give the oracle's trajectories, with graph replay
    import torch
    w = W.config_sise()
    code, U0, V0, R0, err = orc.run(w)
    s = torch.cuda.Stream()
    for persistent in (True, False, True):
        m = gpu.Model(w)
        m.set_persistent(persistent)
        u0, v0, U, V = _dev(w)
        for _ in range(2):
            U.fill_(-1)
            rc, st, er = m.run(w.tspan, w.seed, 1, u0, v0, U, V, stream=s)
            s.synchronize()
            assert np.array_equal(U.cpu().numpy(), U0)
            assert np.array_equal(V.cpu().numpy().view(np.uint64), V0.view(np.uint64))
            assert st["reactions"] == int(R0.sum())
            assert (st["kernel_launches"] <= 3) == persistent
        m.close()


def test_draw_limit_reports_the_same_error(orc, gpu):
    # SIS with beta = gamma = 1e5: node 1 (S = I = 1000) flips between the
    # two transitions at ~1e8 per day, so its first node-day needs more than
    # 2^24 draws and both sides stop with SG_ERR_STEP_LIMIT at node 1, day 1
    w = W.plain_model(W.SIS, [[10, 0], [1000, 1000], [5, 5]], np.arange(0, 3), [1e5, 1e5])
    code, U0, V0, R0, err = orc.run(w)
    assert code == -9 and err["node"] == 1 and err["day"] == 1
    m = gpu.Model(w)
    u0, v0, U, V = _dev(w)
    rc, st, er = m.run(w.tspan, w.seed, 1, u0, v0, U, V, check=False)
    assert rc == -9 and er["node"] == 1 and er["day"] == 1
    m.close()


def test_empty_model(orc, gpu):
    w = W.plain_model(W.SIR, np.zeros((0, 3), np.int32), np.arange(0, 5), [0.5, 0.1])
    code, U0, V0, R0, err = orc.run(w)
    assert code == 0 and U0.shape == (1, 5, 0, 3)
    U1, V1, st = gpu.simulate(w)
    assert U1.shape == (1, 5, 0, 3) and st["reactions"] == 0


@pytest.mark.parametrize("tuning", [(64, 2), (2000, 2)])
def test_large_events_sampled_by_warps(orc, gpu, tuning):
    # events that move thousands of animals are sampled by a whole warp
    # (32 draws per round): exits, ageing internal transfers and external
    # transfers by count and by proportion (80%, 25%, 20%) on herds of 10^4,
    # and on two herds of about 2e9 animals, where Lemire's method rejects
    # 2-7% of the words (2^32 mod s is large for s near 2e9), so rounds end
    # early and the retry takes the next word; every outcome equals the
    # oracle's sequential urn bit for bit
    n = 40
    big = 2_000_000_000
    u0 = np.tile([[6000, 2000, 5000, 1000, 9000, 3000]], (n, 1)).astype(np.int32)
    u0[0] = [big, 100_000_000, 10, 0, 10, 0]
    u0[1] = [big, 0, 0, 0, 0, 0]
    rows = []
    for t in range(1, 6):
        rows.append((EXIT, t, 0, 0, 4000 + t, 0.0, 3, -1))          # 4,000 draws at s ~ 2.1e9
        rows.append((EXTERNAL, t, 1, 2 + t, 3000, 0.0, 0, -1))       # 3,000 draws at s ~ 2e9
        for i in range(2, n):
            rows.append((EXIT, t, i, 0, 0, 0.25, 3 + (i % 3), -1))
            rows.append((INTERNAL, t, i, 0, 0, 0.8, 3 + (i % 2), i % 2))
            rows.append((EXTERNAL, t, i, (i + 7) % n, 0, 0.2, 3 + (i % 3), -1))
            rows.append((EXTERNAL, t, i, (i + 3) % n, 40 + i, 0.0, 5, -1))
    gd = W.sise3_gdata(upsilons=(0.0,) * 3, gammas=(0.0,) * 3, alpha=0.0, betas=(0.0,) * 4)
    w = W.plain_model(W.SISE3, u0, np.arange(0, 7), gd, seed=99, events=W.make_events(rows))
    code, U0, V0, R0, err = orc.run(w)
    assert code == 0, err
    U1, V1, st = gpu.simulate(w, tuning=tuning)
    assert np.array_equal(U0, U1)
    assert st["events_applied"] == len(rows)
