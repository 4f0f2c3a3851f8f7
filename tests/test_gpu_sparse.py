"""Parity of the sparse-activity day schedule (nodes_per_block > 128: a block
owns a range of units in global memory, skips the provably empty days of
quiescent units, and runs the SSA of the units with a positive total rate
from a shared list) with the CPU oracle: bit-exact U and V, identical
reaction counts and identical errors, for every built-in kind, with and
without scheduled events, several replicates, ranges that need more than one
pass through the list (more units per block than the list holds), blocks
that hold a whole replicate or several (with the replicates' external
transfers run by the block), and every hand-off setting."""
import numpy as np
import pytest

from paper_1605_01421_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EXIT, ENTER, INTERNAL, EXTERNAL = 0, 1, 2, 3
SPLITS = [(129, 0), (1000, 2), (5000, 1 << 20), (9000, 8)]


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_01421_gb300 import binding
    binding.build()
    binding.lib()
    return binding


def _compare(orc, gpu, w, tuning, n_rep=None):
    code, U0, V0, R0, err0 = orc.run(w, n_rep=n_rep)
    assert code == 0, err0
    U1, V1, st = gpu.simulate(w, n_rep=n_rep, tuning=tuning)
    diff_nodes = np.any(U0 != U1, axis=(1, 3)).sum()
    assert diff_nodes == 0, f"{diff_nodes} node trajectories diverge"
    assert np.array_equal(U0, U1)
    assert np.array_equal(V0.view(np.uint64), V1.view(np.uint64))
    assert st["reactions"] == int(R0.sum())
    return st


@pytest.mark.parametrize("tuning", SPLITS)
def test_sise_with_events(orc, gpu, tuning):
    w = W.config_sise(n_nodes=1600, days=120, gen_seed=41)
    st = _compare(orc, gpu, w, tuning)
    assert st["events_applied"] > 0


@pytest.mark.parametrize("tuning", SPLITS)
def test_sise3_with_all_event_types_and_replicates(orc, gpu, tuning):
    w = W.config_batched(n_rep=3, n_nodes=2200, days=60, gen_seed=42)
    _compare(orc, gpu, w, tuning)


@pytest.mark.parametrize("tuning", [(300, 0), (4500, 2), (4000, 2)])
def test_sir_and_sis_without_events(orc, gpu, tuning):
    # no external transfers: whole runs of days inside one launch, the post
    # time step and recording of each day before the next day's SSA
    rng = np.random.default_rng(43)
    u0 = np.stack([rng.integers(0, 300, 4000), rng.integers(0, 3, 4000),
                   rng.integers(0, 30, 4000)], 1).astype(np.int32)
    w = W.plain_model(W.SIR, u0, np.arange(0, 61), [0.16, 0.077], seed=5, n_rep=2)
    _compare(orc, gpu, w, tuning)
    w = W.plain_model(W.SIS, u0[:, :2], np.array([0, 3, 10, 11, 40]), [0.002, 0.1], seed=6)
    _compare(orc, gpu, w, tuning)


@pytest.mark.parametrize("tuning", [(129, 2), (3000, 0)])
def test_sise3_quiescent_and_endemic_mix(orc, gpu, tuning):
    # most herds without infection and phi = 0 (their days are skipped),
    # a few endemic herds with hundreds of transitions a day (handed to
    # warps), seasonal decay crossing the season ends
    rng = np.random.default_rng(44)
    n = 6000
    herd = np.clip(np.rint(np.exp(np.log(60) + 1.2 * rng.standard_normal(n))), 1, 8000)
    ages = W.split_ages(herd.astype(np.int64))
    I = np.zeros_like(ages)
    hot = rng.random(n) < 0.03
    I[hot] = np.rint(0.4 * ages[hot]).astype(np.int64)
    S = ages - I
    u0 = np.stack([S[:, 0], I[:, 0], S[:, 1], I[:, 1], S[:, 2], I[:, 2]], 1).astype(np.int32)
    v0 = np.where(hot, 2.0, 0.0)[:, None]
    w = W.plain_model(W.SISE3, u0, np.arange(80, 101), W.sise3_gdata(), seed=7, v0=v0,
                      ldata=W.seasons_ldata(n))
    _compare(orc, gpu, w, tuning)


def test_nonfinite_unused_parameter_takes_the_full_path(orc, gpu):
    # beta of season 4 is NaN but the run stays in seasons 1-3: the result is
    # defined, and with a non-finite parameter no day is skipped
    w = W.config_sise3(n_nodes=3000, days=40, gen_seed=45)
    w.gdata = np.array(w.gdata, dtype=np.float64)
    w.gdata[10] = np.nan
    _compare(orc, gpu, w, (1500, 2))


@pytest.mark.parametrize("tuning", [(129, 2), (2000, 0)])
def test_event_underflow_and_rate_errors(orc, gpu, tuning):
    rows = [(ENTER, 1, 0, 0, 2, 0.0, 0, -1), (EXIT, 2, 0, 0, 50, 0.0, 2, -1)]
    w = W.plain_model(W.SISE, [[5, 0], [5, 0]], np.arange(0, 5), W.sise_gdata(),
                      events=W.make_events(rows))
    code, U, V, R, err = orc.run(w)
    assert code == -2 and err["event"] == 1 and err["day"] == 2
    m = gpu.Model(w)
    m.set_tuning(*tuning)
    u0, v0, Ud, Vd = _dev(w)
    rc, st, er = m.run(w.tspan, w.seed, 1, u0, v0, Ud, Vd, check=False)
    assert rc == -2 and er["event"] == 1 and er["day"] == 2 and er["node"] == 0
    m.set_events(W.make_events(rows[:1]))
    rc, st, er = m.run(w.tspan, w.seed, 1, u0, v0, Ud, Vd, check=False)
    assert rc == 0
    m.close()
    # a negative rate
    w = W.plain_model(W.SIR, [[5, 1, 0]] * 300, np.arange(0, 3), [-0.5, 0.1])
    assert orc.run(w)[0] == -4
    m = gpu.Model(w)
    m.set_tuning(*tuning)
    u0, v0, Ud, Vd = _dev(w)
    rc, st, er = m.run(w.tspan, w.seed, 1, u0, v0, Ud, Vd, check=False)
    assert rc == -4
    m.close()


@pytest.mark.parametrize("tuning", [(1000, 8), (300, 0), (2000, 1 << 20)])
def test_sise3_rate_error_after_transitions_on_warps(orc, gpu, tuning):
    # age class 2 has a negative upsilon and no susceptible animal: its
    # infection rate is -0 until a recovery makes it negative, deep inside
    # the SSA of heavy herds (several per warp) and of light ones
    rng = np.random.default_rng(50)
    n = 3000
    u0 = np.zeros((n, 6), dtype=np.int32)
    u0[:, 0] = rng.integers(0, 200, n)
    u0[:, 1] = rng.integers(0, 3, n)
    hot = rng.choice(n, 40, replace=False)
    u0[hot, 2] = 0
    u0[hot, 3] = rng.integers(100, 1500, hot.size)
    g = W.sise3_gdata(upsilons=(0.0173, -0.01, 0.0173))
    w = W.plain_model(W.SISE3, u0, np.arange(10, 16), g, seed=9, v0=np.ones((n, 1)))
    code, U, V, R, err = orc.run(w)
    assert code == -4
    m = gpu.Model(w)
    m.set_tuning(*tuning)
    u0d, v0d, Ud, Vd = _dev(w)
    rc, st, er = m.run(w.tspan, w.seed, 1, u0d, v0d, Ud, Vd, check=False)
    m.close()
    assert rc == -4 and er["day"] == err["day"]
    assert er["node"] in set(hot.tolist())


def test_draw_limit(orc, gpu):
    # node 1 needs more than 2^24 draws on its first day
    w = W.plain_model(W.SIS, [[10, 0], [1000, 1000], [5, 5]], np.arange(0, 3), [1e5, 1e5])
    code, U0, V0, R0, err = orc.run(w)
    assert code == -9 and err["node"] == 1 and err["day"] == 1
    m = gpu.Model(w)
    m.set_tuning(300, 4)
    u0, v0, U, V = _dev(w)
    rc, st, er = m.run(w.tspan, w.seed, 1, u0, v0, U, V, check=False)
    assert rc == -9 and er["day"] == 1 and er["node"] == 1
    m.close()


@pytest.mark.parametrize("tuning", [(700, 2), (1500, 32)])
def test_sparse_output_and_prevalence(orc, gpu, tuning):
    # U_sparse / V_sparse and the prevalence counters from the sparse
    # schedule equal the oracle's dense trajectory read at the pattern (also
    # with one replicate per block, where each day's record is written by
    # the next day's first passes)
    import torch
    from oracle import outputs
    w = W.config_batched(n_rep=2, n_nodes=1500, days=30, gen_seed=46)
    R, M, Nn, C = w.n_rep, len(w.tspan), w.n_nodes, 6
    rng = np.random.default_rng(5)
    colptr, row = [0], []
    for t in range(M):
        r = np.sort(rng.choice(Nn * C, size=rng.integers(0, 40), replace=False))
        row.extend(r.tolist())
        colptr.append(len(row))
    up = (np.array(colptr, np.int64), np.array(row, np.int32))
    uval = torch.full((R, len(row)), -1, dtype=torch.int32, device="cuda")
    pout = torch.zeros((R, M, 4), dtype=torch.int64, device="cuda")
    m = gpu.Model(w)
    m.set_tuning(*tuning)
    m.set_output(dense=False, n_tspan=M, u_pattern=up, u_values=uval,
                 prevalence=([1, 3, 5], list(range(6))), prev_out=pout)
    u0, v0, _, _ = _dev(w)
    rc, st, er = m.run(w.tspan, w.seed, R, u0, v0, None, None)
    m.close()
    code, U0, V0, R0, err = orc.run(w)
    assert np.array_equal(uval.cpu().numpy(), outputs.sparse_values(U0, *up, C))
    assert np.array_equal(pout.cpu().numpy(), outputs.prevalence_counts(U0, [1, 3, 5], range(6)))


@pytest.mark.parametrize("tuning", [(1000, 0), (900, 8)])
def test_replicate_shards_on_the_sparse_schedule(orc, gpu, tuning):
    import torch
    w = W.config_batched(n_rep=4, n_nodes=900, days=25, gen_seed=47)
    U_all, V_all, _ = gpu.simulate(w, tuning=(600, 2))
    s = W.replicate_range(w, 1, 2)
    m = gpu.Model(s)
    m.set_replicate_range(1, 4)
    m.set_tuning(*tuning)
    u0, v0, U, V = _dev(s)
    m.run(s.tspan, s.seed, 2, u0, v0, U, V)
    m.close()
    assert np.array_equal(U.cpu().numpy(), U_all[1:3])
    code, Uo, Vo, Ro, err = orc.run(w, rep0=1, n_rep=2)
    assert np.array_equal(Uo, U_all[1:3])


def test_aem_fallback_and_fused_external_transfers(orc, gpu):
    # the all events method takes the thread-per-node kernel whatever the
    # split; with fused external transfers the sparse kernel's last block of
    # each replicate runs them in its tail (same results either way)
    w = W.config_sise(n_nodes=900, days=40, gen_seed=48)
    w.solver = W.AEM
    _compare(orc, gpu, w, (2000, 2))
    w = W.config_sise(n_nodes=900, days=40, gen_seed=48)
    code, U0, V0, R0, err = orc.run(w)
    m = gpu.Model(w)
    m.set_tuning(2000, 2)
    m.set_fused_events(True)
    u0, v0, U, V = _dev(w)
    m.run(w.tspan, w.seed, 1, u0, v0, U, V)
    m.close()
    assert np.array_equal(U.cpu().numpy(), U0)


@pytest.mark.parametrize("per_block,heavy", [(1, 8), (2, 0), (3, 1 << 20)])
def test_whole_replicates_per_block(orc, gpu, per_block, heavy):
    # nodes per block a multiple of the node count: one launch for every
    # day, each block running its replicates' external transfers between the
    # day's E1 events and its post time step (own events per replicate, and
    # one list shared by the replicates)
    w = W.config_batched(n_rep=5, n_nodes=700, days=50, gen_seed=49)
    st = _compare(orc, gpu, w, (700 * per_block, heavy))
    assert st["kernel_launches"] <= 5  # not two per day
    w = W.config_sise3(n_nodes=400, days=90, gen_seed=5, n_rep=6)
    _compare(orc, gpu, w, (400 * per_block, heavy))


@pytest.mark.parametrize("tuning", [(9000, 8), (18000, 2), (20000, 32)])
def test_blocks_of_several_chunks(orc, gpu, tuning):
    # more units per block than one chunk of the shared lists holds (8,192):
    # each day runs the passes and the SSA chunk by chunk, with whole
    # replicates per block (9,000 and 18,000) and without (20,000)
    w = W.config_batched(n_rep=3, n_nodes=9000, days=20, gen_seed=51)
    _compare(orc, gpu, w, tuning)


def test_whole_replicates_per_block_transfer_underflow(orc, gpu):
    # an external transfer of more animals than the source holds, on day 2
    # of replicate 1: the same error and no post time step of that day
    rows = [(EXTERNAL, 1, 0, 1, 3, 0.0, 2, -1), (EXTERNAL, 2, 1, 0, 500, 0.0, 2, -1)]
    u0 = [[40, 2], [30, 0]] + [[20, 1]] * 198
    w = W.plain_model(W.SISE, u0, np.arange(0, 6), W.sise_gdata(), n_rep=3,
                      events=W.make_events(rows))
    code, U, V, R, err = orc.run(w)
    assert code == -2 and err["event"] == 1 and err["day"] == 2
    m = gpu.Model(w)
    m.set_tuning(200, 2)
    u0d, v0d, Ud, Vd = _dev(w)
    rc, st, er = m.run(w.tspan, w.seed, 3, u0d, v0d, Ud, Vd, check=False)
    assert rc == -2 and er["event"] == 1 and er["day"] == 2 and er["node"] == 1
    m.set_events(W.make_events(rows[:1]))
    rc, st, er = m.run(w.tspan, w.seed, 3, u0d, v0d, Ud, Vd, check=False)
    assert rc == 0
    m.close()


def _dev(w, n_rep=None):
    import torch
    n_rep = w.n_rep if n_rep is None else n_rep
    u0 = torch.as_tensor(np.ascontiguousarray(w.u0[:n_rep]), device="cuda")
    v0 = torch.as_tensor(np.ascontiguousarray(w.v0[:n_rep]), device="cuda")
    M = len(w.tspan)
    U = torch.empty((n_rep, M, w.n_nodes, w.n_comp), dtype=torch.int32, device="cuda")
    V = torch.empty((n_rep, M, w.n_nodes, w.n_v), dtype=torch.float64, device="cuda")
    return u0, v0, U, V
