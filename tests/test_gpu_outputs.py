"""Output selection on the GPU (Sec. 3.2 U_sparse / V_sparse and the
prevalence summary of Sec. 4.2): the sparse values equal the oracle's dense
trajectory at the pattern, bit for bit; the prevalence counters equal the
plain reductions of the oracle's trajectory; dense output can be switched
off; patterns are checked."""
import numpy as np
import pytest

from oracle import outputs
from paper_1605_01421_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_01421_gb300 import binding
    binding.build()
    binding.lib()
    return binding


def _pattern(rng, M, rows, per_col_max):
    colptr, row = [0], []
    for m in range(M):
        k = int(rng.integers(0, per_col_max + 1))
        r = np.sort(rng.choice(rows, size=min(k, rows), replace=False))
        row.extend(int(x) for x in r)
        colptr.append(len(row))
    return np.array(colptr, np.int64), np.array(row, np.int32)


def _run(gpu, w, dense, up, vp, prev, stream=None):
    import torch
    R, M, Nn, C, Nv = w.n_rep, len(w.tspan), w.n_nodes, w.n_comp, w.n_v
    m = gpu.Model(w)
    uval = torch.full((R, len(up[1])), -7, dtype=torch.int32, device="cuda") if up else None
    vval = torch.full((R, len(vp[1])), -7.0, dtype=torch.float64, device="cuda") if vp else None
    pout = torch.full((R, M, 4), -1, dtype=torch.int64, device="cuda") if prev else None
    m.set_output(dense=dense, n_tspan=M, u_pattern=up, u_values=uval, v_pattern=vp,
                 v_values=vval, prevalence=prev, prev_out=pout)
    u0 = torch.as_tensor(np.ascontiguousarray(w.u0), device="cuda")
    v0 = torch.as_tensor(np.ascontiguousarray(w.v0), device="cuda")
    U = V = None
    if dense:
        U = torch.empty((R, M, Nn, C), dtype=torch.int32, device="cuda")
        V = torch.empty((R, M, Nn, Nv), dtype=torch.float64, device="cuda")
    rc, st, er = m.run(w.tspan, w.seed, R, u0, v0, U, V, stream=stream)
    if stream is not None:
        stream.synchronize()
    res = (None if U is None else U.cpu().numpy(), None if uval is None else uval.cpu().numpy(),
           None if vval is None else vval.cpu().numpy(), None if pout is None else pout.cpu().numpy())
    return m, res


def _check(orc, gpu, w, dense, per_col=25, prev=None, seed=0):
    code, U0, V0, R0, err = orc.run(w)
    assert code == 0, err
    rng = np.random.default_rng(seed)
    M, Nn, C, Nv = len(w.tspan), w.n_nodes, w.n_comp, w.n_v
    up = _pattern(rng, M, Nn * C, per_col)
    vp = _pattern(rng, M, Nn * Nv, per_col) if Nv else None
    m, (U, uval, vval, pout) = _run(gpu, w, dense, up, vp, prev)
    m.close()
    if dense:
        assert np.array_equal(U, U0)
    assert np.array_equal(uval, outputs.sparse_values(U0, *up, C))
    if vp is not None:
        assert np.array_equal(vval.view(np.uint64),
                              outputs.sparse_values(V0, *vp, Nv).view(np.uint64))
    if prev is not None:
        assert np.array_equal(pout, outputs.prevalence_counts(U0, *prev))


def test_sparse_alongside_dense_sise(orc, gpu):
    _check(orc, gpu, W.config_sise(n_nodes=700, days=60, gen_seed=3), True,
           prev=([1], [0, 1]))


def test_sparse_only_sise3_replicates_with_events(orc, gpu):
    w = W.config_sise3(n_nodes=500, days=70, gen_seed=5, n_rep=3)
    _check(orc, gpu, w, False, per_col=60, prev=([1, 3, 5], [0, 1, 2, 3, 4, 5]))


def test_prevalence_only_sir_many_blocks(orc, gpu):
    # ragged node count, units spread over many warps and a replicate boundary
    # inside warps (1037 nodes, 3 replicates)
    w = W.plain_model(W.SIR, np.tile([[995, 5, 0]], (1037, 1)), np.arange(3, 61),
                      [0.6, 0.2], seed=5, n_rep=3)
    code, U0, V0, R0, err = orc.run(w)
    m, (U, uval, vval, pout) = _run(gpu, w, False, None, None, ([1], [0, 1]))
    m.close()
    assert np.array_equal(pout, outputs.prevalence_counts(U0, [1], [0, 1]))


def test_sise_sp_sparse_and_prevalence(orc, gpu):
    _check(orc, gpu, W.config_sise_sp(n_nodes=500, days=60, gen_seed=44), False,
           prev=([1], [0, 1]))


def test_aem_with_prevalence(orc, gpu):
    w = W.config_sise(n_nodes=600, days=80, gen_seed=12)
    w.solver = W.AEM
    _check(orc, gpu, w, True, prev=([1], [0, 1]))


def test_graph_replay_keeps_outputs(orc, gpu):
    import torch
    w = W.config_sise(n_nodes=400, days=40, gen_seed=31)
    code, U0, V0, R0, err = orc.run(w)
    rng = np.random.default_rng(1)
    M = len(w.tspan)
    up = _pattern(rng, M, w.n_nodes * 2, 10)
    s = torch.cuda.Stream()
    m, (U, uval, vval, pout) = _run(gpu, w, False, up, None, ([1], [0, 1]), stream=s)
    # replay the captured run twice more
    u0 = torch.as_tensor(np.ascontiguousarray(w.u0), device="cuda")
    v0 = torch.as_tensor(np.ascontiguousarray(w.v0), device="cuda")
    for _ in range(2):
        m._out_refs[0].fill_(-3)
        m.run(w.tspan, w.seed, 1, u0, v0, None, None, stream=s)
        s.synchronize()
        assert np.array_equal(m._out_refs[0].cpu().numpy(), outputs.sparse_values(U0, *up, 2))
        assert np.array_equal(m._out_refs[2].cpu().numpy(),
                              outputs.prevalence_counts(U0, [1], [0, 1]))
    m.close()


def test_bad_patterns_are_rejected(gpu):
    import torch
    w = W.plain_model(W.SIR, np.tile([[5, 1, 0]], (4, 1)), np.arange(0, 3), [0.5, 0.1])
    m = gpu.Model(w)
    val = torch.zeros((1, 3), dtype=torch.int32, device="cuda")
    bad = [((0, 2, 2, 3), (5, 4, 1)),      # rows not increasing in column 0
           ((0, 1, 2, 3), (1, 12, 0)),     # row out of range (4 nodes x 3)
           ((1, 1, 2, 3), (1, 2, 3))]      # colptr[0] != 0
    for cp, rw in bad:
        with pytest.raises(gpu.SimInfError):
            m.set_output(dense=True, n_tspan=3, u_pattern=(np.array(cp), np.array(rw)),
                         u_values=val)
    # a good pattern, then a run with another number of tspan points
    m.set_output(dense=False, n_tspan=3, u_pattern=(np.array([0, 1, 2, 3]), np.array([0, 4, 11])),
                 u_values=val)
    u0 = torch.as_tensor(np.ascontiguousarray(w.u0), device="cuda")
    v0 = torch.zeros((1, 4, 0), dtype=torch.float64, device="cuda")
    rc, st, er = m.run(np.arange(0, 4), 1, 1, u0, v0, None, None, check=False)
    assert rc == -1
    rc, st, er = m.run(np.arange(0, 3), 1, 1, u0, v0, None, None, check=False)
    assert rc == 0
    m.close()


def test_run_host_without_dense_output(orc, gpu):
    import torch
    w = W.config_sise(n_nodes=300, days=30, gen_seed=2)
    code, U0, V0, R0, err = orc.run(w)
    M = len(w.tspan)
    m = gpu.Model(w)
    pout = torch.zeros((1, M, 4), dtype=torch.int64, device="cuda")
    m.set_output(dense=False, n_tspan=M, prevalence=([1], [0, 1]), prev_out=pout)
    m.run_host(w.tspan, w.seed, 1, np.ascontiguousarray(w.u0), np.ascontiguousarray(w.v0),
               None, None)
    assert np.array_equal(pout.cpu().numpy(), outputs.prevalence_counts(U0, [1], [0, 1]))
    m.close()


def test_full_size_batched_on_sampled_replicates(orc, gpu):
    # 256 replicates x 5,000 SISe3 nodes x 365 days, each replicate with its
    # own ~175k events, tuned by the autotuner as the benchmark is; dense
    # output off (it would be 11 GB), U_sparse holds every node at days 30 and
    # 365, prevalence counters every day.  The oracle runs replicates 0, 101
    # and 255 on their own; every replicate's population follows its events
    import torch
    w = W.config_batched()
    R, M, Nn, C = w.n_rep, len(w.tspan), w.n_nodes, 6
    m = gpu.Model(w)
    cols = {30: np.arange(Nn * C, dtype=np.int32), 365: np.arange(Nn * C, dtype=np.int32)}
    colptr, row = [0], []
    for t in range(M):
        row.extend(cols.get(t, []))
        colptr.append(len(row))
    up = (np.array(colptr, np.int64), np.array(row, np.int32))
    uval = torch.full((R, len(row)), -1, dtype=torch.int32, device="cuda")
    pout = torch.zeros((R, M, 4), dtype=torch.int64, device="cuda")
    u0 = torch.as_tensor(np.ascontiguousarray(w.u0), device="cuda")
    v0 = torch.as_tensor(np.ascontiguousarray(w.v0), device="cuda")
    Ud = torch.empty((R, M, Nn, C), dtype=torch.int32, device="cuda")
    Vd = torch.empty((R, M, Nn, 1), dtype=torch.float64, device="cuda")
    m.autotune(w.tspan, w.seed, R, u0, v0, Ud, Vd)
    del Ud, Vd
    m.set_output(dense=False, n_tspan=M, u_pattern=up, u_values=uval,
                 prevalence=([1, 3, 5], list(range(6))), prev_out=pout)
    rc, st, er = m.run(w.tspan, w.seed, R, u0, v0, None, None)
    assert st["node_days"] == R * Nn * 365
    vals, prev = uval.cpu().numpy(), pout.cpu().numpy()
    m.close()
    for r in (0, 101, 255):
        code, U0, V0, R0, err = orc.run(w, rep0=r, n_rep=1)
        assert code == 0
        assert np.array_equal(vals[r], outputs.sparse_values(U0, *up, C)[0])
        assert np.array_equal(prev[r], outputs.prevalence_counts(U0, [1, 3, 5], range(6))[0])
    # every replicate, every day: the population is u0 plus enters minus exits
    ev = w.events
    assert ev["n"].min() > 0 and ev["time"].min() >= 1
    delta = np.zeros((R, M), np.int64)
    for etype, sign in ((1, 1), (0, -1)):  # enter, exit
        sel = ev["event"] == etype
        np.add.at(delta, (ev["rep"][sel], ev["time"][sel]), sign * ev["n"][sel].astype(np.int64))
    expected = w.u0.sum(axis=(1, 2)).astype(np.int64)[:, None] + np.cumsum(delta, axis=1)
    assert np.array_equal(prev[:, :, 1], expected)


@pytest.mark.parametrize("solver", [0, 1])
def test_replicate_shards_reproduce_the_whole_job(orc, gpu, solver):
    # a job of 6 replicates with their own events, run whole and as shards
    # 0..1, 2..4, 5..5 (global replicate index in every stream, the whole
    # job's event table given to every shard): every shard's U and V equal
    # the whole run's rows bit for bit, and the middle shard equals the
    # oracle's run of those replicates
    import torch
    w = W.config_batched(n_rep=6, n_nodes=300, days=40, gen_seed=77)
    w.solver = solver
    U_all, V_all, st_all = gpu.simulate(w)
    for rep0, n in ((0, 2), (2, 3), (5, 1)):
        s = W.replicate_range(w, rep0, n)
        m = gpu.Model(s)
        m.set_replicate_range(rep0, w.n_rep)
        M = len(s.tspan)
        u0 = torch.as_tensor(np.ascontiguousarray(s.u0), device="cuda")
        v0 = torch.as_tensor(np.ascontiguousarray(s.v0), device="cuda")
        U = torch.empty((n, M, s.n_nodes, 6), dtype=torch.int32, device="cuda")
        V = torch.empty((n, M, s.n_nodes, 1), dtype=torch.float64, device="cuda")
        rc, st, er = m.run(s.tspan, s.seed, n, u0, v0, U, V)
        m.close()
        assert np.array_equal(U.cpu().numpy(), U_all[rep0:rep0 + n])
        assert np.array_equal(V.cpu().numpy().view(np.uint64),
                              V_all[rep0:rep0 + n].view(np.uint64))
        if rep0 == 2:
            code, Uo, Vo, Ro, err = orc.run(w, rep0=rep0, n_rep=n)
            assert code == 0
            assert np.array_equal(Uo, U.cpu().numpy())
            assert st["reactions"] == int(Ro.sum())


def test_replicate_range_arguments(gpu):
    w = W.config_batched(n_rep=4, n_nodes=50, days=5, gen_seed=78)
    s = W.replicate_range(w, 1, 2)
    m = gpu.Model(s)
    with pytest.raises(gpu.SimInfError):
        m.set_replicate_range(4, 4)  # rep0 beyond the job
    with pytest.raises(gpu.SimInfError):
        m.set_replicate_range(1, 0)  # an offset without a job size
    m.set_replicate_range(3, 4)  # 3 + 2 replicates > 4: rejected by the run
    import torch
    u0 = torch.as_tensor(np.ascontiguousarray(s.u0), device="cuda")
    v0 = torch.as_tensor(np.ascontiguousarray(s.v0), device="cuda")
    U = torch.empty((2, len(s.tspan), 50, 6), dtype=torch.int32, device="cuda")
    V = torch.empty((2, len(s.tspan), 50, 1), dtype=torch.float64, device="cuda")
    rc, st, er = m.run(s.tspan, s.seed, 2, u0, v0, U, V, check=False)
    assert rc == -1
    m.close()
