"""Parity of the CUDA all events method ('aem', Sec. 3.4.2) with the oracle:
bit-exact U and V, identical reaction counts and error codes, for every
model kind, with scheduled events of all types, replicates (shared and
replicate-specific events), several work splits, graph capture and the
SISe_sp coupled post time step; channel firing times carry across days and
kernel boundaries, so runs span many days and E2 days."""
import numpy as np
import pytest

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


def _aem(w):
    w.solver = W.AEM
    return w


def _compare(orc, gpu, w, n_rep=None, seed=None, tuning=None):
    code, U0, V0, R0, err0 = orc.run(w, seed=seed, n_rep=n_rep)
    assert code == 0, err0
    U1, V1, st = gpu.simulate(w, seed=seed, n_rep=n_rep, tuning=tuning)
    diff_nodes = np.any(U0 != U1, axis=(1, 3)).sum()
    assert diff_nodes == 0, f"{diff_nodes} node trajectories diverge"
    assert np.array_equal(V0.view(np.uint64), V1.view(np.uint64))
    assert st["reactions"] == int(R0.sum())
    return U0, st


def test_sir_and_sis(orc, gpu):
    _compare(orc, gpu, _aem(W.plain_model(W.SIR, np.tile([[995, 5, 0]], (1037, 1)),
                                          np.arange(3, 61), [0.6, 0.2], seed=5)))
    _compare(orc, gpu, _aem(W.plain_model(W.SIS, np.tile([[40, 2]], (300, 1)),
                                          np.arange(1, 181, 7), [0.02, 0.3], seed=6)))


def test_sise_full_size_with_events(orc, gpu):
    # 1,600 nodes x 365 days, ~200k scheduled events of all four types
    U, st = _compare(orc, gpu, _aem(W.config_sise()))
    assert st["reactions"] > 0 and st["events_applied"] > 0


def test_sise3_with_events_and_shared_replicates(orc, gpu):
    _compare(orc, gpu, _aem(W.config_sise3(n_nodes=2500, days=200, gen_seed=33)))
    _compare(orc, gpu, _aem(W.config_sise3(n_nodes=400, days=90, gen_seed=5, n_rep=6)))


def test_replicate_specific_events(orc, gpu):
    w = W.config_sise3(n_nodes=300, days=80, gen_seed=6, n_rep=5,
                       per_rep_events=True, median=50, sigma=1.0, hi=5000)
    assert w.events["rep"] is not None
    _compare(orc, gpu, _aem(w))


@pytest.mark.parametrize("tuning", [(1, 0), (32, 0), (128, 0)])
def test_work_split_never_changes_results(orc, gpu, tuning):
    _compare(orc, gpu, _aem(W.config_sise(n_nodes=700, days=120, gen_seed=21)), tuning=tuning)


def test_sise_sp(orc, gpu):
    _compare(orc, gpu, _aem(W.config_sise_sp(n_nodes=600, days=120, gen_seed=44)))


def test_negative_rate_reports_rate_error(orc, gpu):
    w = _aem(W.plain_model(W.SIR, [[5, 1, 0]], np.arange(0, 3), [-0.5, 0.1]))
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
    m.close()


def test_graph_replay_and_solver_switch(orc, gpu):
    import torch
    w = W.config_sise(n_nodes=400, days=50, gen_seed=31)
    code, Us, Vs, Rs, err = orc.run(w, solver=W.SSM)
    code, Ua, Va, Ra, err = orc.run(w, solver=W.AEM)
    assert not np.array_equal(Us, Ua)
    m = gpu.Model(w)
    u0 = torch.as_tensor(np.ascontiguousarray(w.u0), device="cuda")
    v0 = torch.as_tensor(np.ascontiguousarray(w.v0), device="cuda")
    U = torch.empty((1, len(w.tspan), w.n_nodes, w.n_comp), dtype=torch.int32, device="cuda")
    V = torch.empty((1, len(w.tspan), w.n_nodes, w.n_v), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    for solver, Ue, Re in ((W.AEM, Ua, Ra), (W.AEM, Ua, Ra), (W.SSM, Us, Rs), (W.AEM, Ua, Ra)):
        m.set_solver(solver)
        U.fill_(-1)
        rc, st, er = m.run(w.tspan, w.seed, 1, u0, v0, U, V, stream=s)
        s.synchronize()
        assert np.array_equal(U.cpu().numpy(), Ue)
        assert st["reactions"] == int(Re.sum())


def test_unknown_solver_is_rejected(gpu):
    w = W.plain_model(W.SIR, [[5, 1, 0]], np.arange(0, 3), [0.5, 0.1])
    m = gpu.Model(w)
    with pytest.raises(gpu.SimInfError):
        m.set_solver(2)
    m.close()
