"""Models from transition strings (Sec. 3.5) on the GPU: the library's own
parser (C++) and NVRTC-compiled kernels against the oracle's independent
parser and gcc-compiled propensities -- the same S and G, bit-exact U and
identical reaction counts for the paper's examples (SIR, SIR with the
incidence counter Icum, the Rosenzweig-MacArthur predator-prey model, the
vaccination model with scheduled events), both solvers, replicates, graph
replay and the prevalence counters; parse errors are reported."""
import numpy as np
import pytest

from oracle import mparse, outputs
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


def _compare(orc, gpu, w, n_rep=None):
    code, U0, V0, R0, err0 = orc.run(w, n_rep=n_rep)
    assert code == 0, err0
    U1, V1, st = gpu.simulate(w, n_rep=n_rep)
    diff_nodes = np.any(U0 != U1, axis=(1, 3)).sum()
    assert diff_nodes == 0, f"{diff_nodes} node trajectories diverge"
    assert st["reactions"] == int(R0.sum())
    return U0, st


@pytest.mark.parametrize("w", [
    W.parsed_model(W.MPARSE_SIR, ["S", "I", "R"], {"b": 0.16, "g": 0.077},
                   np.tile([[99, 5, 0]], (4, 1)), np.arange(1, 5)),
    W.config_sir_icum(n_nodes=4),
    W.config_predator_prey(n_nodes=4),
    W.config_vaccination(n_nodes=40, days=30),
], ids=["sir", "icum", "predator_prey", "vaccination"])
def test_both_parsers_build_the_same_tables(gpu, w):
    m = gpu.Model(w)
    S, G = m.tables()
    m.close()
    p = mparse.parse(w.generic["transitions"], w.generic["compartments"],
                     w.generic["gdata_names"])
    assert np.array_equal(S, p.S)
    assert np.array_equal(G, p.G)


def test_parsed_sir_equals_builtin_sir(orc, gpu):
    u0 = np.tile([[99, 5, 0]], (1000, 1))
    parsed = W.parsed_model(W.MPARSE_SIR, ["S", "I", "R"], {"b": 0.16, "g": 0.077}, u0,
                            np.arange(1, 181), seed=123)
    builtin = W.plain_model(W.SIR, u0, np.arange(1, 181), [0.16, 0.077], seed=123)
    code, Ub, Vb, Rb, err = orc.run(builtin)
    U1, V1, st = gpu.simulate(parsed)
    assert np.array_equal(U1, Ub)
    assert st["reactions"] == int(Rb.sum())


def test_sir_icum(orc, gpu):
    _compare(orc, gpu, W.config_sir_icum())


def test_predator_prey(orc, gpu):
    # five transitions with the type-2 functional response; heavy node-days
    # (thousands of firings), so the warp hand-off is exercised
    U, st = _compare(orc, gpu, W.config_predator_prey(n_nodes=150))
    assert st["reactions"] > 1_000_000


@pytest.mark.parametrize("solver", [W.SSM, W.AEM], ids=["ssm", "aem"])
def test_vaccination_with_events(orc, gpu, solver):
    w = W.config_vaccination(n_nodes=1600, days=120)
    w.solver = solver
    U, st = _compare(orc, gpu, w)
    assert st["events_applied"] > 0


def test_replicates_graph_replay_and_prevalence(orc, gpu):
    import torch
    w = W.config_sir_icum(n_nodes=300, days=60)
    w = W.Workload(**{**w.__dict__, "n_rep": 3, "u0": np.repeat(w.u0, 3, axis=0),
                      "v0": np.repeat(w.v0, 3, axis=0)})
    code, U0, V0, R0, err = orc.run(w)
    assert code == 0
    M = len(w.tspan)
    m = gpu.Model(w)
    pout = torch.zeros((3, M, 4), dtype=torch.int64, device="cuda")
    m.set_output(dense=True, n_tspan=M, prevalence=([1], [0, 1]), prev_out=pout)
    u0 = torch.as_tensor(np.ascontiguousarray(w.u0), device="cuda")
    v0 = torch.zeros((3, w.n_nodes, 0), dtype=torch.float64, device="cuda")
    U = torch.empty((3, M, w.n_nodes, 4), dtype=torch.int32, device="cuda")
    V = torch.empty((3, M, w.n_nodes, 0), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    for _ in range(3):
        U.fill_(-1)
        rc, st, er = m.run(w.tspan, w.seed, 3, u0, v0, U, V, stream=s)
        s.synchronize()
        assert np.array_equal(U.cpu().numpy(), U0)
        assert np.array_equal(pout.cpu().numpy(), outputs.prevalence_counts(U0, [1], [0, 1]))
    m.close()


def test_parse_errors_are_reported(gpu):
    w = W.parsed_model(["S -> b*Q -> I"], ["S", "I"], {"b": 1.0}, [[1, 0]], [0, 1])
    with pytest.raises(gpu.SimInfError) as e:
        gpu.Model(w)
    assert e.value.code == -11
    assert "Q" in e.value.err["message"]
