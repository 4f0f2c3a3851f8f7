"""Pins for the oracle's stochastic simulation against the mathematics.

- The chemical master equation (the forward equation of the CTMC of Eq.
  vectorJSDE) for tiny nodes, solved by a matrix exponential, against the
  oracle's empirical distribution over 1e5 independent nodes (chi-square);
  SIR, SIS, SISe with frozen phi and SISe3 per age class with distinct
  parameters, so that a wrong index, sign or transposed rate fails.
- Pure death: I(t) ~ Binomial(I0, exp(-gamma t)).
- All of the above for both solvers ('ssm' and 'aem').
- Mean-field limit: the ensemble mean of large nodes follows Eq. (ODE).
- Conservation of every node's population under the SSA.
- The post time step: phi follows the closed form of the Euler recursion.
"""
import math

import numpy as np
import pytest

from paper_1605_01421_gb300 import workloads as W

scipy = pytest.importorskip("scipy")
from scipy import stats  # noqa: E402
from scipy.linalg import expm  # noqa: E402
from scipy.integrate import solve_ivp  # noqa: E402


def _chi2_pvalue(observed, expected):
    """Chi-square goodness of fit with bins of expected count < 5 merged."""
    order = np.argsort(expected)
    obs, exp = [], []
    acc_o = acc_e = 0.0
    for i in order:
        acc_o += observed[i]
        acc_e += expected[i]
        if acc_e >= 5:
            obs.append(acc_o)
            exp.append(acc_e)
            acc_o = acc_e = 0.0
    if acc_e > 0:
        if exp:
            obs[-1] += acc_o
            exp[-1] += acc_e
        else:
            obs.append(acc_o)
            exp.append(acc_e)
    obs, exp = np.array(obs), np.array(exp)
    if len(obs) < 2:
        return 1.0
    stat = float(np.sum((obs - exp) ** 2 / exp))
    return float(stats.chi2.sf(stat, len(obs) - 1))


def _cme(states, rates_and_targets, p0_index, times):
    """p(t) = p0 expm(Q t) on an enumerated state space."""
    n = len(states)
    index = {s: i for i, s in enumerate(states)}
    Q = np.zeros((n, n))
    for i, s in enumerate(states):
        for rate, tgt in rates_and_targets(s):
            if rate > 0:
                Q[i, index[tgt]] += rate
                Q[i, i] -= rate
    p0 = np.zeros(n)
    p0[p0_index] = 1.0
    return {t: p0 @ expm(Q * t) for t in times}, index


# every law holds for both solvers of Sec. 3.4.2: the direct method and the
# all events method (next reaction method over private channel streams)
SOLVERS = pytest.mark.parametrize("solver", [W.SSM, W.AEM], ids=["ssm", "aem"])

NODES = 100_000
DAYS = (1, 2, 5, 10)


def _empirical(U, comps, index, day):
    X = U[0, day][:, comps]
    counts = np.zeros(len(index))
    keys, c = np.unique(X, axis=0, return_counts=True)
    for k, n in zip(keys, c):
        counts[index[tuple(int(v) for v in k)]] = n
    return counts


@SOLVERS
def test_sir_matches_cme(orc, solver):
    beta, gamma, N = 1.2, 0.4, 5
    states = [(s, i) for s in range(N + 1) for i in range(N + 1 - s)]

    def moves(st):
        s, i = st
        return [(beta * s * i / N, (s - 1, i + 1)), (gamma * i, (s, i - 1))]

    p, index = _cme(states, moves, states.index((4, 1)), DAYS)
    w = W.plain_model(W.SIR, np.tile([[4, 1, 0]], (NODES, 1)),
                      np.arange(0, 11), [beta, gamma], seed=2024)
    w.solver = solver
    code, U, V, R, err = orc.run(w)
    assert code == 0
    for d in DAYS:
        obs = _empirical(U, [0, 1], index, d)
        assert obs.sum() == NODES
        assert _chi2_pvalue(obs, p[d] * NODES) > 1e-3, d


@SOLVERS
def test_sis_matches_cme(orc, solver):
    # Sec. 2.1: R(x) = [beta x1 x2, gamma x2] without division by N
    beta, gamma, N = 0.3, 1.0, 5
    states = [(N - i, i) for i in range(N + 1)]

    def moves(st):
        s, i = st
        return [(beta * s * i, (s - 1, i + 1)), (gamma * i, (s + 1, i - 1))]

    p, index = _cme(states, moves, states.index((3, 2)), DAYS)
    w = W.plain_model(W.SIS, np.tile([[3, 2]], (NODES, 1)), np.arange(0, 11),
                      [beta, gamma], seed=77)
    w.solver = solver
    code, U, V, R, err = orc.run(w)
    assert code == 0
    for d in DAYS:
        obs = _empirical(U, [0, 1], index, d)
        assert _chi2_pvalue(obs, p[d] * NODES) > 1e-3, d


@SOLVERS
def test_sise_frozen_phi_matches_cme(orc, solver):
    # alpha = 0 and zero decay keep phi at v0, so the node is a linear
    # birth-death chain with S -> I at upsilon phi S and I -> S at gamma I
    upsilon, gamma, phi, N = 0.3, 0.7, 2.0, 5
    states = [(N - i, i) for i in range(N + 1)]

    def moves(st):
        s, i = st
        return [(upsilon * phi * s, (s - 1, i + 1)), (gamma * i, (s + 1, i - 1))]

    p, index = _cme(states, moves, states.index((5, 0)), DAYS)
    g = W.sise_gdata(upsilon=upsilon, gamma=gamma, alpha=0.0, betas=(0.0,) * 4)
    w = W.plain_model(W.SISE, np.tile([[5, 0]], (NODES, 1)), np.arange(0, 11),
                      g, seed=5, v0=np.full((NODES, 1), phi))
    w.solver = solver
    code, U, V, R, err = orc.run(w)
    assert code == 0
    assert np.all(V == phi)
    for d in DAYS:
        obs = _empirical(U, [0, 1], index, d)
        assert _chi2_pvalue(obs, p[d] * NODES) > 1e-3, d


@SOLVERS
def test_sise3_each_age_class_matches_cme(orc, solver):
    ups, gams, phi = (0.1, 0.35, 0.8), (0.9, 0.5, 0.2), 1.5
    n_nodes = 50_000
    u0 = np.tile([[4, 0, 3, 1, 2, 2]], (n_nodes, 1))
    g = W.sise3_gdata(upsilons=ups, gammas=gams, alpha=0.0, betas=(0.0,) * 4)
    w = W.plain_model(W.SISE3, u0, np.arange(0, 6), g, seed=9,
                      v0=np.full((n_nodes, 1), phi))
    w.solver = solver
    code, U, V, R, err = orc.run(w)
    assert code == 0
    for a in range(3):
        N = int(u0[0, 2 * a] + u0[0, 2 * a + 1])
        states = [(N - i, i) for i in range(N + 1)]

        def moves(st, a=a):
            s, i = st
            return [(ups[a] * phi * s, (s - 1, i + 1)),
                    (gams[a] * i, (s + 1, i - 1))]

        p, index = _cme(states, moves,
                        states.index((int(u0[0, 2 * a]), int(u0[0, 2 * a + 1]))),
                        (1, 5))
        for d in (1, 5):
            obs = _empirical(U, [2 * a, 2 * a + 1], index, d)
            assert _chi2_pvalue(obs, p[d] * n_nodes) > 1e-3, (a, d)


@SOLVERS
def test_pure_death_is_binomial(orc, solver):
    gamma, I0 = 0.25, 12
    w = W.plain_model(W.SIR, np.tile([[0, I0, 0]], (40_000, 1)),
                      np.arange(0, 9), [0.0, gamma], seed=31)
    w.solver = solver
    code, U, V, R, err = orc.run(w)
    assert code == 0
    for d in (1, 3, 8):
        q = math.exp(-gamma * d)
        obs = np.bincount(U[0, d][:, 1], minlength=I0 + 1).astype(float)
        exp = stats.binom.pmf(np.arange(I0 + 1), I0, q) * obs.sum()
        assert _chi2_pvalue(obs, exp) > 1e-3
    # reactions are the recoveries: total drop of I
    assert R[0] == I0 * 40_000 - U[0, -1][:, 1].sum()


@SOLVERS
def test_mean_field_limit(orc, solver):
    beta, gamma, N, I0 = 0.5, 0.2, 20_000, 400
    nodes = 60
    w = W.plain_model(W.SIR, np.tile([[N - I0, I0, 0]], (nodes, 1)),
                      np.arange(0, 31), [beta, gamma], seed=8)
    w.solver = solver
    code, U, V, R, err = orc.run(w)
    assert code == 0

    def f(t, x):
        s, i = x[0], x[1]
        return [-beta * s * i / N, beta * s * i / N - gamma * i]

    sol = solve_ivp(f, (0, 30), [N - I0, I0], t_eval=np.arange(31),
                    rtol=1e-10, atol=1e-8)
    for d in (5, 10, 20, 30):
        mean = U[0, d].mean(axis=0)
        assert abs(mean[0] - sol.y[0, d]) / N < 0.01
        assert abs(mean[1] - sol.y[1, d]) / N < 0.01


@SOLVERS
def test_ssa_conserves_population(orc, solver):
    w = W.config_sise3(n_nodes=300, days=60, gen_seed=4, events_per_node_day=0)
    w.solver = solver
    code, U, V, R, err = orc.run(w)
    assert code == 0 and R[0] > 0
    for a in range(3):
        tot = U[0][:, :, 2 * a] + U[0][:, :, 2 * a + 1]
        assert np.all(tot == tot[0:1])
    w = W.config_sir(n_nodes=50, days=40)
    code, U, V, R, err = orc.run(w)
    assert np.all(U[0].sum(axis=2) == 100)


def test_post_time_step_closed_form(orc):
    # no transitions (upsilon = gamma = 0): I/N is constant, so the Euler
    # recursion phi_{n+1} = phi_n + alpha I/N - beta phi_n has the closed form
    # phi_n = (1-beta)^n phi_0 + (alpha I/N / beta) (1 - (1-beta)^n).
    alpha, b = 1.3, 0.1
    u0 = np.array([[90, 10], [40, 60], [0, 0]])
    v0 = np.array([[0.0], [2.5], [4.0]])
    g = W.sise_gdata(upsilon=0.0, gamma=0.0, alpha=alpha, betas=(b,) * 4)
    w = W.plain_model(W.SISE, u0, np.arange(0, 366), g, v0=v0)
    code, U, V, R, err = orc.run(w)
    assert code == 0
    n = np.arange(366)
    for k in range(3):
        N = u0[k].sum()
        shed = alpha * u0[k, 1] / N if N > 0 else 0.0
        ref = (1 - b) ** n * v0[k, 0] + shed / b * (1 - (1 - b) ** n)
        assert np.allclose(V[0, :, k, 0], ref, rtol=1e-12, atol=1e-14)


def test_post_time_step_seasons(orc):
    # piecewise-constant decay: each season restarts the closed form
    alpha, betas, ends = 1.0, (0.05, 0.2, 0.12, 0.3), (91, 182, 273, 365)
    u0 = np.array([[80, 20]])
    g = W.sise_gdata(upsilon=0.0, gamma=0.0, alpha=alpha, betas=betas)
    w = W.plain_model(W.SISE, u0, np.arange(0, 731), g,
                      ldata=W.seasons_ldata(1, ends))
    code, U, V, R, err = orc.run(w)
    assert code == 0
    phi = V[0, :, 0, 0]
    shed = alpha * 0.2
    for T in range(1, 731):
        doy = (T - 1) % 365 + 1
        b = betas[0] if doy <= ends[0] else betas[1] if doy <= ends[1] else \
            betas[2] if doy <= ends[2] else betas[3]
        # one step of the recursion from the recorded previous value
        assert math.isclose(phi[T], (1 - b) * phi[T - 1] + shed,
                            rel_tol=1e-13, abs_tol=1e-15)


def test_initial_column_is_u0(orc):
    w = W.config_sir(n_nodes=20, days=10)
    code, U, V, R, err = orc.run(w)
    assert np.array_equal(U[0, 0], w.u0[0])


def test_node_without_infection_is_frozen(orc):
    # lambda = 0: nothing can fire, the node keeps its state
    u0 = np.array([[10, 0, 0], [9, 1, 0]])
    w = W.plain_model(W.SIR, u0, np.arange(0, 30), [0.5, 0.1], seed=3)
    code, U, V, R, err = orc.run(w)
    assert code == 0
    assert np.all(U[0, :, 0] == [10, 0, 0])
    assert np.all(U[0].sum(axis=2) == 10)


def test_sise_sp_two_farms_follow_the_linear_recursion(orc):
    # no transitions: the coupled Euler step is a linear recursion
    # phi' = A phi + b, A = [[1 - c - beta, c N2 / N1], [c N1 / N2, 1 - c - beta]],
    # c = D / d, b = alpha I / N
    alpha, beta, D, d = 0.7, 0.1, 0.2, 1500.0
    u0 = np.array([[30, 10], [5, 15]])
    g = W.sise_sp_gdata(upsilon=0.0, gamma=0.0, alpha=alpha, betas=(beta,) * 4,
                        coupling=D)
    w = W.plain_model(W.SISE_SP, u0, np.arange(0, 41), g, v0=np.array([[0.3], [1.1]]))
    w.neighbors = (np.array([0, 1, 2]), np.array([1, 0], np.int32), np.array([d, d]))
    code, U, V, R, err = orc.run(w)
    assert code == 0
    N = u0.sum(1).astype(float)
    c = D / d
    A = np.array([[1 - c - beta, c * N[1] / N[0]], [c * N[0] / N[1], 1 - c - beta]])
    b = alpha * u0[:, 1] / N
    phi = np.array([0.3, 1.1])
    for t in range(1, 41):
        phi = A @ phi + b
        assert np.allclose(V[0, t, :, 0], phi, rtol=1e-12, atol=0)


def test_sise_sp_coupling_conserves_total_pressure(orc):
    # alpha = 0 and no decay: the coupling only moves N_i phi_i between
    # farms with symmetric distances, so sum_i N_i phi_i stays constant
    rng = np.random.default_rng(3)
    n = 60
    x, y = rng.uniform(0, 5000, n), rng.uniform(0, 5000, n)
    u0 = np.stack([rng.integers(5, 50, n), rng.integers(0, 10, n)], 1)
    g = W.sise_sp_gdata(upsilon=0.0, gamma=0.0, alpha=0.0, betas=(0.0,) * 4,
                        coupling=0.05)
    w = W.plain_model(W.SISE_SP, u0, np.arange(0, 50), g,
                      v0=rng.uniform(0, 2, (n, 1)))
    w.neighbors = W.distance_neighbors(x, y, 1500.0)
    assert len(w.neighbors[1]) > n
    code, U, V, R, err = orc.run(w)
    assert code == 0
    tot = (V[0, :, :, 0] * u0.sum(1)).sum(axis=1)
    assert np.allclose(tot, tot[0], rtol=1e-11)
    assert not np.allclose(V[0, -1, :, 0], V[0, 0, :, 0])


def test_sise_sp_without_coupling_is_sise(orc):
    w = W.config_sise(n_nodes=300, days=60, gen_seed=5)
    g = w.gdata
    w_sp = W.plain_model(W.SISE_SP, w.u0, w.tspan, np.r_[g, 0.0], events=w.events,
                         seed=w.seed)
    rng = np.random.default_rng(1)
    w_sp.neighbors = W.distance_neighbors(rng.uniform(0, 1e4, 300), rng.uniform(0, 1e4, 300),
                                          2000.0)
    c1, U1, V1, R1, e1 = orc.run(w)
    c2, U2, V2, R2, e2 = orc.run(w_sp)
    assert c1 == 0 and c2 == 0
    assert np.array_equal(U1, U2) and np.array_equal(V1, V2)
