"""Pins for the oracle's all events method ('aem', Sec. 3.4.2) beyond the
laws it shares with the direct method (those run for both solvers in
test_oracle_law.py).

- Channel streams: a node whose only live channel is I -> R fires at
  t + E / a with E = -log u, u from the channel's own Philox counter
  (draw, node, transition, 3 << 24 | replicate); recomputed here from the
  Philox known-answer-pinned generator, the open-interval uniform's
  definition and math.log, for several nodes, replicates and two
  consecutive firings of the same channel.
- Rates that change at day boundaries (post time step, events): the CME with
  a generator that is constant within each day, and a pure-death process
  with an enter event (a sum of two binomials).
- The same model with events under both solvers: equal laws of the final
  state (two-sample test).
"""
import math

import numpy as np
import pytest

from paper_1605_01421_gb300 import workloads as W

scipy = pytest.importorskip("scipy")
from scipy import stats  # noqa: E402
from scipy.linalg import expm  # noqa: E402


def _chi2(obs, exp):
    keep = exp >= 5
    o = np.r_[obs[keep], obs[~keep].sum()]
    e = np.r_[exp[keep], exp[~keep].sum()]
    if e[-1] == 0:
        o, e = o[:-1], e[:-1]
    e = e * o.sum() / e.sum()
    return stats.chisquare(o, e).pvalue


def _u01(a, b):
    # the open interval uniform: 52 bits k, (k + 1/2) 2^-52
    k = (int(b) << 20) | (int(a) >> 12)
    return (k + 0.5) * 2.0 ** -52


def _channel_E(orc, seed, node, j, rep, c):
    x = orc.philox4x32_10([c, node, j, (3 << 24) | rep],
                          [seed & 0xFFFFFFFF, seed >> 32])
    return -math.log(_u01(x[0], x[1]))


def test_channel_streams_fix_the_firing_times(orc):
    gamma, seed, n_nodes, n_rep = 0.37, 0x1234_5678_9ABC, 40, 3
    # I0 = 2: the recovery channel (j = 1) fires at E0 / (2 gamma), then at
    # that time plus E1 / gamma (the fired channel draws again)
    u0 = np.tile([[0, 2, 0]], (n_nodes, 1))
    days = 40
    w = W.plain_model(W.SIR, u0, np.arange(0, days + 1), [0.8, gamma], seed=seed,
                      n_rep=n_rep)
    w.solver = W.AEM
    code, U, V, R, err = orc.run(w)
    assert code == 0
    checked = 0
    for r in range(n_rep):
        for i in range(n_nodes):
            t1 = 0.0 + _channel_E(orc, seed, i, 1, r, 0) / (2 * gamma)
            t2 = t1 + _channel_E(orc, seed, i, 1, r, 1) / gamma
            I = U[r, :, i, 1]
            for d in range(days + 1):
                want = 2 - (t1 < d) - (t2 < d)
                if min(abs(t1 - d), abs(t2 - d)) < 1e-9:
                    continue  # a firing time within rounding of a day
                assert I[d] == want, (r, i, d, t1, t2)
                checked += 1
            # the infection channel (j = 0) never wakes: S = 0 throughout
            assert np.all(U[r, :, i, 0] == 0)
    assert checked > 0.99 * n_rep * n_nodes * (days + 1)


def test_rates_changed_by_the_post_time_step(orc):
    # SISe with alpha = 0: phi_{d+1} = phi_d - beta phi_d, deterministic, so
    # S -> I runs at upsilon phi_d S during day d + 1 and the law is
    # p(d) = p0 prod_k expm(Q(phi_k))
    ups, gamma, beta, phi0, N = 0.5, 0.3, 0.35, 3.0, 4
    nodes, days = 60_000, 6
    g = W.sise_gdata(upsilon=ups, gamma=gamma, alpha=0.0, betas=(beta,) * 4)
    for solver in (W.SSM, W.AEM):
        w = W.plain_model(W.SISE, np.tile([[4, 0]], (nodes, 1)), np.arange(0, days + 1),
                          g, seed=11, v0=np.full((nodes, 1), phi0))
        w.solver = solver
        code, U, V, R, err = orc.run(w)
        assert code == 0
        p = np.zeros(N + 1)
        p[0] = 1.0  # index = I
        phi = phi0
        for d in range(1, days + 1):
            Q = np.zeros((N + 1, N + 1))
            for i in range(N + 1):
                s = N - i
                if s > 0:
                    Q[i, i + 1] += ups * phi * s
                    Q[i, i] -= ups * phi * s
                if i > 0:
                    Q[i, i - 1] += gamma * i
                    Q[i, i] -= gamma * i
            p = p @ expm(Q)
            assert V[0, d, 0, 0] == pytest.approx(phi - beta * phi, rel=1e-12)
            phi = phi - beta * phi
            obs = np.bincount(U[0, d][:, 1], minlength=N + 1).astype(float)
            assert _chi2(obs, p * nodes) > 1e-3, (solver, d)


def test_rates_changed_by_an_enter_event(orc):
    # pure death I -> R at gamma I; at t = 3, five individuals enter I:
    # I(d) = Bin(I0, e^{-gamma d}) + Bin(5, e^{-gamma (d - 3)})
    gamma, I0, k, nodes = 0.3, 6, 5, 40_000
    rows = [(1, 3, i, 0, k, 0.0, 1, -1)  # enter into {I}
            for i in range(nodes)]
    w = W.plain_model(W.SIR, np.tile([[0, I0, 0]], (nodes, 1)), np.arange(0, 9),
                      [0.0, gamma], seed=21, events=W.make_events(rows))
    w.solver = W.AEM
    code, U, V, R, err = orc.run(w)
    assert code == 0
    for d in (2, 3, 4, 8):
        a = stats.binom.pmf(np.arange(I0 + 1), I0, math.exp(-gamma * d))
        b = (stats.binom.pmf(np.arange(k + 1), k, math.exp(-gamma * (d - 3)))
             if d >= 3 else np.r_[1.0])
        pmf = np.convolve(a, b)
        obs = np.bincount(U[0, d][:, 1], minlength=pmf.size).astype(float)
        assert obs.size == pmf.size
        assert _chi2(obs, pmf * nodes) > 1e-3, d


def test_both_solvers_agree_in_law_with_events(orc):
    w = W.config_sise3(n_nodes=3000, days=60, gen_seed=4)
    res = {}
    for solver in (W.SSM, W.AEM):
        w.solver = solver
        code, U, V, R, err = orc.run(w)
        assert code == 0, err
        res[solver] = U[0, -1]
    a, b = res[W.SSM], res[W.AEM]
    # events move the same animals' counts: the herd sizes agree exactly only
    # where the samplers agree, so compare the laws of the infected counts
    for c in (1, 3, 5):
        assert stats.ks_2samp(a[:, c], b[:, c]).pvalue > 1e-3, c
    # and the sample paths differ (different random streams)
    assert not np.array_equal(a, b)
