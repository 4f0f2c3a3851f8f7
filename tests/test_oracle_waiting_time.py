"""Direct pins of the direct method's waiting-time law (Appendix A: with
total rate lambda, the next transition comes after tau = -log(r1) / lambda,
r1 uniform on (0, 1), i.e. tau ~ Exp(lambda)).

The oracle records, through a test hook, the waiting time of the first
draw of every node-day with lambda > 0 (whether or not it passes the day's
end).  At the first day the state is u0, so lambda is known here from the
rate definitions (SIR: beta S I / N + gamma I, Eq. (SIR)):

- lambda tau over thousands of nodes with different lambda follows Exp(1)
  (Kolmogorov-Smirnov, p > 0.001), and the fraction of first draws that pass
  the day's end is e^-lambda on average (the probability of no transition in
  a unit of time);
- each tau equals -log(u) / lambda with u the open-interval uniform built,
  by its definition, from words 0-1 of Philox call (0, node, T, replicate)
  (the known-answer-pinned generator) and math.log, for every recorded
  node-day, replicate and day;
- node-days with lambda = 0 take no draw (no record).
Planted mistakes in the oracle (a missing division by lambda, words 2-3
instead of 0-1, the day or the node missing from the counter) each fail one
of these checks.
"""
import math

import numpy as np
import pytest

from paper_1605_01421_gb300 import workloads as W

scipy = pytest.importorskip("scipy")
from scipy import stats  # noqa: E402

BETA, GAMMA = 0.16, 0.077


def _u01(a, b):
    # the open-interval uniform: 52 bits k = (b << 20) | (a >> 12), (k + 1/2) 2^-52
    k = (int(b) << 20) | (int(a) >> 12)
    return (k + 0.5) * 2.0 ** -52


def _sir_nodes(n, seed):
    rng = np.random.default_rng(seed)
    S = rng.integers(0, 400, n)
    I = rng.integers(0, 60, n)
    R = rng.integers(0, 50, n)
    I[rng.random(n) < 0.05] = 0  # some nodes with lambda = 0
    return np.stack([S, I, R], axis=1).astype(np.int32)


def _lambda_sir(u):
    S, I, R = (u[:, k].astype(np.float64) for k in range(3))
    n = S + I + R
    inf = np.where(n > 0, (BETA * S * I) / np.where(n > 0, n, 1.0), 0.0)
    return inf + GAMMA * I


def test_first_waiting_time_is_exponential(orc):
    n = 20_000
    u0 = _sir_nodes(n, 3)
    w = W.plain_model(W.SIR, u0, np.arange(0, 2), [BETA, GAMMA], seed=77)
    rec, (code, U, V, R, err) = orc.first_waiting_times(w, cap=2 * n)
    assert code == 0
    lam = _lambda_sir(u0)
    live = lam > 0
    # one record per node-day with lambda > 0, none for the others
    assert rec["T"].size == int(live.sum())
    assert np.all(rec["T"] == 1)
    assert np.array_equal(np.sort(rec["node"]), np.flatnonzero(live))
    x = lam[rec["node"]] * rec["tau"]
    assert stats.kstest(x, "expon").pvalue > 1e-3
    # the first draw passes the day's end (t + tau >= 1) with probability e^-lambda
    passed = (rec["tau"] >= 1.0).astype(np.float64)
    p = np.exp(-lam[rec["node"]])
    z = (passed.sum() - p.sum()) / math.sqrt((p * (1 - p)).sum())
    assert abs(z) < 4.0


def test_first_waiting_time_from_the_stream(orc):
    # every recorded tau equals -log(u) / lambda, u from Philox call
    # (0, node, T, (0 << 24) | rep); on day 1 lambda is known from u0, on
    # later days from the recorded state at the start of that day
    n, days, n_rep, seed = 300, 6, 3, 0x0BAD_5EED_1234
    u0 = _sir_nodes(n, 4)
    w = W.plain_model(W.SIR, u0, np.arange(0, days + 1), [BETA, GAMMA], seed=seed,
                      n_rep=n_rep)
    rec, (code, U, V, R, err) = orc.first_waiting_times(w, cap=n * days * n_rep)
    assert code == 0
    checked = 0
    for r, i, T, tau in zip(rec["rep"], rec["node"], rec["T"], rec["tau"]):
        lam = float(_lambda_sir(U[r, T - 1, i][None, :])[0])
        assert lam > 0
        x = orc.philox4x32_10([0, int(i), int(T), (0 << 24) | int(r)],
                              [seed & 0xFFFFFFFF, seed >> 32])
        want = -math.log(_u01(x[0], x[1])) / lam
        assert tau == pytest.approx(want, rel=4e-16, abs=0.0), (r, i, T)
        checked += 1
    # every node-day with lambda > 0 at its start has a record
    lam_all = _lambda_sir(U[:, :-1].reshape(-1, 3)).reshape(n_rep, days, n)
    assert checked == int((lam_all > 0).sum())
