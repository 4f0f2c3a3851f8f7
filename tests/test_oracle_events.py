"""Pins for the oracle's scheduled-event stage (Sec. 3.3, Appendix B).

Forced outcomes reproduce the five illustrated events of Appendix B (the
count to move equals the selectable total, so the sample is determined); the
SIR event table of Sec. 4.1 and the vaccination matrices E (5 x 3) and N
(5 x 1) of Sec. 5.1 fix select / shift semantics; the urn sampling is
checked against the exact multivariate hypergeometric law; same-time order
and error checks follow Sec. 3.3 and Sec. 4.1.
"""
import itertools
import math

import numpy as np
import pytest

from paper_1605_01421_gb300 import workloads as W

EXIT, ENTER, INTERNAL, EXTERNAL = 0, 1, 2, 3


def sise3_tables():
    S, G, E, N = W.sise3_tables()
    return E, N


def test_appendix_b_forced_outcomes(orc):
    E, N = sise3_tables()
    # exit: remove one individual of age class 3 ({S3, I3} = E[, 6], 1-based)
    u = [3, 2, 4, 1, 0, 1]
    rc, out, _ = orc.apply_event(E, N, EXIT, u, n=1, select=5)
    assert rc == 0 and list(out) == [3, 2, 4, 1, 0, 0]
    # enter: three susceptibles into age class 1 (E[, 1] = {S1})
    rc, out, _ = orc.apply_event(E, N, ENTER, u, n=3, select=0)
    assert rc == 0 and list(out) == [6, 2, 4, 1, 0, 1]
    # external transfer: one individual of age 3 from node 14 to node 23
    dest = [5, 0, 2, 2, 7, 1]
    rc, out, dst = orc.apply_event(E, N, EXTERNAL, u, dest, n=1, select=5)
    assert rc == 0 and list(out) == [3, 2, 4, 1, 0, 0]
    assert list(dst) == [5, 0, 2, 2, 7, 2]
    # internal transfer (ageing) of three individuals of age 1 via N[, 1]
    u2 = [2, 1, 4, 1, 0, 1]
    rc, out, _ = orc.apply_event(E, N, INTERNAL, u2, n=3, select=3, shift=0)
    assert rc == 0 and list(out) == [0, 0, 6, 2, 0, 1]
    # external transfer with shift: age class 2 moved and aged via N[, 2]
    u3 = [1, 1, 2, 1, 0, 0]
    rc, out, dst = orc.apply_event(E, N, EXTERNAL, u3, dest, n=3, select=4,
                                   shift=1)
    assert rc == 0 and list(out) == [1, 1, 0, 0, 0, 0]
    assert list(dst) == [5, 0, 2, 2, 9, 2]


def test_sir_event_table_semantics(orc):
    # Sec. 4.1 event table, with forced sizes where the sample is random
    S, G, E, N = W.sir_tables()
    # 1: enter 5 into S (select 1) of node 3
    rc, out, _ = orc.apply_event(E, N, ENTER, [0, 0, 0], n=5, select=0)
    assert list(out) == [5, 0, 0]
    # 2: move 7 from node 1 to node 3 among S, I, R (select 4)
    rc, src, dst = orc.apply_event(E, N, EXTERNAL, [4, 2, 1], [5, 0, 0], n=7,
                                   select=3)
    assert rc == 0 and list(src) == [0, 0, 0] and list(dst) == [9, 2, 1]
    # 3: exit 20% of node 2 (select 4): round(0.2 * 20) = 4 individuals
    for seed in range(20):
        rc, out, _ = orc.apply_event(E, N, EXIT, [10, 6, 4], n=0,
                                     proportion=0.2, select=3, seed=seed)
        assert rc == 0 and sum(out) == 16 and np.all(out >= 0)
        assert np.all(out <= [10, 6, 4])
    # 4: enter 1 infected (select 2) into node 1
    rc, out, _ = orc.apply_event(E, N, ENTER, [3, 0, 0], n=1, select=1)
    assert list(out) == [3, 1, 0]


def test_vaccination_matrices(orc):
    # Sec. 5.1: compartments S, I, Icum, R, V; E[, 3] = {S, I, R};
    # N[, 1] moves S +4, I +3, R +1 into V; Icum is never selected
    E = np.array([[1, 1, 1], [0, 1, 1], [0, 0, 0], [0, 1, 1], [0, 1, 0]])
    N = np.array([[4], [3], [0], [1], [0]])
    u = [6, 3, 9, 2, 0]
    rc, out, _ = orc.apply_event(E, N, INTERNAL, u, n=11, select=2, shift=0)
    assert rc == 0 and list(out) == [0, 0, 9, 0, 11]
    for seed in range(30):
        rc, out, _ = orc.apply_event(E, N, INTERNAL, u, n=5, select=2, shift=0,
                                     seed=seed, event_index=seed)
        assert rc == 0
        assert out[2] == 9 and out[4] == 5
        assert out[0] + out[1] + out[3] == 6
        assert out[0] <= 6 and out[1] <= 3 and out[3] <= 2
    # proportion 0.8 of S + I + R = 11 -> round(8.8) = 9 vaccinated
    rc, out, _ = orc.apply_event(E, N, INTERNAL, u, n=0, proportion=0.8,
                                 select=2, shift=0)
    assert rc == 0 and out[4] == 9 and out[2] == 9


def test_proportion_rounds_half_away_from_zero(orc):
    E = np.array([[1], [1]])
    N = np.zeros((2, 1), int)
    # 0.5 * 3 = 1.5 -> 2;  0.5 * 5 = 2.5 -> 3;  0.25 * 2 = 0.5 -> 1
    for u, p, k in (([2, 1], 0.5, 2), ([3, 2], 0.5, 3), ([1, 1], 0.25, 1),
                    ([4, 0], 0.0, 0), ([4, 3], 1.0, 7)):
        rc, out, _ = orc.apply_event(E, N, EXIT, u, n=0, proportion=p, select=0)
        assert rc == 0 and sum(u) - sum(out) == k


def test_urn_sampling_is_multivariate_hypergeometric(orc):
    stats = pytest.importorskip("scipy.stats")
    E = np.array([[1], [1], [1]])
    N = np.zeros((3, 1), int)
    u, k = [5, 3, 2], 4
    draws = 20000
    counts = {}
    for e in range(draws):
        rc, out, _ = orc.apply_event(E, N, EXIT, u, n=k, select=0, seed=17,
                                     event_index=e)
        taken = tuple(int(a - b) for a, b in zip(u, out))
        counts[taken] = counts.get(taken, 0) + 1
    support = [t for t in itertools.product(range(6), range(4), range(3))
               if sum(t) == k]
    pmf = np.array([math.comb(5, a) * math.comb(3, b) * math.comb(2, c)
                    for a, b, c in support], float) / math.comb(10, k)
    obs = np.array([counts.get(t, 0) for t in support], float)
    assert obs.sum() == draws
    p = stats.chisquare(obs, pmf * draws).pvalue
    assert p > 1e-3


def test_event_errors(orc):
    E, N = sise3_tables()
    # more individuals than the selected compartments hold (Sec. 4.1)
    rc, _, _ = orc.apply_event(E, N, EXIT, [1, 1, 0, 0, 0, 0], n=3, select=3)
    assert rc == -2
    # a shift that leaves the compartments
    Nbad = N.copy()
    Nbad[4, 1] = 5
    rc, _, _ = orc.apply_event(E, Nbad, INTERNAL, [0, 0, 0, 0, 2, 0], n=1,
                               select=5, shift=1)
    assert rc == -3


def _run_events(orc, kind, u0, rows, tspan=(0, 1, 2), rep=None):
    g = {W.SIR: [0.0, 0.0], W.SISE: W.sise_gdata(0.0, 0.0, 0.0, (0.0,) * 4)}[kind]
    w = W.plain_model(kind, u0, np.asarray(tspan), g,
                      events=W.make_events(rows, rep))
    return orc.run(w)


def test_same_time_order_exit_before_enter(orc):
    # listed enter-then-exit at the same time: the exit runs first (Sec. 3.3)
    rows = [(ENTER, 1, 0, 0, 5, 0.0, 0, -1), (EXIT, 1, 0, 0, 8, 0.0, 0, -1)]
    code, U, V, R, err = _run_events(orc, W.SIR, [[5, 0, 0]], rows)
    assert code == -2 and err["event"] == 1 and err["day"] == 1
    rows = [(ENTER, 1, 0, 0, 3, 0.0, 0, -1), (EXIT, 1, 0, 0, 5, 0.0, 0, -1)]
    code, U, V, R, err = _run_events(orc, W.SIR, [[5, 0, 0]], rows)
    assert code == 0 and list(U[0, 1, 0]) == [3, 0, 0]


def test_e1_before_e2(orc):
    # an external transfer listed before an enter into its source still sees
    # the entered individuals: E1 events run before E2 events
    rows = [(EXTERNAL, 1, 0, 1, 3, 0.0, 0, -1), (ENTER, 1, 0, 0, 3, 0.0, 0, -1)]
    code, U, V, R, err = _run_events(orc, W.SIR, [[0, 0, 0], [1, 0, 0]], rows)
    assert code == 0
    assert list(U[0, 1, 0]) == [0, 0, 0] and list(U[0, 1, 1]) == [4, 0, 0]


def test_e2_list_order_chain(orc):
    # a chain of transfers within one day runs in list order
    rows = [(EXTERNAL, 2, 0, 1, 4, 0.0, 0, -1),
            (EXTERNAL, 2, 1, 2, 6, 0.0, 0, -1),
            (EXTERNAL, 2, 2, 0, 7, 0.0, 0, -1)]
    code, U, V, R, err = _run_events(orc, W.SIR, [[4, 0, 0], [2, 0, 0], [1, 0, 0]],
                                     rows)
    assert code == 0
    assert [int(x) for x in U[0, 2, :, 0]] == [7, 0, 0]
    assert [int(x) for x in U[0, 1, :, 0]] == [4, 2, 1]


def test_events_before_start_run_at_first_step_and_after_end_never(orc):
    rows = [(ENTER, -3, 0, 0, 2, 0.0, 0, -1), (ENTER, 0, 0, 0, 1, 0.0, 0, -1),
            (ENTER, 3, 0, 0, 50, 0.0, 0, -1)]
    code, U, V, R, err = _run_events(orc, W.SIR, [[0, 0, 0]], rows)
    assert code == 0
    assert [int(x) for x in U[0, :, 0, 0]] == [0, 3, 3]


def test_replicate_specific_events(orc):
    rows = [(ENTER, 1, 0, 0, 2, 0.0, 0, -1), (ENTER, 1, 0, 0, 5, 0.0, 0, -1)]
    g = [0.0, 0.0]
    w = W.plain_model(W.SIR, [[0, 0, 0]], np.arange(0, 3), g, n_rep=2,
                      events=W.make_events(rows, rep=[1, 0]))
    code, U, V, R, err = orc.run(w)
    assert code == 0
    assert U[0, 2, 0, 0] == 5 and U[1, 2, 0, 0] == 2


def test_invalid_tables_rejected(orc):
    for row in [(4, 1, 0, 0, 1, 0.0, 0, -1),      # unknown type
                (EXIT, 1, 7, 0, 1, 0.0, 0, -1),   # node out of range
                (EXTERNAL, 1, 0, 9, 1, 0.0, 0, -1),  # dest out of range
                (EXIT, 1, 0, 0, 1, 0.0, 9, -1),   # select out of range
                (EXIT, 1, 0, 0, -1, 0.0, 0, -1),  # negative n
                (EXIT, 1, 0, 0, 0, 1.5, 0, -1),   # proportion > 1
                (INTERNAL, 1, 0, 0, 1, 0.0, 0, -1)]:  # internal without shift
        code, U, V, R, err = _run_events(orc, W.SIR, [[5, 0, 0]], [row])
        assert code == -1, row


def test_whole_pipeline_conserves_totals(orc):
    # total population changes exactly by enters minus exits each day
    w = W.config_sise(n_nodes=200, days=60, gen_seed=12)
    code, U, V, R, err = orc.run(w)
    assert code == 0
    ev = w.events
    tot = U[0].sum(axis=(1, 2)).astype(np.int64)
    for T in range(1, 61):
        sel = ev["time"] == T
        enters = ev["n"][sel & (ev["event"] == ENTER)].sum()
        exits = ev["n"][sel & (ev["event"] == EXIT)].sum()
        assert tot[T] - tot[T - 1] == enters - exits
    assert np.all(U >= 0)


def test_replicate_range_equals_the_slice_of_a_full_run(orc):
    # each replicate's streams and events depend on its index only, so running
    # replicates 1-2 or 3-4 alone gives the same trajectories as the full run
    w = W.config_sise3(n_nodes=200, days=30, gen_seed=6, n_rep=5, per_rep_events=True,
                       median=50, sigma=1.0, hi=5000)
    code, U, V, R, err = orc.run(w)
    assert code == 0
    for r0 in (1, 3):
        c2, U2, V2, R2, e2 = orc.run(w, rep0=r0, n_rep=2)
        assert c2 == 0
        assert np.array_equal(U2, U[r0:r0 + 2])
        assert np.array_equal(V2.view(np.uint64), V[r0:r0 + 2].view(np.uint64))
        assert np.array_equal(R2, R[r0:r0 + 2])
