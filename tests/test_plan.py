"""The engine's host event schedule (sg_plan_events, host only) against a
plain restatement of the rules of Sec. 3.3 / Appendix A written here:

- E1 events (exit, enter, internal transfer) of a node run in the order of
  the day they fall on, the time on the first day (which also takes every
  earlier time), the event type, then their place in the list;
- E2 events (external transfers) of a day run in list order; the engine
  splits them into waves: an event goes one wave after the last earlier
  event of the same day that sampled its source, added to its source or
  sampled its destination, so that every node sees its samples and
  additions in list order.

Small tables check a hand-worked example; random tables (with replicate
event lists, events before the window and after it, and sizes that take the
parallel planner) check the whole schedule element by element."""
import numpy as np
import pytest

from paper_1605_01421_gb300 import binding


@pytest.fixture(scope="module")
def lib():
    try:
        return binding.lib()
    except (RuntimeError, OSError) as exc:  # library not built here
        pytest.skip(str(exc))


def _events(rows):
    cols = list(zip(*rows))
    return {"event": np.array(cols[0], np.int32), "time": np.array(cols[1], np.int32),
            "node": np.array(cols[2], np.int32), "dest": np.array(cols[3], np.int32),
            "rep": np.array(cols[4], np.int32) if len(cols) > 4 else None}


def _reference(ev, n_nodes, t0, t_end, slots):
    n = len(ev["event"])
    typ, tim, nod, dst = ev["event"], ev["time"], ev["node"], ev["dest"]
    rep = ev["rep"] if slots > 1 else np.zeros(n, np.int32)

    def day(e):
        return max(0, int(tim[e]) - t0 - 1)

    keep = [e for e in range(n) if tim[e] <= t_end]
    e1 = sorted((e for e in keep if typ[e] != 3),
                key=lambda e: (rep[e], nod[e], day(e), tim[e] if day(e) == 0 else 0, typ[e], e))
    buckets = {}
    for e in keep:
        if typ[e] == 3:
            buckets.setdefault((day(e), rep[e]), []).append(e)
    waves, wave_off = [], [0]
    for d in range(t_end - t0):
        for s in range(slots):
            b = sorted(buckets.get((d, s), []), key=lambda e: (tim[e], e))
            sampled, added, w_of = {}, {}, []
            for e in b:
                a, c = int(nod[e]), int(dst[e])
                w = max(sampled.get(a, 0), added.get(a, 0), sampled.get(c, 0)) + 1
                sampled[a] = w
                added[c] = max(added.get(c, 0), w)
                w_of.append(w)
            for w in range(1, max(w_of, default=0) + 1):
                waves.append([e for e, x in zip(b, w_of) if x == w])
            wave_off.append(len(waves))
    off = np.zeros(slots * n_nodes + 1, np.int64)
    for e in e1:
        off[rep[e] * n_nodes + nod[e] + 1] += 1
    return e1, np.cumsum(off), waves, wave_off, [day(e) for e in e1]


def _check(ev, n_nodes, t0, t_end, slots):
    got = binding.plan_events(ev, n_nodes, t0, t_end, slots)
    e1, off, waves, wave_off, days = _reference(ev, n_nodes, t0, t_end, slots)
    n_e1 = len(e1)
    assert got["n_e1"] == n_e1 and got["n_waves"] == len(waves)
    assert got["order"][:n_e1].tolist() == e1
    assert got["e1_day"].tolist() == days
    assert np.array_equal(got["e1_node_off"], off)
    assert got["e2_wave_off"].tolist() == wave_off
    we = got["wave_ev"]
    assert we[0] == n_e1 and len(we) == len(waves) + 1
    for w, members in enumerate(waves):
        assert got["order"][we[w]:we[w + 1]].tolist() == members
    return got


def test_hand_worked_waves(lib):
    # one day, three nodes: 0 -> 1, 1 -> 2, 0 -> 2, 2 -> 0
    #   0 -> 1: first touch of 0 and 1                          wave 1
    #   1 -> 2: samples 1, which received in wave 1              wave 2
    #   0 -> 2: samples 0 again (sampled in wave 1)              wave 2
    #   2 -> 0: samples 2, which received in wave 2              wave 3
    ev = _events([(3, 1, 0, 1), (3, 1, 1, 2), (3, 1, 0, 2), (3, 1, 2, 0)])
    got = _check(ev, 3, 0, 1, 1)
    we, order = got["wave_ev"], got["order"]
    assert [order[we[w]:we[w + 1]].tolist() for w in range(3)] == [[0], [1, 2], [3]]


def test_hand_worked_e1_order(lib):
    # node 0: enter (day 2), exit (day 1), internal (day 1), exit (time -3 ->
    # day 0), enter (time 0 -> day 0); window t0 = 0 .. 5
    ev = _events([(1, 2, 0, 0), (0, 1, 0, 0), (2, 1, 0, 0), (0, -3, 0, 0), (1, 0, 0, 0),
                  (0, 9, 0, 0)])
    got = _check(ev, 1, 0, 5, 1)
    # day 0 by time (-3, then 0), day 1 by type (exit, internal), then day 2;
    # the event at time 9 is past the window
    assert got["order"].tolist() == [3, 4, 1, 2, 0]
    assert got["e1_day"].tolist() == [0, 0, 0, 0, 1]


@pytest.mark.parametrize("n,slots", [(3000, 1), (3000, 3), (40_000, 1), (40_000, 4)])
def test_random_tables(lib, n, slots):
    rng = np.random.default_rng(n + slots)
    n_nodes, t0, t_end = 37, 3, 40
    ev = {"event": rng.integers(0, 4, n).astype(np.int32),
          "time": rng.integers(-2, 46, n).astype(np.int32),
          "node": rng.integers(0, n_nodes, n).astype(np.int32),
          "dest": rng.integers(0, n_nodes, n).astype(np.int32),
          "rep": rng.integers(0, slots, n).astype(np.int32)}
    _check(ev, n_nodes, t0, t_end, slots)


def test_wave_invariant(lib):
    # inside a wave no node is sampled twice, and no sampled node is also a
    # destination of the same wave
    rng = np.random.default_rng(9)
    n, n_nodes = 5000, 25
    ev = {"event": np.full(n, 3, np.int32), "time": rng.integers(1, 6, n).astype(np.int32),
          "node": rng.integers(0, n_nodes, n).astype(np.int32),
          "dest": rng.integers(0, n_nodes, n).astype(np.int32), "rep": None}
    got = binding.plan_events(ev, n_nodes, 0, 5)
    we, order = got["wave_ev"], got["order"]
    for w in range(got["n_waves"]):
        members = order[we[w]:we[w + 1]]
        src, dst = ev["node"][members], ev["dest"][members]
        assert len(set(src.tolist())) == len(src)
        assert not set(src.tolist()) & set(dst.tolist()) - set(
            src[src == dst].tolist())


def test_rejects_out_of_range(lib):
    ev = _events([(3, 1, 0, 5)])
    with pytest.raises(binding.SimInfError):
        binding.plan_events(ev, 3, 0, 2)
    ev = _events([(0, 1, 0, 0, 2)])
    with pytest.raises(binding.SimInfError):
        binding.plan_events(ev, 3, 0, 2, slots=2)
