"""Seeded synthetic inputs for the SimInf split-step method.

This module only builds input data: model tables (the matrices S, G, E, N and
the data vectors ldata / gdata that the paper's model slots hold, Sec. 3.2),
initial states and scheduled-event tables (Sec. 3.3).  It does none of the
method's arithmetic.  Both the CUDA path and the CPU oracle consume what it
returns, so their results can be compared on identical inputs.

The paper's datasets (Swedish cattle data, Sec. 1; the package's ``nodes``,
``u0_SISe`` and ``events_SISe`` data, Sec. 4.2) are not available, so the
cattle-shaped workloads are synthetic: log-normal herd sizes, a directed
heavy-tailed movement network, and daily enter / exit / internal-transfer /
external-transfer events whose sizes are geometric with mean 3.  The
generator tracks every node's per-age-class totals through the event order
the solver uses, which the SSA leaves unchanged, so every generated event is
valid whatever the stochastic trajectory.

All layouts are 0-based: ``node``, ``dest``, ``select`` and ``shift`` index
from 0 and ``shift = -1`` means "no shift".
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SIR, SIS, SISE, SISE3, SISE_SP, GENERIC = 0, 1, 2, 3, 4, 5
# solvers (Sec. 3.4.2): split-step direct SSA, all events method
SSM, AEM = 0, 1
EXIT, ENTER, INTERNAL, EXTERNAL = 0, 1, 2, 3
KIND_NAMES = {SIR: "SIR", SIS: "SIS", SISE: "SISe", SISE3: "SISe3", SISE_SP: "SISe_sp",
              GENERIC: "mparse"}


@dataclass
class Workload:
    name: str
    kind: int
    S: np.ndarray          # (n_comp, n_trans) int32
    G: np.ndarray          # (n_trans, n_trans) int32
    E: np.ndarray          # (n_comp, n_select) int32
    N: np.ndarray          # (n_comp, n_shift) int32
    gdata: np.ndarray      # (n_gdata,) float64
    ldata: np.ndarray      # (n_ldata, n_nodes) float64
    n_v: int
    u0: np.ndarray         # (n_rep, n_nodes, n_comp) int32
    v0: np.ndarray         # (n_rep, n_nodes, n_v) float64
    tspan: np.ndarray      # (M,) int32, strictly increasing
    events: dict | None    # event table, see empty_events()
    seed: int
    n_rep: int = 1
    meta: dict = field(default_factory=dict)
    # SISe_sp: neighbour lists (ptr (n_nodes + 1,), idx, distance) or None
    neighbors: tuple | None = None
    # solver: SSM (direct SSA per day) or AEM (all events method)
    solver: int = 0
    # GENERIC: the model as transition strings (Sec. 3.5): a dict with
    # "transitions", "compartments", "gdata_names"; S and G are then None
    # (each side derives them from the strings)
    generic: dict | None = None

    @property
    def n_nodes(self) -> int:
        return int(self.u0.shape[1])

    @property
    def n_comp(self) -> int:
        if self.generic is not None:
            return len(self.generic["compartments"])
        return int(self.S.shape[0])

    @property
    def n_days(self) -> int:
        return int(self.tspan[-1] - self.tspan[0])

    @property
    def n_events(self) -> int:
        return 0 if self.events is None else int(len(self.events["event"]))


def empty_events():
    return {k: np.zeros(0, dtype=np.float64 if k == "proportion" else np.int32)
            for k in ("event", "time", "node", "dest", "n", "proportion",
                      "select", "shift")} | {"rep": None}


def make_events(rows, rep=None):
    """Event table from rows (event, time, node, dest, n, proportion, select,
    shift), all 0-based."""
    ev = empty_events()
    if rows:
        cols = list(zip(*rows))
        for k, c in zip(("event", "time", "node", "dest", "n", "proportion",
                         "select", "shift"), cols):
            ev[k] = np.asarray(c, dtype=np.float64 if k == "proportion"
                               else np.int32)
    ev["rep"] = None if rep is None else np.asarray(rep, dtype=np.int32)
    return ev


# --------------------------------------------------------------------------
# Model tables (Sec. 3.2 slots).  G[k, j] != 0 marks that rate k must be
# recomputed after transition j.
# --------------------------------------------------------------------------

def sir_tables():
    """SIR, Eq. (SIR): S -> I, I -> R.  E columns: {S}, {I}, {R}, {S,I,R}
    as in the SIR event example of Sec. 4.1."""
    S = np.array([[-1, 0], [1, -1], [0, 1]], dtype=np.int32)
    G = np.array([[1, 1], [1, 1]], dtype=np.int32)
    E = np.array([[1, 0, 0, 1], [0, 1, 0, 1], [0, 0, 1, 1]], dtype=np.int32)
    N = np.zeros((3, 1), dtype=np.int32)
    return S, G, E, N


def sis_tables():
    """SIS of Sec. 2.1: S + I -> 2I, I -> S.  E columns: {S}, {I}, {S,I}."""
    S = np.array([[-1, 1], [1, -1]], dtype=np.int32)
    G = np.array([[1, 1], [1, 1]], dtype=np.int32)
    E = np.array([[1, 0, 1], [0, 1, 1]], dtype=np.int32)
    N = np.zeros((2, 1), dtype=np.int32)
    return S, G, E, N


def sise_tables():
    """SISe (Sec. 4.2 without spatial coupling): S -> I at upsilon phi S,
    I -> S at gamma I.  Each rate depends only on its own source
    compartment."""
    S = np.array([[-1, 1], [1, -1]], dtype=np.int32)
    G = np.array([[1, 1], [1, 1]], dtype=np.int32)
    E = np.array([[1, 0, 1], [0, 1, 1]], dtype=np.int32)
    N = np.zeros((2, 1), dtype=np.int32)
    return S, G, E, N


def sise3_tables():
    """SISe3: compartments [S1, I1, S2, I2, S3, I3], transitions
    S_a -> I_a (2a) and I_a -> S_a (2a + 1).  E columns 0-2 = {S_a} (enter),
    3-5 = {S_a, I_a} (exit, transfers), as in the event table of Appendix B.
    N column 0 ages {S1, I1} into {S2, I2}; column 1 ages {S2, I2} into
    {S3, I3}."""
    S = np.zeros((6, 6), dtype=np.int32)
    G = np.zeros((6, 6), dtype=np.int32)
    for a in range(3):
        S[2 * a, 2 * a], S[2 * a + 1, 2 * a] = -1, 1
        S[2 * a, 2 * a + 1], S[2 * a + 1, 2 * a + 1] = 1, -1
        for j in (2 * a, 2 * a + 1):
            G[2 * a, j] = 1
            G[2 * a + 1, j] = 1
    E = np.zeros((6, 6), dtype=np.int32)
    for a in range(3):
        E[2 * a, a] = 1
        E[2 * a, 3 + a] = 1
        E[2 * a + 1, 3 + a] = 1
    N = np.zeros((6, 2), dtype=np.int32)
    N[0, 0] = N[1, 0] = 2
    N[2, 1] = N[3, 1] = 2
    return S, G, E, N


def seasons_ldata(n_nodes, ends=(91, 182, 273, 365)):
    return np.tile(np.asarray(ends, dtype=np.float64)[:, None], (1, n_nodes))


def sise_gdata(upsilon=0.0173, gamma=0.1, alpha=1.0, betas=(0.1,) * 4):
    return np.array([upsilon, gamma, alpha, *betas], dtype=np.float64)


def sise_sp_gdata(upsilon=0.012, gamma=0.1, alpha=1.0, betas=(0.10, 0.12, 0.12, 0.10),
                  coupling=0.2):
    """SISe_sp global data of Sec. 4.2: [upsilon, gamma, alpha, beta_t1..t4,
    coupling D] (the paper's example values by default)."""
    return np.array([upsilon, gamma, alpha, *betas, coupling], dtype=np.float64)


def sise3_gdata(upsilons=(0.0173,) * 3, gammas=(0.1,) * 3, alpha=1.0,
                betas=(0.10, 0.12, 0.12, 0.10)):
    return np.array([*upsilons, *gammas, alpha, *betas], dtype=np.float64)


def _tile_rep(a, n_rep):
    # a C-ordered, writable copy (np.array would keep the broadcast's order)
    return np.broadcast_to(a[None], (n_rep,) + a.shape).copy(order="C")


def plain_model(kind, u0, tspan, gdata, seed=42, n_rep=1, events=None,
                ldata=None, v0=None, name=None):
    """A workload on explicit initial state ``u0`` (n_nodes, n_comp) or
    (n_rep, n_nodes, n_comp)."""
    tables = {SIR: sir_tables, SIS: sis_tables, SISE: sise_tables,
              SISE3: sise3_tables, SISE_SP: sise_tables}[kind]()
    S, G, E, N = tables
    u0 = np.asarray(u0, dtype=np.int32)
    if u0.ndim == 2:
        u0 = _tile_rep(u0, n_rep)
    n_nodes = u0.shape[1]
    n_v = 1 if kind in (SISE, SISE3, SISE_SP) else 0
    if ldata is None:
        ldata = (seasons_ldata(n_nodes) if n_v
                 else np.zeros((0, n_nodes), dtype=np.float64))
    if v0 is None:
        v0 = np.zeros((n_rep, n_nodes, n_v), dtype=np.float64)
    v0 = np.asarray(v0, dtype=np.float64)
    if v0.ndim == 2:
        v0 = _tile_rep(v0, n_rep)
    return Workload(name or KIND_NAMES[kind], kind, S, G, E, N,
                    np.asarray(gdata, dtype=np.float64),
                    np.asarray(ldata, dtype=np.float64), n_v, u0, v0,
                    np.asarray(tspan, dtype=np.int32),
                    events if events is not None else empty_events(),
                    int(seed), int(n_rep))


def parsed_model(transitions, compartments, gdata, u0, tspan, seed=42, n_rep=1,
                 events=None, E=None, N=None, name="mparse model"):
    """A model given as transition strings "LHS -> propensity -> RHS" (Sec.
    3.5); gdata is an ordered mapping name -> value.  S and G are left to the
    parsers of the two sides."""
    comps = list(compartments)
    C = len(comps)
    u0 = np.asarray(u0, dtype=np.int32)
    if u0.ndim == 2:
        u0 = _tile_rep(u0, n_rep)
    n_nodes = u0.shape[1]
    E = np.zeros((C, 0), np.int32) if E is None else np.asarray(E, np.int32)
    N = np.zeros((C, 0), np.int32) if N is None else np.asarray(N, np.int32)
    return Workload(name, GENERIC, None, None, E, N,
                    np.array(list(gdata.values()), dtype=np.float64),
                    np.zeros((0, n_nodes), dtype=np.float64), 0, u0,
                    np.zeros((u0.shape[0], n_nodes, 0), dtype=np.float64),
                    np.asarray(tspan, dtype=np.int32),
                    events if events is not None else empty_events(), int(seed),
                    int(u0.shape[0]),
                    generic={"transitions": list(transitions), "compartments": comps,
                             "gdata_names": list(gdata.keys())})


# The model-parser examples of Sec. 3.5 (transition strings as printed).
MPARSE_SIR = ["S -> b*S*I/(S+I+R) -> I", "I -> g*I -> R"]
MPARSE_SIR_ICUM = ["S -> b*S*I/(S+I+R) -> I + Icum", "I -> g*I -> R"]
MPARSE_PREDATOR_PREY = ["@ -> bR*R -> R", "R -> (dR+(bR-dR)*R/K)*R -> @",
                        "R -> alpha/(1+w*R)*R*F -> @", "@ -> bF*alpha/(1+w*R)*R*F -> F",
                        "F -> dF*F -> @"]
PREDATOR_PREY_GDATA = {"bR": 2.0, "bF": 2.0, "dR": 1.0, "K": 1000.0, "alpha": 0.007,
                       "w": 0.0035, "dF": 2.0}


def config_predator_prey(n_nodes=1000, days=99, seed=123, n_rep=1):
    """The Rosenzweig-MacArthur predator-prey model of Sec. 3.5 from its
    transition strings: R = 1000 prey and F = 100 predators in every node,
    tspan 1..days+1, the paper's parameters."""
    u0 = np.tile(np.array([[1000, 100]], dtype=np.int32), (n_nodes, 1))
    return parsed_model(MPARSE_PREDATOR_PREY, ["R", "F"], PREDATOR_PREY_GDATA, u0,
                        np.arange(1, days + 2), seed=seed, n_rep=n_rep,
                        name=f"PredatorPrey {n_nodes} nodes x {days} days")


def config_sir_icum(n_nodes=1000, days=149, seed=123):
    """SIR with the incidence counter Icum (Sec. 3.5): S=99 I=1 Icum=0 R=0,
    b = 0.16, g = 0.077, tspan 1..days+1."""
    u0 = np.tile(np.array([[99, 1, 0, 0]], dtype=np.int32), (n_nodes, 1))
    return parsed_model(MPARSE_SIR_ICUM, ["S", "I", "Icum", "R"], {"b": 0.16, "g": 0.077},
                        u0, np.arange(1, days + 2), seed=seed,
                        name=f"SIR+Icum {n_nodes} nodes x {days} days")


def config_vaccination(n_nodes=1600, days=300, gen_seed=1005, seed=42, vaccinate=True,
                       events_per_node_day=0.41, n_seeded=16):
    """The vaccination example of Sec. 3.5 on a synthetic stand-in for its
    1,600 cattle herds: compartments S, I, Icum, R, V, the printed E and N
    (enter -> S; exit and external transfer sample S, I, R, V; vaccination
    samples S, I, R and shifts them to V), synthetic births, deaths and
    movements, one infected animal in each of `n_seeded` herds (the paper
    introduces one and averages 1,000 runs), and vaccination of 80% of the
    animals in herds 1-50 on day 21, 51-100 on day 22, ... (internal transfer,
    select 3, shift 1 in the paper's 1-based numbering)."""
    rng = np.random.default_rng(gen_seed)
    herd = lognormal_herds(rng, n_nodes, 50, 1.0, 2, 5000)
    S = herd.copy()
    I = np.zeros(n_nodes, dtype=np.int64)
    j = rng.choice(n_nodes, size=n_seeded, replace=False)
    S[j] -= 1
    I[j] = 1
    u0 = np.stack([S, I, np.zeros_like(S), np.zeros_like(S), np.zeros_like(S)],
                  axis=1).astype(np.int32)
    E = np.array([[1, 1, 1], [0, 1, 1], [0, 0, 0], [0, 1, 1], [0, 1, 0]], dtype=np.int32)
    N = np.array([[4], [3], [0], [1], [0]], dtype=np.int32)
    net = powerlaw_network(rng, n_nodes)
    totals = herd[:, None].copy()
    # herds never empty: the printed propensity divides by S + I + R + V
    ev = _cattle_events(rng, totals, days, 0, events_per_node_day,
                        (1 / 3, 1 / 3, 0.0, 1 / 3), 1, net, enter_sel=0,
                        exit_sel=[1], ages_shift=None, keep=1)
    if vaccinate:
        t = np.repeat(np.arange(21, 21 + (n_nodes + 49) // 50), 50)[:n_nodes]
        rows = [(2, int(t[i]), i, 0, 0, 0.8, 2, 0) for i in range(n_nodes) if t[i] <= days]
        vac = make_events(rows)
        ev = {k: (np.concatenate([ev[k], vac[k]]) if k != "rep" else None) for k in ev}
    trans = ["S -> b*S*I/(S+I+R+V) -> I + Icum", "I -> g*I -> R"]
    w = parsed_model(trans, ["S", "I", "Icum", "R", "V"], {"b": 0.16, "g": 0.077}, u0,
                     np.arange(0, days + 1), seed=seed, events=ev, E=E, N=N,
                     name=f"SIR+Icum+V {n_nodes} nodes x {days} days"
                          + (" with vaccination" if vaccinate else ""))
    w.meta = {"gen_seed": gen_seed}
    return w


# --------------------------------------------------------------------------
# Synthetic cattle-shaped populations and event streams.
# --------------------------------------------------------------------------

def lognormal_herds(rng, n, median, sigma, lo, hi):
    z = rng.standard_normal(n)
    return np.clip(np.rint(np.exp(np.log(median) + sigma * z)), lo, hi
                   ).astype(np.int64)


def split_ages(herd, fracs=(0.2, 0.2, 0.6)):
    """Largest-remainder split of each herd into age classes."""
    fr = np.asarray(fracs, dtype=np.float64)
    raw = herd[:, None] * fr[None, :]
    base = np.floor(raw).astype(np.int64)
    rem = raw - base
    short = herd - base.sum(axis=1)
    order = np.argsort(-rem, axis=1, kind="stable")
    for i in range(len(fr)):
        add = short > i
        base[np.arange(len(herd))[add], order[add, i]] += 1
    return base


def powerlaw_network(rng, n_nodes, exponent=2.2, kmax=1000):
    """Directed graph: out-degree k in [1, kmax] with P(k) ~ k^-exponent,
    out-neighbours uniform without self-loops.  Returns CSR (ptr, adj)."""
    kmax = max(1, min(kmax, n_nodes - 1))
    ks = np.arange(1, kmax + 1, dtype=np.float64)
    p = ks ** (-exponent)
    p /= p.sum()
    deg = rng.choice(np.arange(1, kmax + 1), size=n_nodes, p=p)
    ptr = np.zeros(n_nodes + 1, dtype=np.int64)
    ptr[1:] = np.cumsum(deg)
    adj = np.empty(ptr[-1], dtype=np.int64)
    for i in range(n_nodes):
        d = int(deg[i])
        nb = rng.choice(n_nodes - 1, size=d, replace=False)
        nb[nb >= i] += 1
        adj[ptr[i]:ptr[i + 1]] = nb
    return ptr, adj, deg


def _geometric3(rng, size):
    # Geometric on {1, 2, ...} with mean 3.
    return rng.geometric(1.0 / 3.0, size=size).astype(np.int64)


def _cattle_events(rng, totals, n_days, t0, rate, mix, n_ages, net, enter_sel,
                   exit_sel, ages_shift, keep=0):
    """Daily events with exact tracking of per-age totals.  Exits and
    external transfers leave at least `keep` individuals in each group.

    totals: (n_nodes, n_ages) int64, modified in place.
    mix: fractions (exit, enter, internal, external).
    Within a day the solver runs exits, then enters, then internal
    transfers, then external transfers in list order, so the totals are
    tracked in that order.  The final list is shuffled, keeping the relative
    order of each day's external transfers.
    """
    n_nodes = totals.shape[0]
    ptr, adj, deg = net
    src_p = deg / deg.sum()
    rows = []          # (event, time, node, dest, n, select, shift)
    for d in range(n_days):
        T = t0 + 1 + d
        n_today = rng.poisson(rate * n_nodes)
        n_exit, n_enter, n_int, n_ext = rng.multinomial(n_today, mix)
        # exits: clamp cumulatively per (node, age) group
        if n_exit:
            nodes = rng.integers(0, n_nodes, n_exit)
            ages = rng.integers(0, n_ages, n_exit)
            want = _geometric3(rng, n_exit)
            key = nodes * n_ages + ages
            order = np.argsort(key, kind="stable")
            k_s, w_s = key[order], want[order]
            starts = np.r_[True, k_s[1:] != k_s[:-1]]
            grp = np.cumsum(starts) - 1
            cs = np.cumsum(w_s)
            base = np.r_[0, cs][np.flatnonzero(starts)][grp]
            cum = cs - base
            avail = np.maximum(totals.reshape(-1)[k_s] - keep, 0)
            capped = np.minimum(cum, avail)
            got = capped - np.r_[0, capped[:-1]]
            got[starts] = capped[starts]
            np.subtract.at(totals.reshape(-1), k_s, got)
            ok = got > 0
            for i in np.flatnonzero(ok):
                nd, ag = divmod(int(k_s[i]), n_ages)
                rows.append((EXIT, T, nd, 0, int(got[i]), exit_sel[ag], -1))
        if n_enter:
            nodes = rng.integers(0, n_nodes, n_enter)
            want = _geometric3(rng, n_enter)
            np.add.at(totals[:, 0], nodes, want)
            for nd, w in zip(nodes.tolist(), want.tolist()):
                rows.append((ENTER, T, nd, 0, w, enter_sel, -1))
        if n_int and ages_shift:
            for _ in range(n_int):
                nd = int(rng.integers(0, n_nodes))
                a = int(rng.integers(0, len(ages_shift)))
                sel, q = ages_shift[a]
                avail = int(totals[nd, a])
                w = min(int(_geometric3(rng, 1)[0]), avail)
                if w <= 0:
                    continue
                totals[nd, a] -= w
                totals[nd, a + 1] += w
                rows.append((INTERNAL, T, nd, 0, w, sel, q))
        if n_ext:
            srcs = rng.choice(n_nodes, size=n_ext, p=src_p)
            picks = rng.random(n_ext)
            want = _geometric3(rng, n_ext)
            ages = rng.integers(0, n_ages, n_ext)
            for s, pk, w, a in zip(srcs.tolist(), picks.tolist(),
                                   want.tolist(), ages.tolist()):
                nb = adj[ptr[s]:ptr[s + 1]]
                dst = int(nb[int(pk * len(nb))])
                avail = int(totals[s, a]) - keep
                w = min(w, avail)
                if w <= 0:
                    continue
                totals[s, a] -= w
                totals[dst, a] += w
                rows.append((EXTERNAL, T, s, dst, w, exit_sel[a], -1))
    if not rows:
        return empty_events()
    arr = np.asarray(rows, dtype=np.int64)
    n = len(arr)
    perm = rng.permutation(n)
    shuffled = arr[perm]
    # Internal and external transfers may depend on earlier ones of the same
    # day and type (the solver runs them in list order), so each day keeps
    # their relative order: the positions that a day's events of one such
    # type occupy receive those events in generation order.
    for etype in (INTERNAL, EXTERNAL):
        pos = np.flatnonzero(shuffled[:, 0] == etype)
        if pos.size == 0:
            continue
        orig = perm[pos]
        tday = shuffled[pos, 1]
        o_pos = np.lexsort((pos, tday))
        o_orig = np.lexsort((orig, tday))
        shuffled[pos[o_pos]] = arr[orig[o_orig]]
    ev = empty_events()
    ev["event"] = shuffled[:, 0].astype(np.int32)
    ev["time"] = shuffled[:, 1].astype(np.int32)
    ev["node"] = shuffled[:, 2].astype(np.int32)
    ev["dest"] = shuffled[:, 3].astype(np.int32)
    ev["n"] = shuffled[:, 4].astype(np.int32)
    ev["proportion"] = np.zeros(n, dtype=np.float64)
    ev["select"] = shuffled[:, 5].astype(np.int32)
    ev["shift"] = shuffled[:, 6].astype(np.int32)
    return ev


def config_sir(n_nodes=100, days=99, seed=42):
    """SIR without events: every node S=99 I=1 R=0, beta 0.16, gamma 0.077,
    tspan = 1..days+1 (the first-example parameters of Sec. 4.1)."""
    u0 = np.tile(np.array([[99, 1, 0]], dtype=np.int32), (n_nodes, 1))
    return plain_model(SIR, u0, np.arange(1, days + 2), [0.16, 0.077],
                       seed=seed, name=f"SIR {n_nodes} nodes x {days} days")


def config_sise(n_nodes=1600, days=365, gen_seed=1002, seed=42,
                events_per_node_day=0.41, median=50, sigma=1.0, hi=5000):
    """SISe with scheduled events: log-normal herds (median 50, sigma 1.0,
    clamp 1..5000), 1% of nodes seeded with 10% infected, phi updated daily
    (alpha 1.0, decay 0.1), upsilon 0.0173, gamma 0.1; one year of enter /
    exit / external-transfer events (thirds), ~0.34 events per node-day."""
    rng = np.random.default_rng(gen_seed)
    herd = lognormal_herds(rng, n_nodes, median, sigma, 1, hi)
    I = np.zeros(n_nodes, dtype=np.int64)
    seeded = rng.choice(n_nodes, size=max(1, n_nodes // 100), replace=False)
    I[seeded] = np.maximum(1, np.rint(0.1 * herd[seeded])).astype(np.int64)
    S = herd - I
    u0 = np.stack([S, I], axis=1).astype(np.int32)
    net = powerlaw_network(rng, n_nodes)
    totals = herd[:, None].copy()
    ev = _cattle_events(rng, totals, days, 0, events_per_node_day,
                        (1 / 3, 1 / 3, 0.0, 1 / 3), 1, net, enter_sel=0,
                        exit_sel=[2], ages_shift=None)
    w = plain_model(SISE, u0, np.arange(0, days + 1), sise_gdata(),
                    seed=seed, events=ev,
                    name=f"SISe {n_nodes} nodes x {days} days with events")
    w.meta = {"gen_seed": gen_seed}
    return w


def config_sise3(n_nodes=37000, days=3650, gen_seed=1003, seed=42,
                 events_per_node_day=0.111, median=60, sigma=1.2, hi=10000,
                 n_rep=1, per_rep_events=False):
    """SISe3 (three age classes): log-normal herds split 0.2/0.2/0.6 by age,
    1% of nodes seeded with 10% infected per age class, seasonal decay per
    quarter; events: exit 30%, enter 30%, internal transfer (ageing) 20%,
    external transfer 20% on a power-law network."""
    rng = np.random.default_rng(gen_seed)
    herd = lognormal_herds(rng, n_nodes, median, sigma, 1, hi)
    ages = split_ages(herd)
    I = np.zeros_like(ages)
    seeded = rng.choice(n_nodes, size=max(1, n_nodes // 100), replace=False)
    I[seeded] = np.rint(0.1 * ages[seeded]).astype(np.int64)
    S = ages - I
    u0 = np.stack([S[:, 0], I[:, 0], S[:, 1], I[:, 1], S[:, 2], I[:, 2]],
                  axis=1).astype(np.int32)
    net = powerlaw_network(rng, n_nodes)
    mix = (0.3, 0.3, 0.2, 0.2)
    evs = []
    reps = n_rep if per_rep_events else 1
    for r in range(reps):
        totals = ages.copy()
        ev = _cattle_events(rng, totals, days, 0, events_per_node_day, mix, 3,
                            net, enter_sel=0, exit_sel=[3, 4, 5],
                            ages_shift=[(3, 0), (4, 1)])
        if per_rep_events:
            ev["rep"] = np.full(len(ev["event"]), r, dtype=np.int32)
        evs.append(ev)
    if per_rep_events:
        ev = empty_events()
        for k in ("event", "time", "node", "dest", "n", "proportion",
                  "select", "shift", "rep"):
            ev[k] = np.concatenate([e[k] for e in evs])
    else:
        ev = evs[0]
    w = plain_model(SISE3, u0, np.arange(0, days + 1), sise3_gdata(),
                    seed=seed, n_rep=n_rep, events=ev,
                    name=f"SISe3 {n_nodes} nodes x {days} days"
                         + (f" x {n_rep} replicates" if n_rep > 1 else ""))
    w.meta = {"gen_seed": gen_seed}
    return w


def config_batched(n_rep=256, n_nodes=5000, days=365, gen_seed=1004, seed=42,
                   events_per_node_day=0.111, median=50, sigma=1.0, hi=5000):
    """Batched replicates: SISe3 on `n_nodes` log-normal herds (median 50,
    sigma 1.0, clamp 1..5000), `n_rep` independent replicates, each with its
    own event list at the SISe3 density (exit 30%, enter 30%, ageing 20%,
    external transfer 20%) on one shared power-law movement network.  The
    lists are generated for all replicates at once (each day's events of a
    given position in the day are drawn for every replicate in one vector
    step); totals are tracked per replicate in the solver's order."""
    rng = np.random.default_rng(gen_seed)
    herd = lognormal_herds(rng, n_nodes, median, sigma, 1, hi)
    ages = split_ages(herd)
    I = np.zeros_like(ages)
    seeded = rng.choice(n_nodes, size=max(1, n_nodes // 100), replace=False)
    I[seeded] = np.rint(0.1 * ages[seeded]).astype(np.int64)
    S = ages - I
    u0 = np.stack([S[:, 0], I[:, 0], S[:, 1], I[:, 1], S[:, 2], I[:, 2]],
                  axis=1).astype(np.int32)
    ptr, adj, deg = powerlaw_network(rng, n_nodes)
    src_cdf = np.cumsum(deg / deg.sum())
    R, Nn = n_rep, n_nodes
    totals = np.broadcast_to(ages[None], (R, Nn, 3)).copy()
    flat = totals.reshape(-1)
    cols = {k: [] for k in ("rep", "event", "time", "node", "dest", "n", "select", "shift",
                            "order")}

    def emit(rep, etype, T, node, dest, n, sel, shift, order):
        k = len(rep)
        cols["rep"].append(rep.astype(np.int32))
        cols["event"].append(np.full(k, etype, np.int32))
        cols["time"].append(np.full(k, T, np.int32))
        cols["node"].append(node.astype(np.int32))
        cols["dest"].append(np.asarray(dest, dtype=np.int32) * np.ones(k, np.int32))
        cols["n"].append(n.astype(np.int32))
        cols["select"].append(np.asarray(sel, dtype=np.int32) * np.ones(k, np.int32))
        cols["shift"].append(np.asarray(shift, dtype=np.int32) * np.ones(k, np.int32))
        cols["order"].append(np.full(k, order, np.int64))

    reps = np.arange(R)
    for d in range(days):
        T = 1 + d
        n_today = rng.poisson(events_per_node_day * Nn, size=R)
        mix = rng.multinomial(n_today, [0.3, 0.3, 0.2, 0.2])
        # exits: cumulative clamp per (rep, node, age)
        ne = mix[:, 0]
        rep_e = np.repeat(reps, ne)
        if rep_e.size:
            nodes = rng.integers(0, Nn, rep_e.size)
            ag = rng.integers(0, 3, rep_e.size)
            want = _geometric3(rng, rep_e.size)
            key = (rep_e * Nn + nodes) * 3 + ag
            o = np.argsort(key, kind="stable")
            k_s, w_s, r_s = key[o], want[o], rep_e[o]
            starts = np.r_[True, k_s[1:] != k_s[:-1]]
            grp = np.cumsum(starts) - 1
            cs = np.cumsum(w_s)
            base = np.r_[0, cs][np.flatnonzero(starts)][grp]
            capped = np.minimum(cs - base, flat[k_s])
            got = capped - np.r_[0, capped[:-1]]
            got[starts] = capped[starts]
            np.subtract.at(flat, k_s, got)
            ok = got > 0
            nd = (k_s[ok] // 3) % Nn
            emit(r_s[ok], EXIT, T, nd, 0, got[ok], 3 + k_s[ok] % 3, -1, 0)
        # enters into S1
        rep_n = np.repeat(reps, mix[:, 1])
        if rep_n.size:
            nodes = rng.integers(0, Nn, rep_n.size)
            want = _geometric3(rng, rep_n.size)
            np.add.at(totals[:, :, 0], (rep_n, nodes), want)
            emit(rep_n, ENTER, T, nodes, 0, want, 0, -1, 1)
        # ageing, one position of the day at a time for every replicate
        for k in range(int(mix[:, 2].max(initial=0))):
            act = reps[mix[:, 2] > k]
            nodes = rng.integers(0, Nn, act.size)
            a = rng.integers(0, 2, act.size)
            w = np.minimum(_geometric3(rng, act.size), totals[act, nodes, a])
            ok = w > 0
            act, nodes, a, w = act[ok], nodes[ok], a[ok], w[ok]
            totals[act, nodes, a] -= w
            totals[act, nodes, a + 1] += w
            emit(act, INTERNAL, T, nodes, 0, w, 3 + a, a, 2 + k)
        # external transfers, in list order within each replicate
        for k in range(int(mix[:, 3].max(initial=0))):
            act = reps[mix[:, 3] > k]
            src = np.minimum(np.searchsorted(src_cdf, rng.random(act.size)), Nn - 1)
            pick = rng.random(act.size)
            dst = adj[ptr[src] + (pick * deg[src]).astype(np.int64)]
            a = rng.integers(0, 3, act.size)
            w = np.minimum(_geometric3(rng, act.size), totals[act, src, a])
            ok = w > 0
            act, src, dst, a, w = act[ok], src[ok], dst[ok], a[ok], w[ok]
            totals[act, src, a] -= w
            totals[act, dst, a] += w
            emit(act, EXTERNAL, T, src, dst, w, 3 + a, -1, 10_000 + k)
    cat = {k: np.concatenate(v) if v else np.zeros(0, np.int64) for k, v in cols.items()}
    o = np.lexsort((cat["order"], cat["time"], cat["rep"]))
    ev = empty_events()
    for k in ("event", "time", "node", "dest", "n", "select", "shift"):
        ev[k] = np.ascontiguousarray(cat[k][o], dtype=np.int32)
    ev["proportion"] = np.zeros(len(o), dtype=np.float64)
    ev["rep"] = np.ascontiguousarray(cat["rep"][o], dtype=np.int32)
    w = plain_model(SISE3, u0, np.arange(0, days + 1), sise3_gdata(), seed=seed,
                    n_rep=n_rep, events=ev,
                    name=f"SISe3 {n_rep} replicates x {n_nodes} nodes x {days} days, "
                         f"own events per replicate")
    w.meta = {"gen_seed": gen_seed}
    return w


def replicate_range(w, rep0, n):
    """The shard of workload w that holds its replicates rep0 .. rep0 + n - 1:
    their initial states; the event table stays the whole job's (each event
    keeps its replicate and list index, which key its random stream).  Run it
    with the model's replicate range set to (rep0, w.n_rep)."""
    if not (0 <= rep0 and n >= 1 and rep0 + n <= w.n_rep):
        raise ValueError(f"replicates {rep0}..{rep0 + n - 1} outside 0..{w.n_rep - 1}")
    out = Workload(**{**w.__dict__, "u0": w.u0[rep0:rep0 + n].copy(),
                      "v0": w.v0[rep0:rep0 + n].copy(), "n_rep": n,
                      "meta": {**w.meta, "rep0": rep0, "rep_total": w.n_rep}})
    return out


def config_endemic(n_nodes=100_000, days=365, gen_seed=1005, seed=42):
    """SISe3 without events on large endemic herds: herd sizes log-uniform
    in [200, 2000], 40% of each age class infected, phi at its equilibrium
    10 I / N; default rates and seasonal decay.  Every node fires tens to
    hundreds of transitions a day (the SSA's throughput regime)."""
    rng = np.random.default_rng(gen_seed)
    herd = np.rint(np.exp(rng.uniform(np.log(200), np.log(2000), n_nodes))).astype(np.int64)
    ages = split_ages(herd)
    I = np.rint(0.4 * ages).astype(np.int64)
    S = ages - I
    u0 = np.stack([S[:, 0], I[:, 0], S[:, 1], I[:, 1], S[:, 2], I[:, 2]], 1).astype(np.int32)
    phi = 10.0 * I.sum(1) / herd
    w = plain_model(SISE3, u0, np.arange(0, days + 1), sise3_gdata(), seed=seed,
                    v0=phi[:, None], name=f"SISe3 endemic {n_nodes} nodes x {days} days")
    w.meta = {"gen_seed": gen_seed}
    return w


def distance_neighbors(x, y, cutoff):
    """Neighbour lists of points within `cutoff` of each other (self
    excluded): CSR (ptr, idx, distance), neighbours in increasing index."""
    n = len(x)
    ptr = np.zeros(n + 1, dtype=np.int64)
    idx, dist = [], []
    order = np.argsort(x, kind="stable")
    xs = x[order]
    for i in range(n):
        lo = np.searchsorted(xs, x[i] - cutoff, side="left")
        hi = np.searchsorted(xs, x[i] + cutoff, side="right")
        cand = order[lo:hi]
        cand = cand[cand != i]
        d = np.hypot(x[cand] - x[i], y[cand] - y[i])
        keep = d <= cutoff
        c, dd = cand[keep], d[keep]
        o = np.argsort(c)
        idx.append(c[o])
        dist.append(dd[o])
        ptr[i + 1] = ptr[i] + len(c)
    return (ptr, np.concatenate(idx).astype(np.int32) if idx else np.zeros(0, np.int32),
            np.concatenate(dist) if dist else np.zeros(0))


def config_sise_sp(n_nodes=1600, days=365, gen_seed=1006, seed=42, side_m=50000.0,
                   cutoff_m=2500.0, events=True):
    """SISe_sp (Sec. 4.2): SISe with spatial coupling of phi between farms
    within `cutoff_m` metres, farms placed uniformly in a 50 km x 50 km
    square (the paper's "50 square kilometer region", read as 50 km a side:
    about a dozen neighbours within 2,500 m), the paper's example parameters (upsilon 0.012, gamma
    0.1, alpha 1, decay 0.10 / 0.12 / 0.12 / 0.10, season ends 91 / 182 / 273
    / 365, coupling 0.2), 10% of farms with 5% infected, and the SISe
    benchmark's synthetic event stream."""
    base = config_sise(n_nodes=n_nodes, days=days, gen_seed=gen_seed)
    rng = np.random.default_rng(gen_seed + 1)
    x = rng.uniform(0, side_m, n_nodes)
    y = rng.uniform(0, side_m, n_nodes)
    nb = distance_neighbors(x, y, cutoff_m)
    herd = base.u0[0].sum(axis=1).astype(np.int64)
    I = np.zeros(n_nodes, dtype=np.int64)
    inf = rng.choice(n_nodes, size=n_nodes // 10, replace=False)
    I[inf] = (herd[inf] * 0.05).astype(np.int64)
    u0 = np.stack([herd - I, I], axis=1).astype(np.int32)
    w = plain_model(SISE_SP, u0, np.arange(0, days + 1), sise_sp_gdata(), seed=seed,
                    events=base.events if events else None,
                    name=f"SISe_sp {n_nodes} nodes x {days} days")
    w.neighbors = nb
    w.meta = {"gen_seed": gen_seed, "cutoff_m": cutoff_m, "side_m": side_m}
    return w
