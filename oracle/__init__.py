"""CPU oracle for the SimInf split-step method (arXiv 1605.01421).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_1605_01421_gb300``) never imports it and
never falls back to it.

The oracle is plain serial C (``siminf_oracle.c``), compiled here with
``-ffp-contract=off`` so that every double operation happens exactly as
written.  This module compiles it, loads it with ctypes and marshals numpy
arrays.  Nothing here computes any part of the method.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "siminf_oracle.c")
_HDR = os.path.join(_HERE, "siminf_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libsiminf_oracle.so")
# the same source with -fopenmp: node loops in parallel (timing only)
_OMP_LIB_PATH = os.path.join(_OUT_DIR, "libsiminf_oracle_omp.so")

ERR_NAMES = {
    0: "ok",
    -1: "invalid argument",
    -2: "event moves more individuals than exist",
    -3: "shift moves outside the compartments",
    -4: "negative or non-finite transition rate",
    -5: "post time step error",
    -8: "out of memory",
    -9: "more than 2^24 draws in one node-day",
}

_lock = threading.Lock()
_lib = None


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libsiminf_oracle.so`` (or,
    with ``openmp``, the node-parallel timing build
    ``libsiminf_oracle_omp.so`` of the same source)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    path = _OMP_LIB_PATH if openmp else _LIB_PATH
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= newest):
        return path
    tmp = path + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared"] + (["-fopenmp"] if openmp else []) + [
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


class _Model(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int), ("n_nodes", ctypes.c_int),
        ("n_comp", ctypes.c_int), ("n_trans", ctypes.c_int),
        ("S", ctypes.c_void_p), ("G", ctypes.c_void_p),
        ("n_select", ctypes.c_int), ("E", ctypes.c_void_p),
        ("n_shift", ctypes.c_int), ("N", ctypes.c_void_p),
        ("n_v", ctypes.c_int), ("n_ldata", ctypes.c_int),
        ("ldata", ctypes.c_void_p), ("n_gdata", ctypes.c_int),
        ("gdata", ctypes.c_void_p), ("nb_ptr", ctypes.c_void_p),
        ("nb_idx", ctypes.c_void_p), ("nb_dist", ctypes.c_void_p),
        ("solver", ctypes.c_int),
        ("rate_fn", ctypes.c_void_p),
    ]


class _Events(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("event", ctypes.c_void_p), ("time", ctypes.c_void_p),
        ("node", ctypes.c_void_p), ("dest", ctypes.c_void_p),
        ("n_ind", ctypes.c_void_p), ("proportion", ctypes.c_void_p),
        ("select", ctypes.c_void_p), ("shift", ctypes.c_void_p),
        ("rep", ctypes.c_void_p),
    ]


class _Error(ctypes.Structure):
    _fields_ = [("code", ctypes.c_int), ("rep", ctypes.c_int),
                ("node", ctypes.c_int), ("event", ctypes.c_int64),
                ("day", ctypes.c_int)]


class _TauRecord(ctypes.Structure):
    _fields_ = [("rep", ctypes.c_int), ("node", ctypes.c_int), ("T", ctypes.c_int),
                ("tau", ctypes.c_double)]


_omp_lib = None


def lib(openmp: bool = False):
    """The serial oracle (or, with ``openmp``, its node-parallel timing
    build)."""
    global _lib, _omp_lib
    with _lock:
        if openmp:
            if _omp_lib is None:
                _omp_lib = _load(build(openmp=True), openmp=True)
            return _omp_lib
        if _lib is None:
            _lib = _load(build())
    return _lib


def set_threads(n: int) -> None:
    """Threads of the OpenMP timing build's parallel loops."""
    lib(openmp=True).omp_set_num_threads(int(n))


def _load(path, openmp=False):
    L = ctypes.CDLL(path)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.oracle_philox4x32_10.restype = None
    L.oracle_u01.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
    L.oracle_u01.restype = ctypes.c_double
    L.oracle_log.argtypes = [ctypes.c_double]
    L.oracle_log.restype = ctypes.c_double
    L.oracle_bounded_sequence.argtypes = [
        ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, u32p,
        ctypes.c_int, u32p]
    L.oracle_bounded_sequence.restype = ctypes.c_uint32
    ip = ctypes.POINTER(ctypes.c_int)
    L.oracle_apply_event.argtypes = [
        ctypes.c_int, ip, ctypes.c_int, ip, ctypes.c_int, ctypes.c_int,
        ip, ip, ctypes.c_int, ctypes.c_double, ctypes.c_int,
        ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int]
    L.oracle_apply_event.restype = ctypes.c_int
    L.oracle_run.argtypes = [
        ctypes.POINTER(_Model), ctypes.POINTER(_Events),
        ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
        ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_Error)]
    L.oracle_run.restype = ctypes.c_int
    L.oracle_run_reps.argtypes = [
        ctypes.POINTER(_Model), ctypes.POINTER(_Events),
        ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
        ctypes.c_int, ctypes.c_int,
        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
        ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_Error)]
    L.oracle_run_reps.restype = ctypes.c_int
    L.oracle_trace_first_tau.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    L.oracle_trace_first_tau.restype = ctypes.c_int64
    if openmp:
        L.omp_set_num_threads.argtypes = [ctypes.c_int]
        L.omp_set_num_threads.restype = None
    return L


def first_waiting_times(w, cap, **run_kw):
    """Test hook: run the serial oracle on ``w`` and return, for every
    node-day with lambda > 0 (direct method, at most ``cap`` of them in run
    order), the replicate, node, T and the waiting time tau of its first
    draw (whether or not it passes T), plus run()'s return value."""
    L = lib()
    buf = (_TauRecord * int(cap))()
    L.oracle_trace_first_tau(ctypes.cast(buf, ctypes.c_void_p), int(cap))
    try:
        res = run(w, **run_kw)
    finally:
        n = int(L.oracle_trace_first_tau(None, 0))
    rec = np.ctypeslib.as_array(buf)[:n]
    out = {"rep": rec["rep"].copy(), "node": rec["node"].copy(), "T": rec["T"].copy(),
           "tau": rec["tau"].copy()}
    return out, res


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _colmajor_i32(M):
    return np.ascontiguousarray(np.asarray(M, dtype=np.int32).ravel(order="F"))


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def u01(a, b):
    return lib().oracle_u01(int(a) & 0xFFFFFFFF, int(b) & 0xFFFFFFFF)


def log(x):
    return lib().oracle_log(float(x))


def bounded_sequence(seed, event_index, rep, ranges):
    ranges = np.ascontiguousarray(ranges, dtype=np.uint32)
    out = np.zeros_like(ranges)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib().oracle_bounded_sequence(
        int(seed), int(event_index), int(rep),
        ranges.ctypes.data_as(u32p), int(ranges.size), out.ctypes.data_as(u32p))
    return out


def apply_event(E, N, etype, u_node, u_dest=None, n=0, proportion=0.0,
                select=0, shift=-1, seed=0, event_index=0, rep=0):
    """Apply one scheduled event to host state vectors (modified in place
    copies are returned) -> (code, u_node, u_dest)."""
    E = np.asarray(E)
    N = np.asarray(N) if N is not None else np.zeros((E.shape[0], 1), np.int32)
    Ec, Nc = _colmajor_i32(E), _colmajor_i32(N)
    un = _i32(np.array(u_node, copy=True))
    ud = _i32(np.array(u_dest, copy=True)) if u_dest is not None else None
    ip = ctypes.POINTER(ctypes.c_int)
    rc = lib().oracle_apply_event(
        int(E.shape[0]), Ec.ctypes.data_as(ip), int(E.shape[1]),
        Nc.ctypes.data_as(ip), int(N.shape[1]), int(etype),
        un.ctypes.data_as(ip), ud.ctypes.data_as(ip) if ud is not None else None,
        int(n), float(proportion), int(select), int(shift), int(seed),
        int(event_index), int(rep))
    return rc, un, ud


def _generic(w):
    """For a model given by transition strings (kind 5): the oracle's own
    parse (S, G) and the address of its compiled propensity function."""
    g = getattr(w, "generic", None)
    if g is None:
        return None
    from . import mparse
    c = mparse.compiled(g)
    return c.parsed.S, c.parsed.G, c.address


def run(w, seed=None, n_rep=None, u0=None, v0=None, solver=None, rep0=0, openmp=False):
    """Run the oracle on a workload description (see
    ``paper_1605_01421_gb300.workloads.Workload``).

    ``solver`` (default ``w.solver``): 0 the direct-method split step
    ('ssm'), 1 the all events method ('aem').  ``rep0`` > 0 runs replicates
    rep0 .. rep0 + n_rep - 1 of the workload's w.n_rep (their own streams and
    events) and returns only those.

    ``openmp`` runs the node-parallel timing build (same results; threads
    set with ``set_threads``).

    Returns ``(code, U, V, reactions, err)`` with U [R][M][Nn][C] int32,
    V [R][M][Nn][Nv] float64, reactions [R] int64 and err a dict.
    """
    L = lib(openmp)
    seed = w.seed if seed is None else seed
    n_rep = w.n_rep if n_rep is None else n_rep
    if u0 is None:
        u0 = w.u0[rep0:rep0 + n_rep] if rep0 else w.u0
    if v0 is None:
        v0 = w.v0[rep0:rep0 + n_rep] if rep0 else w.v0
    u0 = _i32(u0)
    v0 = _f64(v0)
    gen = _generic(w)
    S0, G0 = (gen[0], gen[1]) if gen else (w.S, w.G)
    S, G = _colmajor_i32(S0), _colmajor_i32(G0)
    E, N = _colmajor_i32(w.E), _colmajor_i32(w.N)
    ldata = _f64(np.asarray(w.ldata, dtype=np.float64).ravel(order="F"))
    gdata = _f64(w.gdata)
    n_comp, n_trans = S0.shape
    n_nodes = u0.shape[1]
    nb = getattr(w, "neighbors", None)
    if nb is not None:
        nb_ptr = np.ascontiguousarray(nb[0], dtype=np.int64)
        nb_idx = _i32(nb[1])
        nb_dist = _f64(nb[2])
    else:
        nb_ptr = nb_idx = nb_dist = None
    m = _Model(int(w.kind), int(n_nodes), int(n_comp), int(n_trans),
               _ptr(S), _ptr(G), int(w.E.shape[1]), _ptr(E),
               int(w.N.shape[1]), _ptr(N), int(w.n_v),
               int(np.asarray(w.ldata).shape[0]), _ptr(ldata) if ldata.size else None,
               int(gdata.size), _ptr(gdata),
               _ptr(nb_ptr) if nb_ptr is not None else None,
               _ptr(nb_idx) if nb_idx is not None and nb_idx.size else None,
               _ptr(nb_dist) if nb_dist is not None and nb_dist.size else None,
               int(getattr(w, "solver", 0) if solver is None else solver),
               gen[2] if gen else None)
    ev = w.events
    keep = []
    if ev is not None and len(ev["event"]) > 0:
        arrs = {k: (_f64(ev[k]) if k == "proportion" else _i32(ev[k]))
                for k in ("event", "time", "node", "dest", "n", "proportion",
                          "select", "shift")}
        rep_arr = _i32(ev["rep"]) if ev.get("rep") is not None else None
        keep = [arrs, rep_arr]
        evs = _Events(int(arrs["event"].size), _ptr(arrs["event"]),
                      _ptr(arrs["time"]), _ptr(arrs["node"]), _ptr(arrs["dest"]),
                      _ptr(arrs["n"]), _ptr(arrs["proportion"]),
                      _ptr(arrs["select"]), _ptr(arrs["shift"]),
                      _ptr(rep_arr) if rep_arr is not None else None)
        evp = ctypes.byref(evs)
    else:
        evp = None
    tspan = _i32(w.tspan)
    M = tspan.size
    U = np.zeros((n_rep, M, n_nodes, n_comp), dtype=np.int32)
    V = np.zeros((n_rep, M, n_nodes, int(w.n_v)), dtype=np.float64)
    reactions = np.zeros(n_rep, dtype=np.int64)
    err = _Error()
    if rep0 or (n_rep < w.n_rep and w.events is not None and w.events.get("rep") is not None):
        # a range of the workload's replicates (events keep their replicate)
        code = L.oracle_run_reps(ctypes.byref(m), evp, _ptr(tspan), int(M), int(seed),
                                 int(rep0), int(n_rep), int(max(w.n_rep, rep0 + n_rep)), _ptr(u0),
                                 _ptr(v0) if v0.size else None, _ptr(U),
                                 _ptr(V) if V.size else None, _ptr(reactions),
                                 ctypes.byref(err))
    else:
        code = L.oracle_run(ctypes.byref(m), evp, _ptr(tspan), int(M), int(seed),
                            int(n_rep), _ptr(u0), _ptr(v0) if v0.size else None,
                            _ptr(U), _ptr(V) if V.size else None, _ptr(reactions),
                            ctypes.byref(err))
    del keep
    e = {"code": err.code, "rep": err.rep, "node": err.node,
         "event": err.event, "day": err.day}
    return code, U, V, reactions, e
