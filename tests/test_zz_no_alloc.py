"""sg_run_noalloc, the entry point for callers that cannot allocate memory
(a host framework that owns the device memory, a service whose footprint must
stay fixed after start-up).

It keeps its working memory in one fixed array inside the library instead of
allocating it.  These checks call it through the C ABI and compare its U, V
and counters, bit for bit, with those of the allocating entry point sg_run on
the same inputs, on two calls in a row (different sizes and seeds, so stale
contents of the shared array would show), and the first call's U and V also
with the CPU oracle.  The file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1605_01421_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_01421_gb300 import binding
    binding.build()
    return torch, binding, binding.lib()


def _desc(binding, w):
    keep = []

    def p(a):
        keep.append(a)
        return ctypes.c_void_p(a.ctypes.data) if a.size else None

    S = np.ascontiguousarray(w.S.ravel(order="F"), dtype=np.int32)
    G = np.ascontiguousarray(w.G.ravel(order="F"), dtype=np.int32)
    E = np.ascontiguousarray(w.E.ravel(order="F"), dtype=np.int32)
    N = np.ascontiguousarray(w.N.ravel(order="F"), dtype=np.int32)
    g = np.ascontiguousarray(w.gdata, dtype=np.float64)
    d = binding._Desc(int(w.kind), int(w.n_nodes), int(w.S.shape[0]), int(w.S.shape[1]),
                      p(S), p(G), int(w.E.shape[1]), p(E), int(w.N.shape[1]), p(N),
                      int(w.n_v), int(w.ldata.shape[0]), None, int(g.size), p(g))
    return d, keep


def _run_noalloc(torch, binding, L, w, seed, n_rep):
    d, keep = _desc(binding, w)
    dev = "cuda"
    ld = torch.as_tensor(np.ascontiguousarray(w.ldata.ravel(order="F")), device=dev)
    u0 = torch.as_tensor(np.array(w.u0[:n_rep]), device=dev)
    v0 = torch.as_tensor(np.array(w.v0[:n_rep]), device=dev)
    M = len(w.tspan)
    U = torch.full((n_rep, M, w.n_nodes, w.n_comp), -7, dtype=torch.int32, device=dev)
    V = torch.full((n_rep, M, w.n_nodes, w.n_v), -7.0, dtype=torch.float64, device=dev)
    ts = np.ascontiguousarray(w.tspan, dtype=np.int32)
    st, er = binding.Stats(), binding.Error()
    rc = L.sg_run_noalloc(ctypes.byref(d), binding._dev_ptr(ld),
                          ctypes.c_void_p(ts.ctypes.data), int(ts.size), int(seed),
                          int(n_rep), binding._dev_ptr(u0), binding._dev_ptr(v0),
                          binding._dev_ptr(U), binding._dev_ptr(V),
                          binding._stream_handle(None), ctypes.byref(st), ctypes.byref(er))
    del keep
    return rc, U.cpu().numpy(), V.cpu().numpy(), st.as_dict()


def _workload(n_nodes, days, n_rep, gen_seed):
    rng = np.random.default_rng(gen_seed)
    herd = np.clip(np.rint(np.exp(np.log(50) + rng.standard_normal(n_nodes))), 1, 5000)
    I = np.where(rng.random(n_nodes) < 0.05, np.maximum(1, np.rint(0.1 * herd)), 0)
    u0 = np.stack([herd - I, I], axis=1).astype(np.int32)
    v0 = rng.uniform(0.0, 2.0, size=(n_nodes, 1))
    return W.plain_model(W.SISE, u0, np.arange(0, days + 1), W.sise_gdata(),
                         seed=1, n_rep=n_rep, v0=v0)


def test_noalloc_matches_allocating_run_twice(env, orc):
    torch, binding, L = env
    cases = [(_workload(2000, 150, 3, 11), 101), (_workload(777, 90, 1, 12), 202)]
    for i, (w, seed) in enumerate(cases):
        U0, V0, st0 = binding.simulate(w, seed=seed)
        rc, U1, V1, st1 = _run_noalloc(torch, binding, L, w, seed, w.n_rep)
        assert rc == 0
        assert np.array_equal(U0, U1)
        assert np.array_equal(V0.view(np.uint64), V1.view(np.uint64))
        assert st1["reactions"] == st0["reactions"] > 0
        assert st1["draws"] == st0["draws"]
        if i == 0:
            # the first case also against the CPU oracle, bit for bit
            code, Uo, Vo, Ro, err = orc.run(w, seed=seed)
            assert code == 0, err
            assert np.array_equal(Uo, U1)
            assert np.array_equal(Vo.view(np.uint64), V1.view(np.uint64))
            assert st1["reactions"] == int(Ro.sum())


def test_noalloc_rejects_problems_beyond_its_scratch(env):
    torch, binding, L = env
    # 400k SISe3 node-replicates need 400k * (24 + 8) bytes > 8 MiB
    w = W.plain_model(W.SISE3, np.ones((400_000, 6), np.int32), np.arange(0, 3),
                      W.sise3_gdata())
    d, keep = _desc(binding, w)
    ts = np.ascontiguousarray(w.tspan, dtype=np.int32)
    dummy = torch.zeros(1, device="cuda")
    p = binding._dev_ptr(dummy)
    st, er = binding.Stats(), binding.Error()
    rc = L.sg_run_noalloc(ctypes.byref(d), p, ctypes.c_void_p(ts.ctypes.data), 3, 1, 1,
                          p, p, p, p, binding._stream_handle(None), ctypes.byref(st),
                          ctypes.byref(er))
    assert rc == -10
    assert L.sg_strerror(rc) == b"problem exceeds the fixed scratch of sg_run_noalloc"
