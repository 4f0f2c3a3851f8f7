"""The OpenMP timing build of the oracle (same source, node loops of a day in
parallel, E2 events serial, Sec. 3.4.2) gives the serial build's results bit
for bit, and reports the same first error.  It is used only to time the CPU
baseline on all host cores."""
import numpy as np
import pytest

from paper_1605_01421_gb300 import workloads as W


@pytest.fixture(scope="module")
def omp(orc):
    try:
        orc.build(openmp=True)
    except Exception as e:  # pragma: no cover - compiler without OpenMP
        pytest.skip(f"no OpenMP build: {e}")
    orc.set_threads(4)
    return orc


def _same(a, b):
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[2].view(np.uint64), b[2].view(np.uint64))
    assert np.array_equal(a[3], b[3])
    assert a[4] == b[4]


@pytest.mark.parametrize("name", ["sise", "sise3", "batched", "sise_sp", "aem"])
def test_parallel_build_equals_serial(omp, name):
    if name == "sise":
        w = W.config_sise(n_nodes=700, days=40)
    elif name == "sise3":
        w = W.config_sise3(n_nodes=2500, days=30)
    elif name == "batched":
        w = W.config_batched(n_rep=3, n_nodes=800, days=25)
    elif name == "sise_sp":
        w = W.config_sise_sp(days=30)
    else:
        w = W.config_sise(n_nodes=500, days=30)
        w.solver = W.AEM
    _same(omp.run(w), omp.run(w, openmp=True))


def test_parallel_build_reports_the_first_failing_event(omp):
    w = W.config_sise(n_nodes=400, days=30)
    ev = w.events
    # two exits that take more animals than exist, on the same day at two
    # nodes: the first of them in sorted order is the one reported
    day = 12
    idx = np.flatnonzero((ev["time"] == day) & (ev["event"] == 0))
    assert idx.size >= 2
    ev["n"][idx[-1]] = 10 ** 6
    ev["n"][idx[0]] = 10 ** 6
    a, b = omp.run(w), omp.run(w, openmp=True)
    assert a[0] == -2
    assert a[4] == b[4] and a[0] == b[0]
    assert a[4]["event"] == idx[0]
