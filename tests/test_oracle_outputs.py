"""Pins for the oracle's output selections (U_sparse / V_sparse of Sec. 3.2
and the prevalence summary of Sec. 4.2): a hand-worked prevalence example
(tests/golden/prevalence_worked_example.txt), sparse values against direct
indexing of a trajectory the oracle computed, and invariants."""
import os
from fractions import Fraction

import numpy as np

from oracle import outputs
from paper_1605_01421_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "prevalence_worked_example.txt")


def _frac(s):
    return float("nan") if s == "nan" else float(Fraction(s))


def test_prevalence_worked_example():
    U = np.zeros((1, 2, 4, 2), dtype=np.int32)
    want = {}
    for line in open(GOLDEN):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "state":
            m, node, s, i = map(int, f[1:])
            U[0, m, node] = (s, i)
        else:
            want[(f[0], int(f[1]))] = [_frac(x) for x in f[2:]]
    for (kind, m), vals in want.items():
        got = outputs.prevalence(U, [1], [0, 1], kind)[0, m]
        np.testing.assert_allclose(np.atleast_1d(got), vals, rtol=0, atol=1e-15)
    k = outputs.prevalence_counts(U, [1], [0, 1])
    assert k[0, 0].tolist() == [6, 19, 2, 3]


def test_sparse_values_are_the_dense_entries(orc):
    w = W.config_sise3(n_nodes=50, days=20, gen_seed=3, n_rep=2)
    code, U, V, R, err = orc.run(w)
    assert code == 0
    rng = np.random.default_rng(0)
    M, Nn, C = U.shape[1], U.shape[2], U.shape[3]
    colptr, row = [0], []
    for m in range(M):
        r = np.sort(rng.choice(Nn * C, size=rng.integers(0, 12), replace=False))
        row.extend(r.tolist())
        colptr.append(len(row))
    vals = outputs.sparse_values(U, colptr, row, C)
    for m in range(M):
        for e in range(colptr[m], colptr[m + 1]):
            assert np.array_equal(vals[:, e], U[:, m, row[e] // C, row[e] % C])
    vv = outputs.sparse_values(V, colptr[:1] + [0] * M, [], 1)
    assert vv.shape == (2, 0)


def test_prevalence_invariants(orc):
    w = W.config_sise(n_nodes=200, days=30, gen_seed=2)
    code, U, V, R, err = orc.run(w)
    pop = outputs.prevalence(U, [1], [0, 1], "pop")
    nop = outputs.prevalence(U, [1], [0, 1], "nop")
    assert np.all((pop >= 0) & (pop <= 1)) and np.all((nop >= 0) & (nop <= 1))
    # cases are among those at risk (I ~ S + I): both counts are ordered
    k = outputs.prevalence_counts(U, [1], [0, 1])
    assert np.all(k[..., 2] <= k[..., 3]) and np.all(k[..., 0] <= k[..., 1])
    # whole-population identity: sum of cases = I total
    assert np.array_equal(k[..., 0], U[..., 1].sum(axis=-1))
