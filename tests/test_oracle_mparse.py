"""Pins for the oracle's model parser (Sec. 3.5, transition strings
"LHS -> propensity -> RHS") and the generic kind it feeds.

- S and G of the paper's examples, worked out by hand.
- Compiled propensities equal Python's own evaluation of the same strings
  (an independent parser with the same precedence and IEEE doubles), bit for
  bit, on random states, including precedence and sign corner cases.
- The parsed SIR of Sec. 3.5 reproduces the built-in SIR (Appendix C, same
  operation order) bit for bit, for both solvers.
- Icum counts infections: Icum(t) = S(0) - S(t) in every node.
- A parsed birth-death process follows its closed form:
  X(t) ~ Bin(X0, e^{-mu t}) + Poisson(lambda / mu (1 - e^{-mu t})).
- The Rosenzweig-MacArthur predator-prey model: the summary table the paper
  prints (Sec. 3.5, 1,000 nodes, R = 1000, F = 100, tspan 1..100).
"""
import math

import numpy as np
import pytest

from oracle import mparse
from paper_1605_01421_gb300 import workloads as W

scipy = pytest.importorskip("scipy")
from scipy import stats  # noqa: E402


def test_tables_of_the_paper_examples():
    p = mparse.parse(W.MPARSE_SIR, ["S", "I", "R"], ["b", "g"])
    assert p.S.tolist() == [[-1, 0], [1, -1], [0, 1]]
    assert p.G.tolist() == [[1, 1], [1, 1]]
    p = mparse.parse(W.MPARSE_SIR_ICUM, ["S", "I", "Icum", "R"], ["b", "g"])
    assert p.S.tolist() == [[-1, 0], [1, -1], [1, 0], [0, 1]]
    assert p.G.tolist() == [[1, 1], [1, 1]]
    p = mparse.parse(W.MPARSE_PREDATOR_PREY, ["R", "F"], list(W.PREDATOR_PREY_GDATA))
    assert p.S.tolist() == [[1, -1, -1, 0, 0], [0, 0, 0, 1, -1]]
    # rate k reads: R; R; R, F; R, F; F -- transitions 0-2 change R, 3-4 F
    assert p.G.tolist() == [[1, 1, 1, 0, 0], [1, 1, 1, 0, 0], [1, 1, 1, 1, 1],
                            [1, 1, 1, 1, 1], [0, 0, 0, 1, 1]]
    p = mparse.parse(["@ -> k -> 2*X + Y", "X + Y -> c*X*Y -> @"], ["X", "Y"], ["k", "c"])
    assert p.S.tolist() == [[2, -1], [1, -1]]
    assert p.G.tolist() == [[0, 0], [1, 1]]


CASES = [
    (W.MPARSE_PREDATOR_PREY, ["R", "F"], list(W.PREDATOR_PREY_GDATA)),
    (W.MPARSE_SIR_ICUM, ["S", "I", "Icum", "R"], ["b", "g"]),
    (["A -> a-b-c -> B", "A -> a/b*c -> B", "A -> -a*b -> B", "A -> a-(b-c)*-A -> B",
      "A -> 2.5e-1*A/(1+B)/3 -> B", "A -> .5*+B - -A -> B", "A -> ((a)) -> B"],
     ["A", "B"], ["a", "b", "c"]),
]


@pytest.mark.parametrize("trans,comps,gnames", CASES)
def test_compiled_propensities_equal_python_evaluation(trans, comps, gnames):
    import ctypes
    c = mparse.compiled({"transitions": trans, "compartments": comps, "gdata_names": gnames})
    rng = np.random.default_rng(5)
    for _ in range(300):
        u = rng.integers(0, 5000, len(comps)).astype(np.int32)
        gd = rng.uniform(0.01, 3.0, len(gnames))
        env = {n: float(x) for n, x in zip(comps, u)}
        env.update({n: float(x) for n, x in zip(gnames, gd)})
        up = u.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        gp = gd.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        for j, tr in enumerate(trans):
            text = tr.split("->")[1]
            want = eval(text, {"__builtins__": {}}, env)  # Python's parser
            got = c.fn(j, up, gp)
            assert np.float64(got).view(np.uint64) == np.float64(want).view(np.uint64), (tr, u, gd)
            assert got == mparse.evaluate(c.parsed.trees[j], u, gd)


@pytest.mark.parametrize("solver", [W.SSM, W.AEM], ids=["ssm", "aem"])
def test_parsed_sir_is_the_builtin_sir(orc, solver):
    u0 = np.tile([[99, 5, 0]], (1000, 1))
    builtin = W.plain_model(W.SIR, u0, np.arange(1, 181), [0.16, 0.077], seed=123)
    parsed = W.parsed_model(W.MPARSE_SIR, ["S", "I", "R"], {"b": 0.16, "g": 0.077}, u0,
                            np.arange(1, 181), seed=123)
    builtin.solver = parsed.solver = solver
    a = orc.run(builtin)
    b = orc.run(parsed)
    assert a[0] == 0 and b[0] == 0
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[3], b[3])


def test_icum_counts_infections(orc):
    w = W.config_sir_icum()
    code, U, V, R, err = orc.run(w)
    assert code == 0
    assert np.array_equal(U[0, :, :, 2], U[0, 0, :, 0][None, :] - U[0, :, :, 0])
    # and S + I + R stays 100
    assert np.all(U[0, :, :, 0] + U[0, :, :, 1] + U[0, :, :, 3] == 100)


def test_parsed_birth_death_closed_form(orc):
    lam, mu, X0, nodes = 3.0, 0.4, 6, 40_000
    w = W.parsed_model(["@ -> lam -> X", "X -> mu*X -> @"], ["X"], {"lam": lam, "mu": mu},
                       np.full((nodes, 1), X0), np.arange(0, 7), seed=17)
    for solver in (W.SSM, W.AEM):
        w.solver = solver
        code, U, V, R, err = orc.run(w)
        assert code == 0
        for d in (1, 3, 6):
            q = math.exp(-mu * d)
            hi = 60
            pmf = np.convolve(stats.binom.pmf(np.arange(X0 + 1), X0, q),
                              stats.poisson.pmf(np.arange(hi), lam / mu * (1 - q)))[:hi]
            obs = np.bincount(U[0, d][:, 0], minlength=hi)[:hi].astype(float)
            exp = pmf * nodes
            keep = exp >= 5
            o = np.r_[obs[keep], nodes - obs[keep].sum()]
            e = np.r_[exp[keep], nodes - exp[keep].sum()]
            assert stats.chisquare(o, e).pvalue > 1e-3, (solver, d)


def test_predator_prey_matches_the_printed_summary(orc):
    # The paper's summary over 1,000 nodes x 100 time points:
    #   R: 1st Qu. 236, median 607, mean 598, 3rd Qu. 975
    #   F: median 35, mean 112, 3rd Qu. 161
    w = W.config_predator_prey(n_nodes=300, seed=7)
    code, U, V, R, err = orc.run(w)
    assert code == 0
    r, f = U[0, :, :, 0].ravel(), U[0, :, :, 1].ravel()
    assert abs(np.percentile(r, 25) / 236 - 1) < 0.25
    assert abs(np.median(r) / 607 - 1) < 0.20
    assert abs(r.mean() / 598 - 1) < 0.10
    assert abs(np.percentile(r, 75) / 975 - 1) < 0.05
    assert np.percentile(f, 25) == 0
    assert abs(f.mean() / 112 - 1) < 0.15
    assert abs(np.percentile(f, 75) / 161 - 1) < 0.25


def test_parse_errors():
    bad = [(["S -> b*Q -> I"], ["S", "I"], ["b"]),        # unknown name
           (["S -> b*(S -> I"], ["S", "I"], ["b"]),       # three arrows, unbalanced
           (["S -> b*(S+I -> I"], ["S", "I"], ["b"]),     # missing ')'
           (["S -> b S -> I"], ["S", "I"], ["b"]),        # missing operator
           (["S -> b -> Z"], ["S", "I"], ["b"]),          # unknown compartment
           (["S -> S -> I"], ["S", "I"], ["S"])]          # name clash
    for t, c, g in bad:
        with pytest.raises(mparse.ParseError):
            mparse.parse(t, c, g)
