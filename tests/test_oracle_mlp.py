"""Pin of the FP64 emulator-network oracle: its analytic gradients equal
central finite differences of its own loss (a check independent of the
chain-rule code)."""
import numpy as np

from oracle import mlp


def _tiny(rng):
    dims = [(8, 5), (7, 8), (mlp.HEADS * mlp.BINS + 2, 7)]
    Ws = [rng.standard_normal(d) * 0.5 for d in dims]
    bs = [rng.standard_normal(d[0]) * 0.1 for d in dims]
    X = rng.standard_normal((6, 5))
    t = rng.integers(0, mlp.BINS, (6, mlp.HEADS))
    return Ws, bs, X, t


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    Ws, bs, X, t = _tiny(rng)
    loss, dW, db = mlp.loss_and_grads(Ws, bs, X, t)
    eps = 1e-6
    for li in range(3):
        for _ in range(12):
            i, j = rng.integers(0, Ws[li].shape[0]), rng.integers(0, Ws[li].shape[1])
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[li][i, j] += eps
            Wm[li][i, j] -= eps
            num = (mlp.loss_and_grads(Wp, bs, X, t)[0] - mlp.loss_and_grads(Wm, bs, X, t)[0]) / (2 * eps)
            assert abs(num - dW[li][i, j]) < 1e-6 * max(1.0, abs(num))
        k = rng.integers(0, bs[li].shape[0])
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[li][k] += eps
        bm[li][k] -= eps
        num = (mlp.loss_and_grads(Ws, bp, X, t)[0] - mlp.loss_and_grads(Ws, bm, X, t)[0]) / (2 * eps)
        assert abs(num - db[li][k]) < 1e-6 * max(1.0, abs(num))


def test_gelu_matches_its_definition_and_derivative():
    x = np.linspace(-6, 6, 2001)
    # the tanh form approximates x Phi(x) to within 1e-3
    from math import erf, sqrt
    exact = np.array([0.5 * v * (1 + erf(v / sqrt(2))) for v in x])
    assert np.abs(mlp.gelu(x) - exact).max() < 1e-3
    h = 1e-6
    num = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.abs(num - mlp.gelu_grad(x)).max() < 1e-7


def test_loss_of_uniform_logits():
    # zero weights and biases: every head is uniform over 129 bins
    dims = [(4, 3), (mlp.HEADS * mlp.BINS, 4)]
    Ws = [np.zeros(d) for d in dims]
    bs = [np.zeros(d[0]) for d in dims]
    X = np.ones((5, 3))
    t = np.zeros((5, mlp.HEADS), dtype=int)
    loss, _, _ = mlp.loss_and_grads(Ws, bs, X, t)
    assert abs(loss - mlp.HEADS * np.log(mlp.BINS)) < 1e-12
