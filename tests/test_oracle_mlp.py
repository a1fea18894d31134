"""Pins of the FP64 reference MLP: finite differences of the loss and a
hand-computed example (no GPU)."""
import numpy as np

from oracle import mlp


def _params(rng, n_in=7, h=5, n_out=3):
    return [rng.standard_normal((h, n_in)) * 0.5, rng.standard_normal(h) * 0.1,
            rng.standard_normal((h, h)) * 0.5, rng.standard_normal(h) * 0.1,
            rng.standard_normal((n_out, h)) * 0.5, rng.standard_normal(n_out) * 0.1]


def test_backward_matches_central_fd():
    rng = np.random.default_rng(0)
    P = _params(rng)
    X = rng.standard_normal((11, 7))
    T = rng.standard_normal((11, 3))
    L, grads = mlp.backward(X, T, P)
    h = 1e-6
    for k, p in enumerate(P):
        fd = np.zeros_like(p)
        it = np.nditer(p, flags=["multi_index"])
        for _ in it:
            i = it.multi_index
            Pp = [q.copy() for q in P]
            Pm = [q.copy() for q in P]
            Pp[k][i] += h
            Pm[k][i] -= h
            fd[i] = (mlp.loss(mlp.forward(X, Pp)[0], T) - mlp.loss(mlp.forward(X, Pm)[0], T)) / (2 * h)
        np.testing.assert_allclose(grads[k], fd, rtol=1e-6, atol=1e-8)


def test_hand_example():
    # one input, two hidden units per layer, one output; relu cuts unit 2
    W1 = np.array([[2.0], [-1.0]]); b1 = np.array([0.5, 0.0])
    W2 = np.array([[1.0, 3.0], [0.0, -1.0]]); b2 = np.array([0.0, 0.25])
    W3 = np.array([[1.0, 2.0]]); b3 = np.array([-1.0])
    X = np.array([[1.0]])
    Y, _ = mlp.forward(X, [W1, b1, W2, b2, W3, b3])
    # Z1 = (2.5, -1) -> H1 = (2.5, 0); Z2 = (2.5, 0.25) -> H2 = (2.5, 0.25); Y = 2.5 + 0.5 - 1
    assert Y.shape == (1, 1) and abs(Y[0, 0] - 2.0) < 1e-15


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, 3.14159, -2.5e-3, 0.0])
    r = mlp.bf16_round(vals)
    assert r[0] == 1.0 and r[1] == 1.0              # tie to even
    assert r[2] == 1.0 + 2 ** -7                    # tie to even (odd -> up)
    assert abs(r[3] - 3.140625) < 1e-15
    assert np.all(np.abs(r - vals) <= np.abs(vals) * 2 ** -8)
