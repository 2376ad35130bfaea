"""CPU pins of the float64 MLP reference in tests/_mlp_ref.py (used by the GPU ranker tests):
its analytic gradient against central differences, and its forward pass against a
hand-written loop over one sample."""
import numpy as np

import pytest

from _mlp_ref import np_forward, np_grad, np_loss, small_problem, unpack


@pytest.mark.parametrize("fw", [0.0, 1.0])
def test_numpy_reference_gradient_matches_central_differences(fw):
    """The analytic gradient of the reference equals central differences of its loss."""
    X, T, H = small_problem()
    rng = np.random.default_rng(5)
    n, F = X.shape
    P = {"mu": X.mean(0).astype(np.float64), "sd": X.std(0).astype(np.float64),
         "tmu": float(np.log(T).mean()), "tsd": float(np.log(T).std()),
         "W1": rng.uniform(-1, 1, (H, F)), "b1": rng.uniform(-0.1, 0.1, H), "W2": rng.uniform(-0.5, 0.5, (H, H)),
         "b2": rng.uniform(-0.1, 0.1, H), "w3": rng.uniform(-0.5, 0.5, H), "b3": 0.05}
    flat = np.concatenate([P["mu"], P["sd"], [P["tmu"], P["tsd"]], P["W1"].ravel(), P["b1"], P["W2"].ravel(),
                           P["b2"], P["w3"], [P["b3"]]])
    g = np_grad(unpack(flat, F, H), X.astype(np.float64), T.astype(np.float64), fw)
    h = 1e-6
    fd = np.zeros_like(g)
    for q in range(2 * F + 2, len(flat)):
        a, b = flat.copy(), flat.copy()
        a[q] += h
        b[q] -= h
        fd[q] = (np_loss(unpack(a, F, H), X, T, fw) - np_loss(unpack(b, F, H), X, T, fw)) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-5, atol=1e-7 * np.abs(g).max())


def test_forward_matches_a_loop_over_one_sample():
    X, T, H = small_problem()
    n, F = X.shape
    rng = np.random.default_rng(11)
    flat = np.concatenate([X.mean(0), X.std(0), [0.1, 0.9], rng.normal(size=H * F), rng.normal(size=H),
                           rng.normal(size=H * H) / 4, rng.normal(size=H), rng.normal(size=H), [0.2]])
    P = unpack(flat, F, H)
    y = np_forward(P, X.astype(np.float64))[3]
    s = 3
    x = [(float(X[s, f]) - flat[f]) / flat[F + f] for f in range(F)]
    W1 = flat[2 * F + 2:2 * F + 2 + H * F]
    o = 2 * F + 2 + H * F
    h1 = [max(0.0, flat[o + j] + sum(W1[j * F + f] * x[f] for f in range(F))) for j in range(H)]
    W2 = flat[o + H:o + H + H * H]
    o2 = o + H + H * H
    h2 = [max(0.0, flat[o2 + j] + sum(W2[j * H + k] * h1[k] for k in range(H))) for j in range(H)]
    w3 = flat[o2 + H:o2 + 2 * H]
    ys = flat[-1] + sum(w3[k] * h2[k] for k in range(H))
    assert abs(y[s] - ys) <= 1e-12 * max(1.0, abs(ys))


def test_weights_favour_fast_samples_and_average_one():
    from _mlp_ref import np_weights
    t = np.array([-2.0, 0.0, 1.5])
    w = np_weights(t, 1.0)
    assert abs(w.mean() - 1.0) < 1e-12 and w[0] > w[1] > w[2]
    assert np.allclose(w[0] / w[1], np.exp(2.0)) and np.allclose(np_weights(t, 0.0), 1.0)
