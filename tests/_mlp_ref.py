"""Float64 numpy restatement of the ranker's MLP (forward pass, loss, analytic gradient), the
reference the GPU tests compare the hand-written training and inference kernels with.

Model (the parameter layout of acs.h): x = (features - mu) / sd, h1 = relu(W1 x + b1),
h2 = relu(W2 h1 + b2), y = w3 . h2 + b3; target t = (log time - tmu) / tsd; loss = mean of
w_i (y - t)^2 over the samples, w_i = exp(-a t_i) normalised to mean 1 (a = fast_weight).
Test infrastructure only.
"""
import numpy as np


def unpack(p, F, H):
    """Split the parameter buffer (layout of acs.h) into named float64 arrays."""
    p = np.asarray(p, dtype=np.float64)
    o = 0
    out = {}
    for name, shape in (("mu", (F,)), ("sd", (F,)), ("tmu", ()), ("tsd", ()), ("W1", (H, F)), ("b1", (H,)),
                        ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", ())):
        size = int(np.prod(shape)) if shape else 1
        out[name] = p[o:o + size].reshape(shape) if shape else p[o]
        o += size
    assert o == len(p)
    return out


def np_forward(P, X):
    x = (X - P["mu"]) / P["sd"]
    z1 = x @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    return x, h1, h2, h2 @ P["w3"] + P["b3"]


def np_weights(t, fast_weight):
    """Sample weights exp(-a t_i) normalised to mean 1 (a = 0: all ones)."""
    w = np.exp(-fast_weight * t)
    return w * len(w) / w.sum()


def np_loss(P, X, T, fast_weight=0.0):
    t = (np.log(T) - P["tmu"]) / P["tsd"]
    return float(np.mean(np_weights(t, fast_weight) * (np_forward(P, X)[3] - t) ** 2))


def np_grad(P, X, T, fast_weight=0.0):
    """Analytic gradient of the weighted mean squared error of the standardised log time
    (float64), flattened in the buffer layout (zeros for the fixed statistics)."""
    n = X.shape[0]
    x, h1, h2, y = np_forward(P, X)
    t = (np.log(T) - P["tmu"]) / P["tsd"]
    dy = 2.0 * np_weights(t, fast_weight) * (y - t) / n
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    dh2 = np.outer(dy, P["w3"]) * (h2 > 0)
    g_W2 = dh2.T @ h1
    g_b2 = dh2.sum(0)
    dh1 = (dh2 @ P["W2"]) * (h1 > 0)
    g_W1 = dh1.T @ x
    g_b1 = dh1.sum(0)
    F = X.shape[1]
    return np.concatenate([np.zeros(2 * F + 2), g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])


def small_problem(seed=77, n=24, F=6, H=16):
    """Seeded features and positive times of a small training set, and the hidden width."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(-2, 5, size=(n, F)).astype(np.float32)
    T = np.exp(0.3 * X[:, 0] - 0.2 * X[:, 2] + rng.normal(0, 0.1, n)).astype(np.float32)
    return X, T, H
