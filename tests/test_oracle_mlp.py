"""Pin of the MLP reference: its chain-rule gradient equals central finite
differences of its loss (float64), on random networks and data."""
import numpy as np

from oracle import mlp_ref as M


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    n_in, H, N = 7, 9, 13
    p = M.init_params(n_in, H, 1) + 0.05 * rng.standard_normal(M.n_params(n_in, H))
    x = rng.standard_normal((N, n_in))
    t = rng.standard_normal(N)
    g = M.gradient(p, x, t, n_in, H)
    h = 1e-6
    idx = rng.choice(len(p), 60, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (M.loss(p + e, x, t, n_in, H) - M.loss(p - e, x, t, n_in, H)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_forward_small_closed_form():
    # one hidden unit each, all weights 1: y = relu(relu(x1 + x2) ) + 0
    n_in, H = 2, 1
    p = np.array([1.0, 1.0, 0.0, 1.0, 0.0, 1.0, 0.0])
    y, _ = M.forward(p, np.array([[1.0, 2.0], [-3.0, 1.0]]), n_in, H)
    assert np.allclose(y, [3.0, 0.0])
