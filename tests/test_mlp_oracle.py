"""The FP64 MLP reference against central finite differences (CPU)."""
import numpy as np

from oracle import mlp


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    nin, nh, nout, n = 4, 8, 5, 7
    P = mlp.num_params(nin, nh, nout)
    p = rng.normal(0, 0.5, P)
    x = rng.normal(0, 1, (n, nin))
    t = rng.normal(0, 1, (n, nout))
    loss, g = mlp.loss_and_grads(p, x, t, nin, nh, nout)
    eps = 1e-6
    for i in range(P):   # every parameter of every tensor
        e = np.zeros(P)
        e[i] = eps
        lp = mlp.loss_and_grads(p + e, x, t, nin, nh, nout)[0]
        lm = mlp.loss_and_grads(p - e, x, t, nin, nh, nout)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) < 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_layout_and_forward():
    nin, nh, nout = 3, 4, 2
    P = mlp.num_params(nin, nh, nout)
    p = np.arange(P, dtype=float) * 1e-3
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, nin, nh, nout)
    assert W1.shape == (4, 3) and W1[1, 0] == 3e-3 and b1[0] == 12e-3
    x = np.ones((1, nin))
    y, _ = mlp.forward(p, x, nin, nh, nout)
    h1 = np.tanh(W1.sum(1) + b1)
    h2 = np.tanh(W2 @ h1 + b2)
    np.testing.assert_allclose(y[0], W3 @ h2 + b3, rtol=1e-15)
