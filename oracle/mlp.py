"""FP64 CPU reference of the surrogate MLP (TEST INFRASTRUCTURE).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it.
Network per member: h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = W3 h2 + b3,
loss = mean over rows and outputs of (y - t)^2.  Backward is the chain rule
written out layer by layer; it is pinned by central finite differences in
tests/test_mlp_oracle.py.
"""
from __future__ import annotations

import numpy as np


def unpack(p, nin, nh, nout):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    out = []
    for shape in ((nh, nin), (nh,), (nh, nh), (nh,), (nout, nh), (nout,)):
        size = int(np.prod(shape))
        out.append(p[o:o + size].reshape(shape))
        o += size
    assert o == p.size
    return out


def num_params(nin, nh, nout):
    return nh * nin + nh + nh * nh + nh + nout * nh + nout


def forward(p, x, nin, nh, nout):
    W1, b1, W2, b2, W3, b3 = unpack(p, nin, nh, nout)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3.T + b3, (x, h1, h2)


def loss_and_grads(p, x, t, nin, nh, nout):
    W1, b1, W2, b2, W3, b3 = unpack(p, nin, nh, nout)
    y, (x, h1, h2) = forward(p, x, nin, nh, nout)
    t = np.asarray(t, dtype=np.float64)
    n = x.shape[0]
    d = y - t
    loss = float(np.mean(d * d))
    dy = 2.0 * d / (n * nout)
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dz2 = (dy @ W3) * (1.0 - h2 * h2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (1.0 - h1 * h1)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return loss, g
