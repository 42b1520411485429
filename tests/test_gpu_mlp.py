"""Surrogate MLP kernels against the FP64 reference (needs a GPU).

Gradients: BF16 operands with FP32 accumulation against FP64; with weights that
BF16 represents exactly, the remaining error comes from rounding activations
and upstream gradients to BF16 (8-bit mantissas), so each parameter tensor's
gradient is required within 1e-2 relative (L2 norm).
"""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0911_0459_gb300.mlp import MLP  # noqa: E402


def bf16_round(a):
    a = np.asarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16       # round to nearest even
    return b.astype(np.uint32).view(np.float32)


def split(g, nin, nh, nout):
    return ref.unpack(g, nin, nh, nout)


@pytest.mark.parametrize("n", [64, 1000, 4096])
def test_gradients_match_fp64_reference(n):
    nin, nh, nout = 4, 256, 64
    net = MLP(nin, nh, nout, members=2, max_batch=4096, seed=3)
    rng = np.random.default_rng(n)
    x = rng.uniform(-1, 1, (n, nin)).astype(np.float32)
    y = rng.normal(0, 1, (n, nout)).astype(np.float32)
    net.set_data(x, y)
    for k in range(2):
        p = bf16_round(net.get_params(k) + rng.normal(0, 0.02, net.P).astype(np.float32))
        net.set_params(k, p)
        loss, g = net.gradients(k)
        rloss, rg = ref.loss_and_grads(p.astype(np.float64), bf16_round(x).astype(np.float64), y, nin, nh, nout)
        assert abs(loss / rloss - 1) < 1e-2
        for name, a, b in zip(("W1", "b1", "W2", "b2", "W3", "b3"), split(g, nin, nh, nout),
                              split(rg, nin, nh, nout)):
            err = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert err < 1e-2, (k, name, err)
    net.close()


def test_training_fits_a_smooth_map_and_ensemble_statistics():
    nin, nh, nout = 4, 256, 64
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, (2048, nin)).astype(np.float32)
    tgrid = np.linspace(0, 1, nout)
    y = (np.sin(2 * x[:, :1] + 3 * tgrid) * (1 + 0.3 * x[:, 1:2]) + 0.5 * x[:, 2:3] * tgrid
         - 0.2 * x[:, 3:4] ** 2).astype(np.float32)
    net = MLP(nin, nh, nout, members=3, max_batch=4096, seed=7)
    net.set_data(x, y)
    l0 = net.gradients(0)[0]
    losses = net.train(1500, lr=3e-3, lr_min=3e-5, wd=1e-5)
    assert np.all(losses < 0.02 * l0), (l0, losses)
    xt = rng.uniform(-1, 1, (300, nin)).astype(np.float32)
    yt = (np.sin(2 * xt[:, :1] + 3 * tgrid) * (1 + 0.3 * xt[:, 1:2]) + 0.5 * xt[:, 2:3] * tgrid
          - 0.2 * xt[:, 3:4] ** 2)
    mean, sd, mem = net.predict(xt, members=True)
    np.testing.assert_allclose(mean, mem.mean(0), atol=1e-5)
    np.testing.assert_allclose(sd, mem.std(0, ddof=1), atol=1e-5)
    assert np.sqrt(np.mean((mean - yt) ** 2)) < 0.05
    # each member's forward against the FP64 reference on its own parameters
    for k in range(3):
        p = net.get_params(k).astype(np.float64)
        yr, _ = ref.forward(p, xt.astype(np.float64), nin, nh, nout)
        assert np.abs(mem[k] - yr).max() < 3e-2 * max(1.0, np.abs(yr).max())
    net.close()
