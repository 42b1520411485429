"""Batched persistent kernel against independent lattices and the oracle (needs a GPU)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0911_0459_gb300 import STORAGE_F16DEV, STORAGE_F32, STORAGE_F64, Batch, Lattice, LbError  # noqa: E402
from paper_0911_0459_gb300 import lb as lbmod  # noqa: E402


def small_sweep(seed=7, n=6):
    """Uneven capillaries shaped like the sweep, shortened so the oracle keeps up."""
    caps = W.sweep(seed=seed, n=n, lengths=(96, 300))
    out = []
    for c in caps:
        c.nx = c.tube_x0 + c.tube_len   # keep the reservoirs, short tubes
        out.append(c)
    return out


@pytest.mark.parametrize("storage", [STORAGE_F32, STORAGE_F64, STORAGE_F16DEV])
def test_batch_is_bitwise_identical_to_independent_lattices(storage):
    caps = small_sweep()
    b = Batch(caps, storage=storage)
    for tx, ty in ((64, 4), (128, 16), (256, 64)):
        b.set_tile(tx, ty)
        b.step(13)
    total = b.time
    for i, c in enumerate(caps):
        lat = Lattice.from_workload(c, storage=storage)
        lat.step(total)
        fb, gb = b.populations(i, rested=False)
        fl, gl = lat.populations(rested=False)
        assert np.array_equal(fb, fl) and np.array_equal(gb, gl), i
        lat.close()
    b.close()


def test_batch_sampled_run_matches_oracle():
    caps = small_sweep(seed=3, n=4)
    b = Batch(caps, storage=STORAGE_F32)
    at = [1, 5, 40, 120, 300]
    out = b.run_sampled(at)
    assert out.shape == (4, 5, 4)
    for i, c in enumerate(caps):
        orc = oracle.Oracle(c, wall_grad=lbmod.binary_wall_gradient(c.theta_deg, c.params.A, c.params.kappa))
        orc.init_default()
        t = 0
        for k, s in enumerate(at):
            orc.step(s - t)
            t = s
            d = orc.filled_length()
            assert abs(out[i, k, 0] - d["l"]) < 0.05, (i, k, out[i, k, 0], d["l"])
            assert abs(out[i, k, 2] / d["mass"] - 1) < 1e-6
            assert abs(out[i, k, 3] - d["phi_sum"]) < 1e-6 * c.nodes
    assert b.time == at[-1]
    # lengths() agrees with the last sample
    np.testing.assert_allclose(b.lengths(), out[:, -1, :], rtol=0, atol=0)
    b.close()


def test_batch_autotune_and_fluid_count():
    caps = small_sweep(seed=11, n=5)
    b = Batch(caps)
    tx, ty, ms = b.autotune(steps=2)
    assert tx in (64, 128, 256) and ms > 0
    assert b.fluid_nodes() == sum(b.fluid_nodes(i) for i in range(len(caps)))
    b.close()


def test_grid_barrier_timeout_is_reported_without_hanging():
    """Failure injection on the host: the barrier waits for an arrival that never
    comes, gives up after its short limit, and the host reads LB_ERR_TIMEOUT."""
    caps = small_sweep(seed=5, n=3)
    b = Batch(caps)
    b.set_barrier(absent_blocks=1, limit_seconds=0.05)
    b.step(3)
    with pytest.raises(LbError) as e:
        b.lengths()
    assert e.value.status == lbmod.LB_ERR_TIMEOUT
    with pytest.raises(LbError) as e:
        b.step(1)
    assert e.value.status == lbmod.LB_ERR_STATE
    b.close()
    # the GPU context stays usable
    b2 = Batch(caps)
    b2.step(4)
    assert np.isfinite(b2.lengths()).all()
    b2.close()
