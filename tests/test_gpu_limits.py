"""Degenerate calls and the largest lattices of each step kernel (needs a GPU)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0911_0459_gb300 import (STORAGE_F16_BLOCKED, STORAGE_F32, STORAGE_F32_BLOCKED, Batch, Lattice,  # noqa: E402
                                   LbError)

# the staged kernel stores at 32-bit element offsets over 9 planes: 9 nx ny < 2^32
STAGED_MAX_NODES = (2 ** 32 - 1) // 9


def small(seed):
    caps = W.sweep(seed=seed, n=2, lengths=(96, 200))
    for c in caps:
        c.nx = c.tube_x0 + c.tube_len
    return caps


def test_zero_steps_and_repeated_samples_change_nothing():
    cap = small(3)[0]
    lat = Lattice.from_workload(cap)
    lat.step(7)
    f0, g0 = lat.populations(rested=False)
    lat.step(0)
    f1, g1 = lat.populations(rested=False)
    assert lat.time == 7 and np.array_equal(f0, f1) and np.array_equal(g0, g1)
    lat.close()

    caps = small(4)
    b = Batch(caps)
    b.step(5)
    before = b.lengths()
    b.step(0)
    assert b.time == 5 and np.array_equal(b.lengths(), before)
    out = b.run_sampled([0, 0, 3])
    assert b.time == 8
    np.testing.assert_array_equal(out[:, 0], before)
    np.testing.assert_array_equal(out[:, 1], before)
    np.testing.assert_array_equal(out[:, 2], b.lengths())
    with pytest.raises(LbError):
        b.run_sampled([])
    with pytest.raises(LbError):
        b.run_sampled([3, 2])
    with pytest.raises(LbError):
        b.step(-1)
    b.close()
    with pytest.raises(LbError):
        Batch([])


@pytest.mark.parametrize("ny,staged", [(7281, True), (7282, False)])
def test_largest_lattices_of_the_staged_kernel(ny, staged):
    """65536 x 7281 = 477,167,616 nodes is the largest 65536-wide lattice the staged kernel
    takes (9 N < 2^32); one more row (477,233,152 nodes, 34 GB in FP32) runs on the
    sliding-window kernel, which the automatic choice picks and an explicit request for the
    staged kernel is refused.  A uniform liquid-gas box at rest: two steps keep it at rest
    with its mass."""
    nx = 65536
    assert (nx * ny <= STAGED_MAX_NODES) == staged
    cap = W.periodic_box(nx, ny, W.lg_params(storage=STORAGE_F32))
    lat = Lattice.from_workload(cap)
    assert lat.kernel() == (2 if staged else 1)
    if not staged:
        with pytest.raises(LbError):
            lat.set_kernel(2)
    m0 = lat.filled_length()["mass"]
    lat.step(2)
    torch.cuda.synchronize()
    m1 = lat.filled_length()["mass"]
    assert np.isfinite(m1) and abs(m1 / m0 - 1) < 1e-6
    assert abs(m0 / (nx * ny) - cap.params.rho_g) < 1e-6 * cap.params.rho_g
    lat.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("nx", [65536, 65535])
@pytest.mark.parametrize("storage,per_node,ny,tol", [(STORAGE_F32_BLOCKED, 18, 3640, 1e-6),
                                                     (STORAGE_F16_BLOCKED, 19, 3449, 1e-5)])
def test_largest_lattices_of_the_block_storages(nx, storage, per_node, ny, tol):
    """The block storages address their state with 32-bit element offsets, 18 (FP32) or 19
    (FP16 halves) x 32 x ceil(N / 32) < 2^32, so at most 238,609,280 or 226,050,880 nodes:
    3640 or 3449 rows of 65536 (rows on block boundaries) or of 65535 (rows starting inside
    blocks) fit (about 34 or 17 GB for both buffers) and run the staged kernel; one more
    row is refused at creation.  Two steps of a binary box keep its mass and its phi sum to
    the storage's rounding."""
    p = W.binary_params(storage=storage)
    assert per_node * 32 * ((nx * ny + 31) // 32) < 2 ** 32 <= per_node * 32 * ((nx * (ny + 1) + 31) // 32)
    with pytest.raises(LbError):
        Lattice.from_workload(W.periodic_box(nx, ny + 1, p))
    lat = Lattice.from_workload(W.periodic_box(nx, ny, p))
    assert lat.kernel() == 2
    d0 = lat.filled_length()
    lat.step(2)
    torch.cuda.synchronize()
    d1 = lat.filled_length()
    assert np.isfinite([d1["mass"], d1["phi_sum"]]).all()
    assert abs(d1["mass"] / d0["mass"] - 1) < tol
    assert abs(d1["phi_sum"] - d0["phi_sum"]) < tol * nx * ny
    lat.close()
    torch.cuda.empty_cache()


def test_fp64_fma_rate_is_measured():
    """lb_fp64_fma_rate times a kernel of independent FP64 FMA chains: a positive rate,
    below the FP32 rate this GPU's SMs could reach (152 SMs x 128 lanes x 2 flops x
    2.1 GHz = 82 TFLOP/s), and the same on a second call within timing noise."""
    from paper_0911_0459_gb300 import lb as lbmod
    a = lbmod.fp64_fma_rate()
    b = lbmod.fp64_fma_rate()
    assert 0.05 < a < 82.0 and 0.05 < b < 82.0, (a, b)
    assert abs(a - b) < 0.2 * max(a, b), (a, b)
