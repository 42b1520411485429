"""FP32 populations in 32-node blocks (LB_STORAGE_F32_BLOCKED) through the C ABI (needs a GPU).

The block storage keeps the values of the FP32 population storage in another order
(f_i of node n at float 576 (n // 32) + 32 i + n % 32, g_i 288 further) and runs the
same arithmetic, so every result equals the FP32 storage's bit for bit: states after
many steps in every kernel variant and tile, through walls, the x-wrap and ragged last
tiles, the reductions and the fields, for rows that start on a block boundary
(nx % 32 == 0) and rows that do not (then a staged row is the whole blocks over its
nodes, and the x-wrap neighbour's block is staged apart).  One step from a random
state also matches the FP64 oracle within FP32's 2e-6 per population, as the FP32
storage does.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0911_0459_gb300 import STORAGE_F32, STORAGE_F32_BLOCKED, Lattice  # noqa: E402

GEOMS = {
    # 352 = 256 + 96: a ragged last tile at every tile width; 37 rows: ragged bands
    "capillary_ragged": lambda p: W.Capillary("br", 352, 37, 64, 224, 5, 27, 12, 8, p, wall_grad=-0.11),
    # the tube wraps through x = 0; the band starts at y = 0
    "tube_wraps_x": lambda p: W.Capillary("bw", 160, 30, 100, 90, 0, 20, 0, 0, p, wall_grad=-0.1),
    # one block per row: both halo blocks wrap
    "one_block": lambda p: W.Capillary("b1", 32, 10, 4, 24, 1, 6, 2, 3, p, wall_grad=-0.15),
    "periodic": lambda p: W.periodic_box(64, 29, p),
    # the fewest rows a tube allows
    "three_rows": lambda p: W.Capillary("b3", 96, 3, 10, 60, 0, 2, 4, 5, p, wall_grad=-0.1),
    # rows that start inside a block
    "unaligned_ragged": lambda p: W.Capillary("u1", 203, 37, 61, 120, 5, 27, 12, 8, p, wall_grad=-0.11),
    "unaligned_tube_wraps": lambda p: W.Capillary("u2", 150, 30, 100, 90, 27, 20, 0, 0, p, wall_grad=-0.1),
    "unaligned_channel": lambda p: W.channel(131, 19, 15, p, wall_grad=-0.15),
    "unaligned_periodic": lambda p: W.periodic_box(77, 29, p),
    "unaligned_three_rows": lambda p: W.Capillary("u3", 45, 3, 10, 25, 0, 2, 4, 5, p, wall_grad=-0.1),
    "unaligned_narrow": lambda p: W.Capillary("u4", 20, 12, 6, 10, 2, 7, 2, 3, p, wall_grad=-0.2),
    # two tiles of 256 and a one-column remainder at the end of every row
    "unaligned_one_column_tail": lambda p: W.Capillary("u5", 513, 9, 100, 300, 1, 6, 20, 10, p, wall_grad=-0.1),
}
# (variant, tile): sliding window, staged shallow ring at three widths, staged deep ring
RUNS = [(1, (128, 16)), (2, (256, 8)), (2, (128, 5)), (2, (64, 1)), (3, (256, 16))]


def to_planes(state, nx, ny):
    """The block storage's saved state as the FP32 storage's (f planes, then g planes)."""
    N = nx * ny
    nb = (N + 31) // 32
    b = np.frombuffer(state.tobytes(), dtype=np.float32).reshape(nb, 18, 32)
    return np.ascontiguousarray(b.transpose(1, 0, 2)).reshape(18, nb * 32)[:, :N].reshape(18 * N)


def planes(lat):
    return np.frombuffer(lat.save_state()[0].tobytes(), dtype=np.float32)


def assert_same_state(blk, ref, nx, ny):
    a, b = to_planes(blk.save_state()[0], nx, ny), planes(ref)
    bad = np.flatnonzero(a.view(np.uint32) != b.view(np.uint32))
    assert bad.size == 0, (bad.size, bad[:5])


def test_saved_state_follows_the_documented_layout():
    """lb_save_state of the block storage holds f_i of node n at float 576 (n // 32) +
    32 i + n % 32 and g_i 288 floats further: read back against lb_get_populations."""
    cap = GEOMS["unaligned_ragged"](W.binary_params(nu_l=0.7, nu_g=0.05))
    lat = Lattice.from_workload(cap, storage=STORAGE_F32_BLOCKED)
    lat.step(37)
    f, g = lat.populations(rested=False)
    st = np.frombuffer(lat.save_state()[0].tobytes(), dtype=np.float32)
    assert st.size == 18 * 32 * ((cap.nx * cap.ny + 31) // 32)
    n = np.arange(cap.nx * cap.ny)
    for i in range(9):
        assert np.array_equal(st[576 * (n // 32) + 32 * i + n % 32].astype(np.float64), f[i].ravel())
        assert np.array_equal(st[288 + 576 * (n // 32) + 32 * i + n % 32].astype(np.float64), g[i].ravel())


@pytest.mark.parametrize("geom", sorted(GEOMS))
def test_one_step_random_state_matches_oracle_and_fp32(geom):
    cap = GEOMS[geom](W.binary_params(nu_l=0.7, nu_g=0.05, M=0.2))
    fields = W.random_state_fields(cap.nx, cap.ny, seed=11, model=W.BINARY)
    orc = oracle.Oracle(cap)
    orc.init_fields(*fields)
    orc.step(1)
    fo, go = orc.populations()
    ref = Lattice.from_workload(cap, storage=STORAGE_F32).init_fields(*fields).step(1)
    for variant, (tx, ty) in RUNS:
        lat = Lattice.from_workload(cap, storage=STORAGE_F32_BLOCKED)
        lat.set_kernel(variant)
        lat.set_tile(tx, min(ty, cap.ny))
        lat.init_fields(*fields)
        lat.step(1)
        f, g = lat.populations(rested=True)
        assert np.abs(f - fo).max() < 2e-6 and np.abs(g - go).max() < 2e-6, (variant, tx, ty)
        assert_same_state(lat, ref, cap.nx, cap.ny)
        lat.close()


@pytest.mark.parametrize("geom", sorted(GEOMS))
def test_many_steps_bitwise_equal_to_fp32(geom):
    """300 steps from the default state (a meniscus moving along the tube), with the
    l(t) reductions every 100 steps: every bit equal to the FP32 storage's run."""
    cap = GEOMS[geom](W.binary_params(nu_l=0.83, nu_g=0.083))
    ref = Lattice.from_workload(cap, storage=STORAGE_F32)
    ls_ref = []
    for _ in range(3):
        ref.step(100)
        ls_ref.append(ref.filled_length())
    rf = ref.fields()
    for variant, (tx, ty) in RUNS:
        lat = Lattice.from_workload(cap, storage=STORAGE_F32_BLOCKED)
        lat.set_kernel(variant)
        lat.set_tile(tx, min(ty, cap.ny))
        ls = []
        for _ in range(3):
            lat.step(100)
            ls.append(lat.filled_length())
        assert ls == ls_ref, (variant, tx, ty)
        assert_same_state(lat, ref, cap.nx, cap.ny)
        for a, b in zip(lat.fields(), rf):
            assert np.array_equal(a, b)
        lat.close()


def test_populations_and_checkpoint_round_trip():
    cap = GEOMS["tube_wraps_x"](W.binary_params(nu_l=0.5, nu_g=0.05))
    lat = Lattice.from_workload(cap, storage=STORAGE_F32_BLOCKED)
    lat.step(50)
    buf, t = lat.save_state()
    f, g = lat.populations(rested=False)
    lat.step(30)
    after = planes(lat).copy()
    # resume from the checkpoint: the same 30 steps give the same bits
    lat.load_state(buf, t)
    lat.step(30)
    assert np.array_equal(planes(lat).view(np.uint32), after.view(np.uint32))
    # populations written back (FP64 -> FP32, exact for FP32 values) restore the state
    other = Lattice.from_workload(cap, storage=STORAGE_F32_BLOCKED)
    other.set_populations(f, g)
    assert np.array_equal(other.save_state()[0], buf)


def test_full_size_16384x256_bitwise_equal_to_fp32():
    """The large capillary at full size: 120 steps in the block storage with its autotuned
    kernel and tile, and in the FP32 storage with its own, give the same bits."""
    cap = W.config_binary_16384x256(STORAGE_F32_BLOCKED)
    blk = Lattice.from_workload(cap)
    blk.autotune()
    ref = Lattice.from_workload(cap, storage=STORAGE_F32)
    ref.autotune()
    for lat in (blk, ref):
        lat.step(120)
    assert blk.filled_length() == ref.filled_length()
    assert_same_state(blk, ref, cap.nx, cap.ny)
