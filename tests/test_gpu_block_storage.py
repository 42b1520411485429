"""Populations in 32-node blocks (LB_STORAGE_F32_BLOCKED, LB_STORAGE_F16_BLOCKED) through
the C ABI (needs a GPU).

A block storage keeps the values of its planar storage in another order and runs the same
arithmetic, so every result equals the planar storage's bit for bit: states after many
steps in every kernel variant and tile, through walls, the x-wrap and ragged last tiles,
the reductions and the fields, for rows that start on a block boundary (nx % 32 == 0) and
rows that do not (then a staged row is the whole blocks over its nodes, and the x-wrap
neighbour's block is staged apart).
  - FP32 blocks (values of LB_STORAGE_F32): f_i of node n at float
    576 (n // 32) + 64 i + 2 (n % 32), g_i the float after it.
  - FP16 blocks (values of LB_STORAGE_F16DEV): 1216-byte blocks, f_0 - w_0 at half
    608 (n // 32) + n % 32, f_i - w_i (i >= 1) at half 608 (n // 32) + 32 + 64 (i - 1)
    + 2 (n % 32), g_i the half after it, g_0 at float 304 (n // 32) + 272 + n % 32.
One step from a random state also matches the FP64 oracle within the planar storage's
tolerance per population (2e-6 for FP32, 1e-4 for FP16).
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0911_0459_gb300 import (STORAGE_F16_BLOCKED, STORAGE_F16DEV, STORAGE_F32,  # noqa: E402
                                   STORAGE_F32_BLOCKED, Lattice)

# precision -> (block storage, planar storage with the same values, one-step tolerance)
PREC = {"f32": (STORAGE_F32_BLOCKED, STORAGE_F32, 2e-6), "f16": (STORAGE_F16_BLOCKED, STORAGE_F16DEV, 1e-4)}

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


def to_planes(state, nx, ny, prec):
    """A block storage's saved state as its planar storage's bytes (f planes, g planes,
    then, for FP16, the FP32 g_0 plane)."""
    N = nx * ny
    nb = (N + 31) // 32
    raw = np.frombuffer(state.tobytes(), dtype=np.uint8)
    if prec == "f32":
        b = raw.view(np.uint32).reshape(nb, 9, 32, 2)          # block, i, node, (f, g)
        return np.ascontiguousarray(b.transpose(3, 1, 0, 2)).reshape(18, nb * 32)[:, :N].tobytes()
    blk = raw.reshape(nb, 1216)
    h = np.ascontiguousarray(blk[:, :1088]).view(np.uint16).reshape(nb, 544)
    pairs = h[:, 32:].reshape(nb, 8, 32, 2)                    # block, i - 1, node, (f, g)
    h17 = np.concatenate([h[:, None, :32], pairs[..., 0], pairs[..., 1]], axis=1)   # f_0..f_8, g_1..g_8
    g0 = np.ascontiguousarray(blk[:, 1088:]).view(np.uint32).reshape(nb * 32)[:N]
    planes = np.ascontiguousarray(h17.transpose(1, 0, 2)).reshape(17, nb * 32)[:, :N]
    return planes.tobytes() + g0.tobytes()


def assert_same_state(blk, ref, nx, ny, prec):
    a = np.frombuffer(to_planes(blk.save_state()[0], nx, ny, prec), dtype=np.uint8)
    b = np.frombuffer(ref.save_state()[0].tobytes(), dtype=np.uint8)
    assert a.size == b.size
    bad = np.flatnonzero(a != b)
    assert bad.size == 0, (bad.size, bad[:5])


def test_saved_state_follows_the_documented_layout():
    """lb_save_state of the FP32 blocks holds f_i of node n at float 576 (n // 32) + 64 i +
    2 (n % 32) and g_i in the float after it: read back against lb_get_populations.  That
    of the FP16 blocks holds, after the same steps, the planar FP16 storage's f_0 - w_0 at
    half 608 (n // 32) + n % 32, its f_i - w_i (i >= 1) at half 608 (n // 32) + 32 +
    64 (i - 1) + 2 (n % 32), its g_i in the half after that and its FP32 g_0 at float
    304 (n // 32) + 272 + n % 32."""
    cap = GEOMS["unaligned_ragged"](W.binary_params(nu_l=0.7, nu_g=0.05))
    N = cap.nx * cap.ny
    n = np.arange(N)
    lat = Lattice.from_workload(cap, storage=STORAGE_F32_BLOCKED)
    lat.step(37)
    f, g = lat.populations(rested=False)
    st = np.frombuffer(lat.save_state()[0].tobytes(), dtype=np.float32)
    assert st.size == 18 * 32 * ((N + 31) // 32)
    for i in range(9):
        assert np.array_equal(st[576 * (n // 32) + 64 * i + 2 * (n % 32)].astype(np.float64), f[i].ravel())
        assert np.array_equal(st[576 * (n // 32) + 64 * i + 2 * (n % 32) + 1].astype(np.float64), g[i].ravel())

    blk = Lattice.from_workload(cap, storage=STORAGE_F16_BLOCKED).step(37)
    ref = Lattice.from_workload(cap, storage=STORAGE_F16DEV).step(37)
    raw = blk.save_state()[0].tobytes()
    assert len(raw) == 1216 * ((N + 31) // 32)
    h = np.frombuffer(raw, dtype=np.uint16)
    s32 = np.frombuffer(raw, dtype=np.uint32)
    pr = ref.save_state()[0].tobytes()
    pf = np.frombuffer(pr[:18 * N], dtype=np.uint16).reshape(9, N)
    pg = np.frombuffer(pr[18 * N:34 * N], dtype=np.uint16).reshape(8, N)
    pg0 = np.frombuffer(pr[34 * N:], dtype=np.uint32)
    assert np.array_equal(h[608 * (n // 32) + n % 32], pf[0])
    for i in range(1, 9):
        assert np.array_equal(h[608 * (n // 32) + 32 + 64 * (i - 1) + 2 * (n % 32)], pf[i])
        assert np.array_equal(h[608 * (n // 32) + 32 + 64 * (i - 1) + 2 * (n % 32) + 1], pg[i - 1])
    assert np.array_equal(s32[304 * (n // 32) + 272 + n % 32], pg0)


@pytest.mark.parametrize("prec", sorted(PREC))
@pytest.mark.parametrize("geom", sorted(GEOMS))
def test_one_step_random_state_matches_oracle_and_planes(geom, prec):
    blocked, planar, tol = PREC[prec]
    cap = GEOMS[geom](W.binary_params(nu_l=0.7, nu_g=0.05, M=0.2))
    fields = W.random_state_fields(cap.nx, cap.ny, seed=11, model=W.BINARY)
    orc = oracle.Oracle(cap)
    orc.init_fields(*fields)
    orc.step(1)
    fo, go = orc.populations()
    ref = Lattice.from_workload(cap, storage=planar).init_fields(*fields).step(1)
    for variant, (tx, ty) in RUNS:
        lat = Lattice.from_workload(cap, storage=blocked)
        lat.set_kernel(variant)
        lat.set_tile(tx, min(ty, cap.ny))
        lat.init_fields(*fields)
        lat.step(1)
        f, g = lat.populations(rested=True)
        assert np.abs(f - fo).max() < tol and np.abs(g - go).max() < tol, (variant, tx, ty)
        assert_same_state(lat, ref, cap.nx, cap.ny, prec)
        lat.close()


@pytest.mark.parametrize("prec", sorted(PREC))
@pytest.mark.parametrize("geom", sorted(GEOMS))
def test_many_steps_bitwise_equal_to_planes(geom, prec):
    """300 steps from the default state (a meniscus moving along the tube), with the
    l(t) reductions every 100 steps: every bit equal to the planar storage's run (state,
    reductions, fields and exported moments)."""
    blocked, planar, _ = PREC[prec]
    cap = GEOMS[geom](W.binary_params(nu_l=0.83, nu_g=0.083))
    ref = Lattice.from_workload(cap, storage=planar)
    ls_ref = []
    for _ in range(3):
        ref.step(100)
        ls_ref.append(ref.filled_length())
    rf = ref.fields()
    rm = ref.moments()
    for variant, (tx, ty) in RUNS:
        lat = Lattice.from_workload(cap, storage=blocked)
        lat.set_kernel(variant)
        lat.set_tile(tx, min(ty, cap.ny))
        ls = []
        for _ in range(3):
            lat.step(100)
            ls.append(lat.filled_length())
        assert ls == ls_ref, (variant, tx, ty)
        assert_same_state(lat, ref, cap.nx, cap.ny, prec)
        for a, b in zip(lat.fields(), rf):
            assert np.array_equal(a, b)
        assert np.array_equal(lat.moments(), rm)
        lat.close()


@pytest.mark.parametrize("prec", sorted(PREC))
def test_populations_and_checkpoint_round_trip(prec):
    blocked = PREC[prec][0]
    cap = GEOMS["tube_wraps_x"](W.binary_params(nu_l=0.5, nu_g=0.05))
    lat = Lattice.from_workload(cap, storage=blocked)
    lat.step(50)
    buf, t = lat.save_state()
    f, g = lat.populations(rested=False)
    lat.step(30)
    after = lat.save_state()[0].copy()
    # resume from the checkpoint: the same 30 steps give the same bits
    lat.load_state(buf, t)
    lat.step(30)
    assert np.array_equal(lat.save_state()[0], after)
    # populations written back: FP32 values return exactly; in either precision they
    # give the planar storage's state from the same populations
    other = Lattice.from_workload(cap, storage=blocked)
    other.set_populations(f, g)
    if prec == "f32":
        assert np.array_equal(other.save_state()[0], buf)
    ref = Lattice.from_workload(cap, storage=PREC[prec][1])
    ref.set_populations(f, g)
    assert_same_state(other, ref, cap.nx, cap.ny, prec)


@pytest.mark.parametrize("prec", sorted(PREC))
def test_full_size_16384x256_bitwise_equal_to_planes(prec):
    """The large capillary at full size: 120 steps in the block storage with its autotuned
    kernel and tile, and in the planar storage with its own, give the same bits."""
    blocked, planar, _ = PREC[prec]
    cap = W.config_binary_16384x256(blocked)
    blk = Lattice.from_workload(cap)
    blk.autotune()
    ref = Lattice.from_workload(cap, storage=planar)
    ref.autotune()
    for lat in (blk, ref):
        lat.step(120)
    assert blk.filled_length() == ref.filled_length()
    assert_same_state(blk, ref, cap.nx, cap.ny, prec)
