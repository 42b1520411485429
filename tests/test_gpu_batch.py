"""Batched persistent kernel against independent lattices and the oracle (needs a GPU)."""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0911_0459_gb300 import (STORAGE_F16_BLOCKED, STORAGE_F16DEV, STORAGE_F32, STORAGE_F32_BLOCKED,  # noqa: E402
                                   STORAGE_F64,
                                   STORAGE_MOMENTS, Batch,
                                   Lattice, LbError)
from paper_0911_0459_gb300 import lb as lbmod  # noqa: E402


def small_sweep(seed=7, n=6, align=8, vary_gamma=False):
    """Uneven capillaries shaped like the sweep, shortened so the oracle keeps up."""
    caps = W.sweep(seed=seed, n=n, lengths=(96, 300), align=align, vary_gamma=vary_gamma)
    out = []
    for c in caps:
        c.nx = c.tube_x0 + c.tube_len   # keep the reservoirs, short tubes
        out.append(c)
    return out


@pytest.mark.parametrize("body", [1, 2, 3])
@pytest.mark.parametrize("storage", [STORAGE_F32, STORAGE_F32_BLOCKED, STORAGE_F64, STORAGE_F16DEV,
                                     STORAGE_F16_BLOCKED])
def test_batch_is_bitwise_identical_to_independent_lattices(storage, body):
    """Every body of the persistent kernel (sliding window; staged with the
    shallow and the deep ring) against one lattice per capillary, over tiles
    that change between launches and ragged last tiles and bands."""
    caps = small_sweep()
    b = Batch(caps, storage=storage)
    assert b.kernel() == 2   # every nx is a multiple of 8: staged by default
    b.set_kernel(body)
    assert b.kernel() == body
    for tx, ty in ((64, 4), (128, 16), (256, 64), (128, 5)):
        b.set_tile(tx, ty)
        b.step(13)
    total = b.time
    red = b.lengths()
    for i, c in enumerate(caps):
        lat = Lattice.from_workload(c, storage=storage)
        lat.step(total)
        fb, gb = b.populations(i, rested=False)
        fl, gl = lat.populations(rested=False)
        assert np.array_equal(fb, fl) and np.array_equal(gb, gl), i
        # the chunked batch reductions against the single-lattice ones: l from the
        # same centre-line values, sums in another order
        d = lat.filled_length()
        assert red[i, 0] == d["l"], i
        np.testing.assert_allclose(red[i, 1:], [d["l_vol"], d["mass"], d["phi_sum"]], rtol=1e-12,
                                   atol=1e-12 * c.nodes)
        lat.close()
    b.close()


def test_fp16_batch_with_a_different_free_energy_per_lattice():
    """FP16 deviations are taken from each lattice's own bulk rest weights (they depend on
    A): a sweep with A = kappa drawn per capillary evolves bit for bit as each alone."""
    caps = small_sweep(seed=8, n=5, vary_gamma=True)
    assert len({c.params.A for c in caps}) == len(caps)
    caps = [dataclasses.replace(c, params=dataclasses.replace(c.params, storage=STORAGE_F16DEV)) for c in caps]
    b = Batch(caps)
    b.step(37)
    for i, c in enumerate(caps):
        lat = Lattice.from_workload(c)
        lat.step(37)
        fb, gb = b.populations(i, rested=False)
        fl, gl = lat.populations(rested=False)
        assert np.array_equal(fb, fl) and np.array_equal(gb, gl), i
        lat.close()
    b.close()


@pytest.mark.parametrize("align", [8, 1])
def test_moment_storage_batch_is_bitwise_identical_to_independent_lattices(align):
    """The persistent moment body runs the single-lattice moment kernel's strips:
    every lattice evolves bit for bit as it does alone, over changing tiles,
    ragged strips and bands, and nx of any residue."""
    caps = small_sweep(seed=6, n=5, align=align)
    b = Batch(caps, storage=STORAGE_MOMENTS)
    assert b.kernel() == 4
    with pytest.raises(LbError):
        b.populations(0)
    for tx, ty in ((64, 4), (128, 20), (256, 7), (128, 64)):
        b.set_tile(tx, ty)
        b.step(11)
    total = b.time
    red = b.lengths()
    for i, c in enumerate(caps):
        lat = Lattice.from_workload(c, storage=STORAGE_MOMENTS)
        lat.step(total)
        assert np.array_equal(b.moments(i), lat.moments()), i
        d = lat.filled_length()
        assert red[i, 0] == d["l"], i
        np.testing.assert_allclose(red[i, 1:], [d["l_vol"], d["mass"], d["phi_sum"]], rtol=1e-12,
                                   atol=1e-12 * c.nodes)
        lat.close()
    tx, ty, ms = b.autotune(steps=2)
    assert tx in (64, 128, 256) and ms > 0
    b.close()


def test_batch_with_unaligned_rows_uses_the_sliding_window_body():
    caps = small_sweep(seed=9, n=4, align=1)
    assert any(c.nx % 8 for c in caps)
    b = Batch(caps)
    assert b.kernel() == 1
    with pytest.raises(LbError):
        b.set_kernel(2)
    b.step(9)
    for i, c in enumerate(caps):
        lat = Lattice.from_workload(c)
        lat.step(9)
        fb, gb = b.populations(i, rested=False)
        fl, gl = lat.populations(rested=False)
        assert np.array_equal(fb, fl) and np.array_equal(gb, gl), i
        lat.close()
    b.close()


@pytest.mark.parametrize("blocked,planar", [(STORAGE_F32_BLOCKED, STORAGE_F32), (STORAGE_F16_BLOCKED, STORAGE_F16DEV)])
@pytest.mark.parametrize("body", [1, 2, 3])
def test_block_storage_batch_with_unaligned_rows_equals_planar_lattices(body, blocked, planar):
    """The 32-node block storages stage whole blocks at any nx, so a batch of lattices
    whose rows start inside blocks runs the staged body too; every lattice equals its
    planar storage (FP32, or the FP16 deviations) run alone, bit for bit (the same
    arithmetic)."""
    caps = small_sweep(seed=9, n=4, align=1)
    assert any(c.nx % 32 for c in caps)
    b = Batch(caps, storage=blocked)
    assert b.kernel() == 2
    b.set_kernel(body)
    for tx, ty in ((64, 4), (128, 16), (256, 64), (128, 5)):
        b.set_tile(tx, ty)
        b.step(11)
    red = b.lengths()
    for i, c in enumerate(caps):
        lat = Lattice.from_workload(c, storage=planar)
        lat.step(b.time)
        fb, gb = b.populations(i, rested=False)
        fl, gl = lat.populations(rested=False)
        assert np.array_equal(fb, fl) and np.array_equal(gb, gl), i
        assert red[i, 0] == lat.filled_length()["l"], i
        lat.close()
    b.close()


def test_staged_body_long_run_matches_sliding_body():
    """Many steps in one persistent launch: the ring counter runs across
    hundreds of tiles and steps (and is renormalised) without drifting."""
    caps = small_sweep(seed=4, n=5)
    a = Batch(caps)
    b = Batch(caps)
    a.set_kernel(1)
    b.set_kernel(3)
    a.set_tile(64, 4)
    b.set_tile(64, 4)
    a.step(400)
    b.step(400)
    for i in range(len(caps)):
        fa, ga = a.populations(i, rested=False)
        fb, gb = b.populations(i, rested=False)
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), i
    np.testing.assert_array_equal(a.lengths(), b.lengths())
    a.close()
    b.close()


def test_batch_sampled_run_matches_oracle():
    caps = small_sweep(seed=3, n=4)
    b = Batch(caps, storage=STORAGE_F32)
    at = [1, 5, 40, 120, 300]
    out = b.run_sampled(at)
    assert out.shape == (4, 5, 4)
    for i, c in enumerate(caps):
        orc = oracle.Oracle(c)
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


@pytest.mark.parametrize("body", [1, 2])
def test_grid_barrier_timeout_is_reported_without_hanging(body):
    """Failure injection on the host: the barrier waits for an arrival that never
    comes, gives up after its short limit, and the host reads LB_ERR_TIMEOUT."""
    caps = small_sweep(seed=5, n=3)
    b = Batch(caps)
    b.set_kernel(body)
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


@pytest.mark.parametrize("storage", [STORAGE_F32, STORAGE_F32_BLOCKED, STORAGE_MOMENTS, STORAGE_F16_BLOCKED])
def test_full_sweep_of_256_capillaries_in_the_benchmarked_configuration(storage):
    """The seeded sweep at full size (256 capillaries, H 16..128, tubes 1024..8192,
    about 88 M fluid nodes), autotuned and run through sampled CUDA-graph launches as the
    benchmark times it.  Six capillaries (the smallest, the largest, four seeded picks)
    then equal the same capillary run alone bit for bit, with the same l(t) samples, and
    the smallest one matches the oracle."""
    caps = W.sweep(seed=0, n=256)
    b = Batch(caps, storage=storage)
    b.autotune(steps=2)
    t0 = b.time
    at = [10, 20, 30, 40]
    out = b.run_sampled(at)
    assert b.time == t0 + 40 and np.isfinite(out).all()
    sizes = [c.nx * c.ny for c in caps]
    rng = np.random.default_rng(1)
    picks = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), *rng.choice(len(caps), 4, replace=False)})
    for i in picks:
        lat = Lattice.from_workload(caps[i], storage=storage)
        lat.step(t0)
        for k, n in enumerate(at):
            lat.step(n - (at[k - 1] if k else 0))
            assert lat.filled_length()["l"] == out[i, k, 0], (i, k)
        if storage == STORAGE_MOMENTS:
            assert np.array_equal(b.moments(i), lat.moments()), i
        else:
            fb, gb = b.populations(i, rested=False)
            fl, gl = lat.populations(rested=False)
            assert np.array_equal(fb, fl) and np.array_equal(gb, gl), i
        if i == int(np.argmin(sizes)):
            orc = oracle.Oracle(caps[i]).init_default().step(b.time)
            g, o = lat.fields(), orc.fields()
            # FP16 deviations keep about 11 bits of each population
            tol = 5e-4 if storage == STORAGE_F16_BLOCKED else 1e-4
            assert max(np.abs(g[0] - o[0]).max(), np.abs(g[3] - o[3]).max()) < tol
            assert abs(lat.filled_length()["l"] - orc.filled_length()["l"]) < 0.05
        lat.close()
    b.close()
