"""CUDA path vs the FP64 oracle, through the C ABI (needs a GB300).

Tolerances (per node, absolute):
  FP64 storage  : 1e-11 after one step, 1e-9 after 2000 steps (same arithmetic,
                  different summation order and collision formulation);
  FP32 storage  : 2e-6 after one step; the method's bar of 1e-4 for rho and phi
                  after 2000 steps and 0.05 lattice units for l(t);
  FP16 deviation: 1e-4 after one step (FP16 keeps ~11 bits of each stored
                  deviation from the bulk rest populations, which are below
                  ~2e-2); after 2000 steps 2e-3 for rho and phi and the method's
                  0.05 lattice units for l(t).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0911_0459_gb300 import (Lattice, LbError, STORAGE_F16DEV, STORAGE_F32,  # noqa: E402
                                   STORAGE_F64, STORAGE_MOMENTS)
from paper_0911_0459_gb300 import lb as lbmod  # noqa: E402

STEP_TOL = {STORAGE_F64: 1e-11, STORAGE_F32: 2e-6, STORAGE_F16DEV: 1e-4}


def pair(cap, storage=None, fields=None):
    lat = Lattice.from_workload(cap, storage=storage)
    orc = oracle.Oracle(cap)
    if fields is None:
        orc.init_default()
    else:
        lat.init_fields(*fields)
        orc.init_fields(*fields)
    return lat, orc


def maxdiff(a, b, mask=None):
    d = np.abs(np.asarray(a) - np.asarray(b))
    return float(d[mask].max() if mask is not None else d.max())


GEOMS = {
    # ragged in x (nx not a multiple of any tile width) and in y
    "capillary_ragged": lambda p: W.Capillary("cr", 203, 37, 61, 120, 5, 27, 12, 8, p, wall_grad=-0.11),
    "thin_wall": lambda p: W.Capillary("tw", 150, 21, 40, 100, 0, 20, 10, 6, p, wall_grad=-0.2),
    "channel": lambda p: W.channel(131, 19, 15, p, wall_grad=-0.15),
    "periodic": lambda p: W.periodic_box(77, 29, p),
    "tube_wraps_x": lambda p: W.Capillary("wx", 140, 30, 100, 90, 27, 20, 0, 0, p, wall_grad=-0.1),
    # nx % 8 == 0: these run the staged (bulk-copy) kernel; ragged last tile in x and y
    "staged_capillary": lambda p: W.Capillary("sc", 200, 37, 64, 120, 5, 27, 12, 8, p, wall_grad=-0.11),
    "staged_tube_wraps": lambda p: W.Capillary("sw", 144, 30, 104, 90, 27, 20, 0, 0, p, wall_grad=-0.1),
    # narrower than one warp, and the fewest rows a tube allows (one solid row)
    "narrow": lambda p: W.Capillary("nw", 20, 12, 6, 10, 2, 7, 2, 3, p, wall_grad=-0.2),
    "three_rows": lambda p: W.Capillary("tr", 45, 3, 10, 25, 0, 2, 4, 5, p, wall_grad=-0.1),
    "staged_narrow": lambda p: W.Capillary("sn", 24, 10, 4, 16, 1, 6, 2, 3, p, wall_grad=-0.15),
}


@pytest.mark.parametrize("geom", sorted(GEOMS))
@pytest.mark.parametrize("storage", [STORAGE_F64, STORAGE_F32, STORAGE_F16DEV])
def test_one_step_binary_random_state(geom, storage):
    cap = GEOMS[geom](W.binary_params(nu_l=0.7, nu_g=0.05, M=0.2))
    f = W.random_state_fields(cap.nx, cap.ny, seed=11, model=W.BINARY)
    lat, orc = pair(cap, storage, f)
    fg0, gg0 = lat.populations()
    fo0, go0 = orc.populations()
    assert maxdiff(fg0, fo0) < STEP_TOL[storage] and maxdiff(gg0, go0) < STEP_TOL[storage]
    lat.step(1)
    orc.step(1)
    fg, gg = lat.populations(rested=True)
    fo, go = orc.populations()
    assert maxdiff(fg, fo) < STEP_TOL[storage], maxdiff(fg, fo)
    assert maxdiff(gg, go) < STEP_TOL[storage], maxdiff(gg, go)


@pytest.mark.parametrize("geom", sorted(GEOMS))
@pytest.mark.parametrize("storage", [STORAGE_F64, STORAGE_F32])
def test_one_step_liquid_gas_random_state(geom, storage):
    cap = GEOMS[geom](W.lg_params())
    f = W.random_state_fields(cap.nx, cap.ny, seed=5, model=W.LG)
    lat, orc = pair(cap, storage, f)
    lat.step(1)
    orc.step(1)
    fg, _ = lat.populations(rested=True)
    fo, _ = orc.populations()
    tol = STEP_TOL[storage] * (8 if storage == STORAGE_F32 else 1)   # rho ~ 4: 4x larger ulps
    assert maxdiff(fg, fo) < tol, maxdiff(fg, fo)


@pytest.mark.parametrize("storage,variant", [(STORAGE_F32, 1), (STORAGE_F32, 2), (STORAGE_MOMENTS, 0)])
def test_more_row_bands_than_a_two_dimensional_grid_holds(storage, variant):
    """A tall periodic box, 8 x 65600, at one-row bands: 65600 bands, more than a grid's
    y dimension takes (65535).  One step from a random state against the oracle at every
    node, for the sliding-window, staged and moment kernels."""
    cap = W.periodic_box(8, 65600, W.binary_params(nu_l=0.4, nu_g=0.05, M=0.2))
    f = W.random_state_fields(cap.nx, cap.ny, seed=23, model=W.BINARY)
    lat, orc = pair(cap, storage, f)
    if variant:
        lat.set_kernel(variant)
    lat.set_tile(64, 1)
    lat.step(1)
    orc.step(1)
    g, o = lat.fields(), orc.fields()
    for k in range(4):
        assert maxdiff(g[k], o[k]) < 2e-6, (k, maxdiff(g[k], o[k]))


def test_default_initial_state_matches_workload_fields():
    for cap in (W.config_lg_256x32(), W.Capillary("b", 200, 30, 50, 120, 4, 22, 16, 10,
                                                  W.binary_params(), theta_deg=50.0)):
        lat = Lattice.from_workload(cap)
        orc = oracle.Oracle(cap).init_default()
        fg, gg = lat.populations()
        fo, go = orc.populations()
        tol = 1e-12 if cap.params.storage == STORAGE_F64 else 2e-7
        assert maxdiff(fg, fo) < tol
        if gg is not None:
            assert maxdiff(gg, go) < tol


def run_both(cap, steps, storage=None, every=None):
    lat, orc = pair(cap, storage)
    ls = []
    done = 0
    every = every or steps
    while done < steps:
        n = min(every, steps - done)
        lat.step(n)
        orc.step(n)
        done += n
        ls.append((lat.filled_length(), orc.filled_length()))
    return lat, orc, ls


def test_liquid_gas_256x32_fp64_2000_steps():
    """Liquid-gas capillary, FP64, 2000 steps, l(t) every 50 steps."""
    cap = W.config_lg_256x32()
    lat, orc, ls = run_both(cap, 2000, every=50)
    rho, ux, uy, _ = lat.fields()
    r_rho, r_ux, r_uy, _ = orc.fields()
    assert maxdiff(rho, r_rho) < 1e-9 and maxdiff(ux, r_ux) < 1e-10 and maxdiff(uy, r_uy) < 1e-10
    for g, o in ls:
        assert abs(g["l"] - o["l"]) < 1e-8 and abs(g["mass"] / o["mass"] - 1) < 1e-13


@pytest.mark.parametrize("storage", [STORAGE_F32, STORAGE_F64])
def test_binary_capillary_2000_steps(storage):
    """Binary capillary 256 x 40, viscosity ratio 10, 60 degrees: the 1e-4 / 0.05 bar."""
    cap = W.Capillary("b2k", 256, 40, 48, 208, 4, 32, 16, 10,
                      W.binary_params(nu_l=0.83, nu_g=0.083), theta_deg=60.0)
    lat, orc, ls = run_both(cap, 2000, storage, every=250)
    rho, ux, uy, phi = lat.fields()
    r_rho, r_ux, r_uy, r_phi = orc.fields()
    tol = 1e-4 if storage == STORAGE_F32 else 1e-10
    assert maxdiff(rho, r_rho) < tol and maxdiff(phi, r_phi) < tol
    for g, o in ls:
        assert abs(g["l"] - o["l"]) < (0.05 if storage == STORAGE_F32 else 1e-8)
        assert abs(g["l_vol"] - o["l_vol"]) < (0.05 if storage == STORAGE_F32 else 1e-8)
    assert ls[-1][1]["l"] > ls[0][1]["l"]   # the meniscus advanced


@pytest.mark.slow
def test_binary_crop_1024x64_2000_steps():
    """1024 x 64 crop of the large capillary (H = 50, ratio 50, 45 degrees), FP32, 2000 steps."""
    cap = W.config_binary_crop_1024x64()
    lat, orc, ls = run_both(cap, 2000, every=1000)
    rho, ux, uy, phi = lat.fields()
    r_rho, r_ux, r_uy, r_phi = orc.fields()
    assert maxdiff(rho, r_rho) < 1e-4 and maxdiff(phi, r_phi) < 1e-4
    for g, o in ls:
        assert abs(g["l"] - o["l"]) < 0.05


def test_fp16_deviation_storage_error_is_bounded():
    cap = W.Capillary("h", 256, 40, 48, 208, 4, 32, 16, 10, W.binary_params(nu_l=0.83, nu_g=0.083),
                      theta_deg=60.0)
    lat, orc, ls = run_both(cap, 2000, STORAGE_F16DEV, every=500)
    rho, _, _, phi = lat.fields()
    r_rho, _, _, r_phi = orc.fields()
    err = max(maxdiff(rho, r_rho), maxdiff(phi, r_phi))
    print(f"FP16-deviation storage: max |d rho|, |d phi| after 2000 steps = {err:.3e}")
    assert err < 2e-3
    for g, o in ls:
        assert abs(g["l"] - o["l"]) < 0.05


@pytest.mark.parametrize("storage", [STORAGE_F32, STORAGE_F16DEV])
def test_full_size_16384x256_one_step_from_gpu_state(storage):
    """The large capillary at full size in the benchmark's launch configuration: after 200
    GPU steps, the oracle advances the GPU's own state by one step and every node of the
    next GPU step is compared (FP64 oracle on the FP32/FP16 state)."""
    cap = W.config_binary_16384x256(storage)
    lat = Lattice.from_workload(cap)
    lat.autotune()
    lat.step(200)
    f0, g0 = lat.populations(rested=False)
    orc = oracle.Oracle(cap)
    orc.set_populations(f0, g0, apply_rest=True)
    del f0, g0
    lat.step(1)
    orc.step(1)
    fg, gg = lat.populations(rested=True)
    fo, go = orc.populations()
    tol = 2e-6 if storage == STORAGE_F32 else 1e-4
    assert maxdiff(fg, fo) < tol and maxdiff(gg, go) < tol
    d, do = lat.filled_length(), orc.filled_length()
    # total mass over 3.3 M nodes: FP32 (FP16) rounding of each node's populations
    mtol = 1e-7 if storage == STORAGE_F32 else 1e-5
    assert abs(d["l"] - do["l"]) < 1e-3 and abs(d["mass"] / do["mass"] - 1) < mtol


def test_reductions_match_oracle_and_conserve_mass():
    cap = W.Capillary("r", 300, 30, 60, 230, 4, 22, 20, 10, W.binary_params(nu_l=0.5, nu_g=0.05),
                      theta_deg=45.0)
    lat, orc, ls = run_both(cap, 600, STORAGE_F64, every=200)
    for g, o in ls:
        for k in ("l", "l_vol", "mass", "phi_sum"):
            assert abs(g[k] - o[k]) < 1e-8 * max(1.0, abs(o[k])), (k, g[k], o[k])
    assert abs(ls[-1][0]["mass"] / ls[0][0]["mass"] - 1) < 1e-13


def test_step_split_and_graph_replay_are_bitwise_identical():
    cap = W.Capillary("s", 180, 28, 40, 120, 3, 22, 12, 8, W.binary_params(nu_l=0.5, nu_g=0.05),
                      theta_deg=60.0)
    a = Lattice.from_workload(cap)
    b = Lattice.from_workload(cap)
    a.step(150)                       # graph replays (64-step chunks) plus single launches
    for n in (1, 2, 61, 7, 79):       # odd splits: parity handling
        b.step(n)
    fa, ga = a.populations(rested=False)
    fb, gb = b.populations(rested=False)
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    # checkpoint / resume through the raw populations
    c = Lattice.from_workload(cap)
    c.set_populations(fa, ga)
    a.step(40)
    c.step(40)
    assert np.array_equal(a.populations(False)[0], c.populations(False)[0])


def test_tile_shapes_are_bitwise_identical_and_autotune_restores_state():
    cap = W.Capillary("t", 333, 45, 70, 230, 5, 35, 20, 10, W.binary_params(nu_l=0.5, nu_g=0.05),
                      theta_deg=60.0)
    ref = None
    for tx, ty in ((64, 1), (128, 7), (256, 16), (128, 45)):
        lat = Lattice.from_workload(cap)
        lat.set_tile(tx, ty)
        lat.step(30)
        f, g = lat.populations(False)
        if ref is None:
            ref = (f, g)
        else:
            assert np.array_equal(f, ref[0]) and np.array_equal(g, ref[1]), (tx, ty)
    lat = Lattice.from_workload(cap)
    lat.step(10)
    before = lat.populations(False)
    tx, ty, us = lat.autotune()
    after = lat.populations(False)
    assert np.array_equal(before[0], after[0]) and us > 0 and lat.tile() == (tx, ty)


def test_nonfinite_state_is_detected_and_poisons_the_context():
    cap = W.Capillary("n", 64, 20, 16, 40, 2, 16, 8, 6, W.binary_params(), theta_deg=60.0)
    lat = Lattice.from_workload(cap)
    f, g = lat.populations(False)
    f0, g0 = f.copy(), g.copy()
    f[3, 10, 5] = np.nan
    lat.set_populations(f, g)
    lat.step(2)
    with pytest.raises(LbError) as e:
        lat.filled_length()
    assert e.value.status == lbmod.LB_ERR_NONFINITE
    with pytest.raises(LbError) as e:
        lat.step(1)
    assert e.value.status == lbmod.LB_ERR_STATE
    lat.fields()   # still readable
    # replacing the state clears the condition: the lattice steps again from it
    lat.set_populations(f0, g0)
    lat.step(3)
    d = lat.filled_length()
    assert np.isfinite(d["mass"]) and np.isfinite(d["l"])


def test_invalid_arguments_are_rejected():
    p = W.binary_params()
    with pytest.raises(LbError) as e:
        Lattice(64, 20, model=1, storage=1, tube_x0=0, tube_len=63, tube_y0=0, tube_h=10)
    assert e.value.status == lbmod.LB_ERR_ARG
    with pytest.raises(LbError):
        Lattice(64, 20, model=1, storage=1, tube_x0=0, tube_len=30, tube_y0=0, tube_h=1)
    with pytest.raises(LbError):
        Lattice(64, 20, model=0, storage=2)
    lat = Lattice(64, 20, model=1, storage=1, A=p.A, kappa=p.kappa)
    with pytest.raises(LbError):
        lat.set_tile(96, 4)
    with pytest.raises(LbError):
        lat.step(-1)


STAGED = [("binary", STORAGE_F64), ("binary", STORAGE_F32), ("binary", STORAGE_F16DEV),
          ("lg", STORAGE_F64), ("lg", STORAGE_F32)]


@pytest.mark.parametrize("model,storage", STAGED)
def test_staged_kernel_is_bitwise_identical_to_sliding_window(model, storage):
    """Both step kernels compute the same update bit for bit, on every tile shape,
    including ragged last tiles, the x-wrap of the tube and single-tile rows."""
    p = W.binary_params(nu_l=0.6, nu_g=0.06) if model == "binary" else W.lg_params()
    caps = [W.Capillary("a", 328, 45, 70, 230, 5, 35, 20, 10, p, wall_grad=-0.12),
            W.Capillary("b", 136, 23, 96, 80, 20, 15, 0, 0, p, wall_grad=-0.2),
            W.periodic_box(64, 20, p)]
    for cap in caps:
        fields = W.random_state_fields(cap.nx, cap.ny, seed=3, model=cap.params.model)
        for tx, ty in ((64, 1), (128, 5), (256, 16), (64, cap.ny)):
            a = Lattice.from_workload(cap, storage=storage).init_fields(*fields)
            a.set_kernel(1)
            a.set_tile(tx, ty)
            a.step(7)
            fa, ga = a.populations(False)
            for variant in (2, 3):   # shallow and deep ring of row stages
                b = Lattice.from_workload(cap, storage=storage).init_fields(*fields)
                b.set_kernel(variant)
                assert b.kernel() == variant
                b.set_tile(tx, ty)
                b.step(7)
                fb, gb = b.populations(False)
                assert np.array_equal(fa, fb), (cap.name, tx, ty, variant)
                if ga is not None:
                    assert np.array_equal(ga, gb), (cap.name, tx, ty, variant)
                b.sync()   # no device-side wait gave up
                b.close()
            a.close()


def test_staged_kernel_rejected_when_rows_are_not_16_byte_aligned():
    lat = Lattice(100, 20, model=1, storage=1)
    with pytest.raises(LbError):
        lat.set_kernel(2)
    lat.set_kernel(1)
    lat.step(3)
