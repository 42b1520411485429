"""Moment storage (six FP32 numbers per node) against the FP64 oracle, through the C ABI.

The oracle keeps populations.  Its moments are taken here from their plain
definitions (sums over the velocity set of Sec. 2.1).  By the oracle pin
test_one_lattice_step_depends_only_on_the_hydrodynamic_moments, any populations
with the same six moments give the same next state.  So a GPU moment state is
handed to the oracle as the populations with those moments and the remaining
modes at zero.

Tolerances (per node, absolute) are those of the FP32 population storage:
2e-6 after one step from the same state; 1e-4 for rho and phi and 0.05 lattice
units for l after 2000 steps.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0911_0459_gb300 import Lattice, LbError, STORAGE_F32, STORAGE_MOMENTS  # noqa: E402

# Velocity set of Sec. 2.1 and the moment rows stored per node.
E = np.array([(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (-1, 1), (1, -1)], float)
EX, EY = E[:, 0], E[:, 1]
ROWS = np.array([np.ones(9), EX, EY, EX ** 2 - EY ** 2, EX * EY])   # rho, jx, jy, pxx - pyy, pxy


def moments_of(f, g):
    """(6, ny, nx) moments of population arrays (9, ny, nx)."""
    m = np.einsum("ki,iyx->kyx", ROWS, f)
    return np.concatenate([m, g.sum(axis=0)[None]], axis=0)


def populations_with(m):
    """Populations whose six moments are m and whose e, eps, qx, qy modes vanish
    (g carries phi in g_0)."""
    ex2, ey2 = EX ** 2, EY ** 2
    e2 = ex2 + ey2
    B = np.array([np.ones(9), -4 + 3 * e2, 4 - 10.5 * e2 + 4.5 * e2 ** 2, EX, (-5 + 3 * e2) * EX,
                  EY, (-5 + 3 * e2) * EY, ex2 - ey2, EX * EY])
    full = np.zeros((9,) + m.shape[1:])
    full[0], full[3], full[5], full[7], full[8] = m[0], m[1], m[2], m[3], m[4]
    f = np.einsum("ik,kyx->iyx", np.linalg.inv(B), full)
    g = np.zeros_like(f)
    g[0] = m[5]
    return f, g


def rested(m, kinds):
    """The rest rule of Sec. 2.2 applied to stored moments: j = 0 at boundary nodes."""
    m = m.copy()
    m[1:3, kinds == 1] = 0.0
    return m


def maxdiff(a, b, mask):
    return float(np.abs(a - b)[:, mask].max())


GEOMS = {
    "capillary_ragged": lambda p: W.Capillary("cr", 203, 37, 61, 120, 5, 27, 12, 8, p, wall_grad=-0.11),
    "thin_wall": lambda p: W.Capillary("tw", 150, 21, 40, 100, 0, 20, 10, 6, p, wall_grad=-0.2),
    "channel": lambda p: W.channel(131, 19, 15, p, wall_grad=-0.15),
    "periodic": lambda p: W.periodic_box(77, 29, p),
    "tube_wraps_x": lambda p: W.Capillary("wx", 140, 30, 100, 90, 27, 20, 0, 0, p, wall_grad=-0.1),
    # narrower than one warp, and the fewest rows a tube allows
    "narrow": lambda p: W.Capillary("nw", 20, 12, 6, 10, 2, 7, 2, 3, p, wall_grad=-0.2),
    "three_rows": lambda p: W.Capillary("tr", 45, 3, 10, 25, 0, 2, 4, 5, p, wall_grad=-0.1),
}
TILES = ((64, 1), (128, 5), (256, 16), (64, 1000))


def pair(cap, fields):
    lat = Lattice.from_workload(cap, storage=STORAGE_MOMENTS)
    orc = oracle.Oracle(cap)
    lat.init_fields(*fields)
    orc.init_fields(*fields)
    return lat, orc


@pytest.mark.parametrize("geom", sorted(GEOMS))
def test_one_step_from_random_state_matches_oracle(geom):
    cap = GEOMS[geom](W.binary_params(nu_l=0.7, nu_g=0.05, M=0.2))
    fields = W.random_state_fields(cap.nx, cap.ny, seed=11, model=W.BINARY)
    lat, orc = pair(cap, fields)
    kinds = orc.node_kinds()
    fluid = kinds != 2
    m0 = rested(lat.moments(), kinds)
    assert maxdiff(m0, moments_of(*orc.populations()), fluid) < 2e-6
    orc.step(1)
    want = moments_of(*orc.populations())
    results = []
    for tx, ty in TILES:
        lat.init_fields(*fields)
        lat.set_tile(tx, min(ty, cap.ny))
        lat.step(1)
        m1 = lat.moments()
        assert maxdiff(rested(m1, kinds), want, fluid) < 2e-6, (tx, ty)
        results.append(m1)
    # every node sums its arrivals in one fixed order: the tile does not matter
    for m in results[1:]:
        assert np.array_equal(m, results[0])


@pytest.mark.parametrize("geom", ["capillary_ragged", "tube_wraps_x", "narrow"])
def test_gpu_state_advanced_by_oracle_matches_gpu_step(geom):
    """After 150 GPU steps the oracle takes the GPU's state (as populations with its
    moments) and both advance one step."""
    cap = GEOMS[geom](W.binary_params(nu_l=0.5, nu_g=0.02, M=0.1))
    fields = W.random_state_fields(cap.nx, cap.ny, seed=4, model=W.BINARY)
    lat, orc = pair(cap, fields)
    lat.step(150)
    f, g = populations_with(lat.moments())
    orc.set_populations(f, g, apply_rest=True)
    kinds = orc.node_kinds()
    lat.step(1)
    orc.step(1)
    assert maxdiff(rested(lat.moments(), kinds), moments_of(*orc.populations()), kinds != 2) < 2e-6


def test_2000_steps_of_a_filling_capillary_stay_within_the_method_tolerance():
    cap = W.Capillary("f", 300, 30, 60, 230, 4, 22, 20, 10, W.binary_params(nu_l=0.5, nu_g=0.05),
                      theta_deg=45.0)
    lat = Lattice.from_workload(cap, storage=STORAGE_MOMENTS)
    orc = oracle.Oracle(cap)
    orc.init_default()
    lat.step(2000)
    orc.step(2000)
    rg, _, _, pg = lat.fields()
    ro, _, _, po = orc.fields()
    assert np.abs(rg - ro).max() < 1e-4 and np.abs(pg - po).max() < 1e-4
    d, do = lat.filled_length(), orc.filled_length()
    assert abs(d["l"] - do["l"]) < 0.05
    assert abs(d["mass"] / do["mass"] - 1) < 1e-6


def test_close_to_the_fp32_population_storage():
    cap = W.Capillary("c", 256, 40, 64, 160, 6, 28, 16, 12, W.binary_params(nu_l=0.83, nu_g=0.0166),
                      theta_deg=45.0)
    a = Lattice.from_workload(cap, storage=STORAGE_F32)
    b = Lattice.from_workload(cap, storage=STORAGE_MOMENTS)
    a.step(500)
    b.step(500)
    fluid = np.ones((cap.ny, cap.nx), bool)
    ma, mb = a.moments(), b.moments()
    assert maxdiff(ma, mb, fluid) < 2e-5
    assert abs(a.filled_length()["l"] - b.filled_length()["l"]) < 1e-3


def test_full_size_16384x256_one_step_from_gpu_state():
    """The large capillary at full size: 200 GPU steps in the autotuned launch
    configuration, then one step of the oracle from the GPU's state against the
    GPU's next step, at every node."""
    cap = W.config_binary_16384x256(STORAGE_MOMENTS)
    lat = Lattice.from_workload(cap)
    lat.autotune()
    lat.step(200)
    f, g = populations_with(lat.moments())
    orc = oracle.Oracle(cap)
    orc.set_populations(f, g, apply_rest=True)
    del f, g
    kinds = orc.node_kinds()
    lat.step(1)
    orc.step(1)
    assert maxdiff(rested(lat.moments(), kinds), moments_of(*orc.populations()), kinds != 2) < 2e-6
    d, do = lat.filled_length(), orc.filled_length()
    assert abs(d["l"] - do["l"]) < 1e-3 and abs(d["mass"] / do["mass"] - 1) < 1e-7


def test_mass_is_conserved_to_fp32_rounding():
    cap = W.Capillary("m", 256, 40, 64, 160, 6, 28, 16, 12, W.binary_params(nu_l=0.83, nu_g=0.0166),
                      theta_deg=30.0)
    lat = Lattice.from_workload(cap, storage=STORAGE_MOMENTS)
    d0 = lat.filled_length()
    lat.step(3000)
    d1 = lat.filled_length()
    assert abs(d1["mass"] / d0["mass"] - 1) < 1e-6
    assert abs(d1["phi_sum"] - d0["phi_sum"]) < 1e-6 * lat.fluid_nodes
    assert d1["l"] > d0["l"]   # the liquid advances into the tube


def test_interface_of_the_moment_storage():
    cap = GEOMS["capillary_ragged"](W.binary_params())
    lat = Lattice.from_workload(cap, storage=STORAGE_MOMENTS)
    assert lat.kernel() == 4
    lat.set_kernel(0)
    for v in (1, 2, 3):
        with pytest.raises(LbError):
            lat.set_kernel(v)
    with pytest.raises(LbError):
        lat.populations()
    # populations in: their moments are stored (FP32)
    rng = np.random.default_rng(2)
    f = rng.uniform(0.0, 0.3, (9, cap.ny, cap.nx))
    g = rng.uniform(-0.1, 0.1, (9, cap.ny, cap.nx))
    lat.set_populations(f, g)
    kinds = oracle.Oracle(cap).node_kinds()
    fluid = kinds != 2
    m = lat.moments()
    np.testing.assert_allclose(m[:, fluid], moments_of(f, g)[:, fluid], rtol=1e-6, atol=1e-7)
    assert np.all(m[:, ~fluid] == 0)
    # fields: rho and phi as stored, u = j / rho away from walls and 0 at boundary nodes
    rho, ux, uy, phi = lat.fields()
    np.testing.assert_array_equal(rho[fluid], m[0][fluid])
    inner = kinds == 0
    np.testing.assert_allclose(ux[inner], (m[1] / m[0])[inner], rtol=1e-6)
    assert np.all(ux[kinds == 1] == 0) and np.all(uy[kinds == 1] == 0)
    tx, ty, us = lat.autotune()
    assert tx in (64, 128, 256) and us > 0
