"""The two further reduced states of the binary model against the FP64 oracle, through
the C ABI (needs a GPU):

- LB_STORAGE_F32_GELIM: the nine f populations in FP32 and phi in place of the nine g
  populations ("g eliminated", 80 bytes per node update).  Every g mode relaxes fully
  to g^eq (App. A, Eq. (latbolt2)), so a step depends on g only through phi.
- LB_STORAGE_MOMENTS_F16: the six moments with rho - 1, j and the two stresses in FP16
  and phi in FP32 (28 bytes per node update), FP32 arithmetic.

As in test_gpu_moments.py the oracle is handed a GPU state as populations with the
GPU's moments (any populations with the same six moments give the same next state, by
the oracle pin test_one_lattice_step_depends_only_on_the_hydrodynamic_moments).
Tolerances: the FP32 population storage's (2e-6 per node after one step; 1e-4 for rho
and phi and 0.05 for l after 2000 steps) for g elimination.  For the FP16 moments a
node's stored moment is rounded to FP16 once per step: one step is held to that
rounding (2^-11 of the moment's size, which for rho is rho - 1) plus the FP32 bound;
after 2000 steps l stays within the method's 0.05, rho and phi within the bound
written in the test (measured, with a margin).
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0911_0459_gb300 import (STORAGE_F32, STORAGE_F32_GELIM, STORAGE_MOMENTS,  # noqa: E402
                                   STORAGE_MOMENTS_F16, Lattice, LbError)
from test_gpu_moments import GEOMS, maxdiff, moments_of, populations_with, rested  # noqa: E402

STORAGES = {"gelim": STORAGE_F32_GELIM, "moments_f16": STORAGE_MOMENTS_F16}


def one_step_tolerance(storage, m):
    """Per-node bound on |GPU - oracle| for the six moments m (6, ny, nx) after one step."""
    if storage == STORAGE_F32_GELIM:
        return 2e-6
    dev = np.abs(m).copy()
    dev[0] = np.abs(m[0] - 1.0)           # rho is stored as rho - 1
    tol = 2e-6 + dev * 2.0 ** -11
    tol[5] = 2e-6                          # phi stays FP32
    return tol


def check_step(lat, orc, kinds, storage):
    """Hand the GPU's state to the oracle, advance both one step, compare every fluid node."""
    m0 = lat.moments()
    f, g = populations_with(m0)
    orc.set_populations(f, g, apply_rest=True)
    lat.step(1)
    orc.step(1)
    got, want = rested(lat.moments(), kinds), moments_of(*orc.populations())
    fluid = kinds != 2
    tol = one_step_tolerance(storage, want)
    excess = np.abs(got - want) - tol
    assert float(excess[:, fluid].max()) <= 0.0, float(np.abs(got - want)[:, fluid].max())
    return got


@pytest.mark.parametrize("storage", sorted(STORAGES))
@pytest.mark.parametrize("geom", sorted(GEOMS))
def test_one_step_matches_oracle(storage, geom):
    st = STORAGES[storage]
    cap = GEOMS[geom](W.binary_params(nu_l=0.7, nu_g=0.05, M=0.2))
    fields = W.random_state_fields(cap.nx, cap.ny, seed=11, model=W.BINARY)
    lat = Lattice.from_workload(cap, storage=st)
    orc = oracle.Oracle(cap)
    kinds = orc.node_kinds()
    results = []
    for tx, ty in ((64, 1), (128, 5), (256, 16), (64, 1000)):
        lat.init_fields(*fields)
        lat.set_tile(tx, min(ty, cap.ny))
        results.append(check_step(lat, orc, kinds, st))
    for m in results[1:]:                  # the tile does not change a bit
        assert np.array_equal(m, results[0])


@pytest.mark.parametrize("storage", sorted(STORAGES))
def test_after_150_steps_one_more_step_matches_oracle(storage):
    st = STORAGES[storage]
    cap = GEOMS["capillary_ragged"](W.binary_params(nu_l=0.5, nu_g=0.02, M=0.1))
    lat = Lattice.from_workload(cap, storage=st)
    lat.init_fields(*W.random_state_fields(cap.nx, cap.ny, seed=4, model=W.BINARY))
    lat.step(150)
    orc = oracle.Oracle(cap)
    check_step(lat, orc, orc.node_kinds(), st)


# after 2000 steps of the filling capillary: (max |d rho|, max |d phi|) allowed
BOUND_2000 = {STORAGE_F32_GELIM: (1e-4, 1e-4), STORAGE_MOMENTS_F16: (1e-3, 5e-3)}


@pytest.mark.parametrize("storage", sorted(STORAGES))
def test_2000_steps_of_a_filling_capillary(storage):
    st = STORAGES[storage]
    cap = W.Capillary("f", 300, 30, 60, 230, 4, 22, 20, 10, W.binary_params(nu_l=0.5, nu_g=0.05),
                      theta_deg=45.0)
    lat = Lattice.from_workload(cap, storage=st)
    orc = oracle.Oracle(cap).init_default()
    lat.step(2000)
    orc.step(2000)
    rg, _, _, pg = lat.fields()
    ro, _, _, po = orc.fields()
    drho, dphi = float(np.abs(rg - ro).max()), float(np.abs(pg - po).max())
    d, do = lat.filled_length(), orc.filled_length()
    print(f"{storage}: max |d rho| {drho:.2e}, max |d phi| {dphi:.2e}, |d l| {abs(d['l'] - do['l']):.2e}")
    br, bp = BOUND_2000[st]
    assert drho < br and dphi < bp
    assert abs(d["l"] - do["l"]) < 0.05


@pytest.mark.parametrize("storage", sorted(STORAGES))
def test_close_to_the_fp32_moment_storage(storage):
    cap = W.Capillary("c", 256, 40, 64, 160, 6, 28, 16, 12, W.binary_params(nu_l=0.83, nu_g=0.0166),
                      theta_deg=45.0)
    a = Lattice.from_workload(cap, storage=STORAGE_MOMENTS)
    b = Lattice.from_workload(cap, storage=STORAGES[storage])
    a.step(500)
    b.step(500)
    da, db = a.filled_length(), b.filled_length()
    assert abs(da["l"] - db["l"]) < (1e-3 if storage == "gelim" else 2e-2)
    assert abs(da["mass"] / db["mass"] - 1) < (1e-6 if storage == "gelim" else 1e-4)


def test_interface_of_the_g_eliminated_storage():
    """populations(): f as stored and g = (phi, 0, ..., 0); set_populations keeps f and the
    sum of g; the pull kernel is the only step kernel."""
    cap = GEOMS["capillary_ragged"](W.binary_params())
    lat = Lattice.from_workload(cap, storage=STORAGE_F32_GELIM)
    assert lat.kernel() == 4
    for v in (1, 2, 3):
        with pytest.raises(LbError):
            lat.set_kernel(v)
    rng = np.random.default_rng(5)
    f = rng.uniform(0.0, 0.3, (9, cap.ny, cap.nx))
    g = rng.uniform(-0.1, 0.1, (9, cap.ny, cap.nx))
    lat.set_populations(f, g)
    kinds = oracle.Oracle(cap).node_kinds()
    fluid = kinds != 2
    f2, g2 = lat.populations(rested=False)
    np.testing.assert_allclose(f2[:, fluid], f[:, fluid], rtol=0, atol=1e-7)
    np.testing.assert_allclose(g2[0][fluid], g.sum(axis=0)[fluid], rtol=1e-6, atol=1e-7)
    assert np.all(g2[1:] == 0) and np.all(f2[:, ~fluid] == 0)
    np.testing.assert_allclose(lat.moments()[:, fluid], moments_of(f, g)[:, fluid], rtol=1e-6, atol=1e-6)


def test_interface_of_the_fp16_moment_storage():
    cap = GEOMS["capillary_ragged"](W.binary_params())
    lat = Lattice.from_workload(cap, storage=STORAGE_MOMENTS_F16)
    assert lat.kernel() == 4
    with pytest.raises(LbError):
        lat.populations()
    rng = np.random.default_rng(6)
    f = rng.uniform(0.05, 0.15, (9, cap.ny, cap.nx))
    g = rng.uniform(-0.1, 0.1, (9, cap.ny, cap.nx))
    lat.set_populations(f, g)
    kinds = oracle.Oracle(cap).node_kinds()
    fluid = kinds != 2
    m, want = lat.moments(), moments_of(f, g)
    # rho - 1, j and the stresses rounded to FP16 once; phi in FP32
    dev = np.abs(want).copy()
    dev[0] = np.abs(want[0] - 1)
    assert np.all(np.abs(m - want)[:5, fluid] <= dev[:5, fluid] * 2.0 ** -11 + 1e-7)
    np.testing.assert_allclose(m[5][fluid], want[5][fluid], rtol=1e-6, atol=1e-7)


def test_batches_refuse_the_two_storages():
    from paper_0911_0459_gb300 import Batch
    caps = [W.Capillary("b", 96, 24, 24, 64, 3, 18, 8, 6, W.binary_params(), theta_deg=45.0)]
    for st in STORAGES.values():
        with pytest.raises(LbError):
            Batch(caps, storage=st)
