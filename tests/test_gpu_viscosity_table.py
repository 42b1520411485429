"""The viscosity table of App. A (nu_table = K) on the CUDA path (needs a GPU).

One step from a random state against the oracle with the same table (K = 2 and 3:
table boundaries at phi = 0 and phi = +-1/2, where no node of the test sits within
rounding of a boundary), for the FP32 populations and the moment storage; and the
size of the paper's approximation: l(t) of a filling capillary with 10^4 entries
against the exact local viscosity, next to a coarse table.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0911_0459_gb300 import Lattice, STORAGE_F32, STORAGE_MOMENTS  # noqa: E402

E = np.array([(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (-1, 1), (1, -1)], float)
ROWS = np.array([np.ones(9), E[:, 0], E[:, 1], E[:, 0] ** 2 - E[:, 1] ** 2, E[:, 0] * E[:, 1]])


def moments_of(f, g):
    return np.concatenate([np.einsum("ki,iyx->kyx", ROWS, f), g.sum(axis=0)[None]], axis=0)


@pytest.mark.parametrize("storage", [STORAGE_F32, STORAGE_MOMENTS])
@pytest.mark.parametrize("K", [2, 3])
def test_one_step_with_a_viscosity_table_matches_oracle(K, storage):
    p = W.binary_params(nu_l=0.7, nu_g=0.05, M=0.2, nu_table=K)
    cap = W.Capillary("t", 203, 37, 61, 120, 5, 27, 12, 8, p, wall_grad=-0.11)
    fields = W.random_state_fields(cap.nx, cap.ny, seed=11, model=W.BINARY)
    lat = Lattice.from_workload(cap, storage=storage).init_fields(*fields)
    orc = oracle.Oracle(cap).init_fields(*fields)
    lat.step(1)
    orc.step(1)
    kinds = orc.node_kinds()
    m = lat.moments()
    m[1:3, kinds == 1] = 0.0        # the rest rule, applied on read
    d = np.abs(m - moments_of(*orc.populations()))[:, kinds != 2]
    assert d.max() < 2e-6
    # and the table is in use: the exact viscosity gives a different step
    exact = oracle.Oracle(W.Capillary("t", 203, 37, 61, 120, 5, 27, 12, 8,
                                      W.binary_params(nu_l=0.7, nu_g=0.05, M=0.2), wall_grad=-0.11)
                          ).init_fields(*fields).step(1)
    assert np.abs(moments_of(*exact.populations()) - moments_of(*orc.populations())).max() > 1e-5


def test_size_of_the_table_approximation_in_a_filling_capillary():
    """Viscosity ratio 50 (0.83 / 0.0166), 45 degrees, 3000 steps: with 10^4 table
    entries l(t) stays within 1e-3 of the exact-viscosity run; a 16-entry table
    moves it by more."""
    def run(K):
        cap = W.Capillary("f", 300, 30, 60, 230, 4, 22, 20, 10,
                          W.binary_params(nu_l=0.83, nu_g=0.0166, nu_table=K), theta_deg=45.0)
        lat = Lattice.from_workload(cap, storage=STORAGE_F32)
        ls = []
        for _ in range(6):
            lat.step(500)
            ls.append(lat.filled_length()["l"])
        lat.close()
        return np.array(ls)
    exact, fine, coarse = run(0), run(10000), run(16)
    d_fine, d_coarse = np.abs(fine - exact).max(), np.abs(coarse - exact).max()
    print(f"max |l_table - l_exact| over 3000 steps: 10^4 entries {d_fine:.2e}, 16 entries {d_coarse:.2e}")
    assert d_fine < 1e-3
    assert d_coarse > d_fine
