"""Contact angles measured by the circle fit of Sec. 3.2 on the CUDA path (needs a GPU):
a liquid plug at rest (the static angle), the dynamic angle of the filling capillary of
Fig. 5 (nu_l = 1.17, nu_g = 0.017, theta_eq = 60), and the mobility study of Sec. 3.3
(Fig. 6, equal viscosities) run as one batch."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0911_0459_gb300 import Batch, Lattice, meniscus  # noqa: E402

H = 39


def paper_capillary(params, theta):
    """700 x 40, one solid row, tube [350, 700) after 334 liquid and 16 gas columns."""
    return W.Capillary("paper", 700, 40, 350, 350, 0, H, 16, 10, params, theta_deg=theta)


def static_angle(theta):
    """A liquid plug at rest in a closed periodic channel (no reservoirs)."""
    cap = W.Capillary("plug", 240, 40, 0, 240, 0, H, 60, 120, W.binary_params(nu_l=1 / 6, nu_g=1 / 6),
                      theta_deg=theta)
    lat = Lattice.from_workload(cap)
    lat.step(40000)
    th = meniscus.lattice_contact_angle(lat)
    lat.close()
    return th


def test_static_angle_of_a_plug_follows_the_wetting_condition():
    th = {t: static_angle(t) for t in (45.0, 60.0, 75.0)}
    print("static circle-fit angles:", th)
    assert th[45.0] < th[60.0] < th[75.0]
    for t, v in th.items():
        assert abs(v - t) < 5.0      # the fit at the boundary-node rows of a narrow interface


def test_dynamic_angle_exceeds_the_static_one_and_relaxes():
    """Sec. 3.2, Fig. 5b: while the meniscus moves the angle is above the equilibrium one
    and it decreases as the filling slows down."""
    static = static_angle(60.0)
    cap = paper_capillary(W.binary_params(nu_l=1.17, nu_g=0.017, M=0.1), 60.0)
    lat = Lattice.from_workload(cap)
    th = []
    for _ in range(40):
        lat.step(6000)
        th.append(meniscus.lattice_contact_angle(lat))
    th = np.array(th)
    print(f"static {static:.1f}; dynamic {th[0]:.1f} .. {th[-1]:.1f}")
    assert np.all(th > static + 3.0)
    assert th[:10].mean() > th[-10:].mean() + 3.0


def test_mobility_scan_in_one_batch():
    """Sec. 3.3, Fig. 6, equal viscosities: the filling velocity (a linear fit of l(t))
    grows with the mobility M and the dynamic contact angle falls."""
    Ms = [0.05, 0.1, 0.2, 0.4, 0.8]
    caps = [paper_capillary(W.binary_params(nu_l=1 / 6, nu_g=1 / 6, M=M), 60.0) for M in Ms]
    b = Batch(caps)
    at = list(range(2000, 40001, 2000))
    out = b.run_sampled(at)
    v = [np.polyfit(np.array(at[5:], float), out[i, 5:, 0], 1)[0] for i in range(len(Ms))]
    c = caps[0]
    th = [meniscus.contact_angle(b.moments(i)[5], c.tube_x0, c.tube_len, c.tube_y0, c.tube_h)
          for i in range(len(Ms))]
    print("M", Ms, "velocity", np.round(v, 6), "theta", np.round(th, 2))
    assert all(v2 > v1 for v1, v2 in zip(v, v[1:]))
    assert all(t2 < t1 for t1, t2 in zip(th, th[1:]))
    b.close()
