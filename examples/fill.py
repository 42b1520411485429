"""Example: one filling capillary and a sweep of 256 uneven capillaries (needs a GPU).

Device memory and streams come from PyTorch; every step runs in the CUDA library.
Run from anywhere:  python examples/fill.py
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import workloads as W  # noqa: E402
from paper_0911_0459_gb300 import STORAGE_F32_BLOCKED, Batch, Lattice, meniscus  # noqa: E402


def main(checkpoint="fill.npz"):
    # one capillary: 700 x 40, one solid row, tube of 350 columns, viscosity ratio ~70, 60 degrees
    cap = W.Capillary("fill", 700, 40, 350, 350, 0, 39, 16, 10,
                      W.binary_params(nu_l=1.17, nu_g=0.017), theta_deg=60.0)
    # FP32 populations in 32-node blocks (the planar FP32 storage's bits, staged with one bulk
    # copy per tile row); or storage=STORAGE_MOMENTS (48 B per update)
    lat = Lattice.from_workload(cap, storage=STORAGE_F32_BLOCKED)
    lat.autotune()                             # kernel variant and tile, timed on this lattice
    lat.step(20000)                            # replayed 64-step CUDA graphs
    d = lat.filled_length()                    # FP64: l, l_vol, mass, phi_sum
    rho, ux, uy, phi = lat.fields()            # host arrays (ny, nx)
    theta = meniscus.lattice_contact_angle(lat)
    lat.save(checkpoint)                       # byte-exact checkpoint; Lattice(...).load() resumes

    # a sweep of 256 uneven capillaries in one persistent launch, l(t) sampled on the way
    b = Batch(W.sweep(seed=0, n=256), storage=STORAGE_F32_BLOCKED)
    b.autotune(steps=2)
    l_t = b.run_sampled([500, 1000, 2000])     # (256, 3, 4): l, l_vol, mass, phi_sum
    return {"lattice": lat, "batch": b, "d": d, "theta": theta, "l_t": l_t, "phi": phi}


if __name__ == "__main__":
    r = main()
    print(f"l = {r['d']['l']:.2f} after 20000 steps, dynamic angle {r['theta']:.1f} deg; "
          f"sweep l(t) at step 2000: {r['l_t'][:4, 2, 0]}")
    r["lattice"].close()
    r["batch"].close()
