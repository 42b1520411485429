"""Run one capillary on the GPU and log a JSON line per output interval.

    python -m paper_0911_0459_gb300.run --config binary_2048x64 --steps 50000 --every 1000

Configurations (synthetic inputs shaped like the paper's runs):
  lg_256x32            liquid-gas capillary, FP64 (Sec. 2.2)
  binary_2048x64       binary capillary, H = 50, viscosity ratio 10, 60 degrees
  binary_16384x256     binary capillary, H = 200, viscosity ratio 50, 45 degrees
  binary_crop_1024x64  its 1024 x 64 crop
  paper_700x40         the paper's binary layout (one solid row, L = 350), nu 1.17 / 0.017

Each line: {"step", "l", "l_vol", "mass", "phi_sum", "MLUPS"} (the FP64 reductions of
lb_filled_length; MLUPS over the interval, fluid nodes, wall clock).  --save / --resume
write and read a byte-exact checkpoint; --fields writes rho, ux, uy, phi at the end.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

from .lb import (STORAGE_F16_BLOCKED, STORAGE_F16DEV, STORAGE_F32, STORAGE_F32_BLOCKED,  # noqa: E402
                 STORAGE_F32_GELIM, STORAGE_F64, STORAGE_MOMENTS, STORAGE_MOMENTS_F16, Lattice)

STORAGES = {"f64": STORAGE_F64, "f32": STORAGE_F32, "f32b": STORAGE_F32_BLOCKED, "f16dev": STORAGE_F16DEV,
            "f16b": STORAGE_F16_BLOCKED, "moments": STORAGE_MOMENTS, "moments_f16": STORAGE_MOMENTS_F16,
            "gelim": STORAGE_F32_GELIM}


def paper_700x40(storage, theta=60.0, M=0.1):
    return W.Capillary("paper_700x40", 700, 40, 350, 350, 0, 39, 16, 10,
                       W.binary_params(nu_l=1.17, nu_g=0.017, M=M, storage=storage), theta_deg=theta)


def make(config, storage=None, theta=None, M=None):
    if config == "lg_256x32":
        cap = W.config_lg_256x32()
        if storage is not None:
            cap.params.storage = storage
        return cap
    st = STORAGE_F32 if storage is None else storage
    if config == "binary_2048x64":
        cap = W.config_binary_2048x64()
        cap.params.storage = st
    elif config == "binary_16384x256":
        cap = W.config_binary_16384x256(st)
    elif config == "binary_crop_1024x64":
        cap = W.config_binary_crop_1024x64(st)
    elif config == "paper_700x40":
        cap = paper_700x40(st, 60.0 if theta is None else theta, 0.1 if M is None else M)
    else:
        raise ValueError(f"unknown configuration {config}")
    if theta is not None and config != "paper_700x40":
        cap.theta_deg, cap.wall_grad = theta, None
    if M is not None:
        cap.params.M = M
    return cap


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--config", default="binary_2048x64",
                    choices=["lg_256x32", "binary_2048x64", "binary_16384x256", "binary_crop_1024x64", "paper_700x40"])
    ap.add_argument("--storage", choices=sorted(STORAGES), default=None,
                    help="state storage (default f64 for lg_256x32, f32 otherwise; f32b holds the same "
                         "values in 32-node blocks, the same bits and faster)")
    ap.add_argument("--theta", type=float, default=None, help="equilibrium contact angle (binary), degrees")
    ap.add_argument("--mobility", type=float, default=None, help="mobility M (binary)")
    ap.add_argument("--steps", type=int, default=2000, help="run until this step count")
    ap.add_argument("--every", type=int, default=100, help="steps between output lines")
    ap.add_argument("--autotune", action="store_true", help="time kernel variants and tiles first")
    ap.add_argument("--save", default=None, help="checkpoint file written at the end")
    ap.add_argument("--resume", default=None, help="checkpoint file to start from")
    ap.add_argument("--fields", default=None, help=".npz file for rho, ux, uy, phi at the end")
    a = ap.parse_args(argv)
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("a CUDA device is required (there is no CPU fallback)")
    cap = make(a.config, STORAGES.get(a.storage), a.theta, a.mobility)
    lat = Lattice.from_workload(cap)
    if a.resume:
        lat.load(a.resume)
    if a.autotune:
        lat.autotune()
    fluid = lat.fluid_nodes
    while lat.time < a.steps:
        n = min(a.every, a.steps - lat.time)
        t0 = time.perf_counter()
        lat.step(n)
        d = lat.filled_length()   # waits for the stream
        dt = time.perf_counter() - t0
        print(json.dumps({"step": lat.time, "l": d["l"], "l_vol": d["l_vol"], "mass": d["mass"],
                          "phi_sum": d["phi_sum"], "MLUPS": fluid * n / dt / 1e6}), flush=True)
    if a.save:
        lat.save(a.save)
    if a.fields:
        rho, ux, uy, phi = lat.fields()
        np.savez(a.fields, rho=rho, ux=ux, uy=uy, phi=phi)
    lat.close()


if __name__ == "__main__":
    main()
