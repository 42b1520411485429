"""Learned surrogate of the filling curve l(t) with lattice Boltzmann fallback.

Inputs of a query: channel width H, viscosity ratio eta_l / eta_g, cos(theta_eq)
and the liquid-gas surface tension gamma (varied through A = kappa of the
phi^4 free energy, gamma = sqrt(8 kappa A / 9)).  Output: l(t_k) at 64
log-spaced times t_k = 100 * 200^(k/63) (100 .. 20000 steps).

Training data come from the batched lattice Boltzmann sweep itself
(Batch.run_sampled); the network is the ensemble MLP of include/lb_mlp.h,
trained on the GPU by its own kernels.  A query whose ensemble spread exceeds
2 % (relative) anywhere on the curve is answered by running the lattice
Boltzmann model instead.  The method without the surrogate is Washburn's law,
Eq. (3), with the equilibrium angle and l_eff = l + H/2.

Sweep for the surrogate (a reading of the workload): the tube length is fixed
at 1024 (it is not an input, so varying it would add noise the network cannot
explain) and the liquid reservoir has 384 columns so it never runs dry.
"""
from __future__ import annotations

import math
import time
from typing import Dict, List

import numpy as np

import workloads as W

SAMPLE_STEPS = np.array([int(round(100 * 200 ** (k / 63))) for k in range(64)], dtype=np.int64)
TUBE_LEN = 1024
LIQUID_COLS = 384


def surrogate_sweep(seed: int, n: int) -> List[W.Capillary]:
    return W.sweep(seed=seed, n=n, steps=int(SAMPLE_STEPS[-1]), fixed_len=TUBE_LEN, vary_gamma=True,
                   liquid_cols=LIQUID_COLS)


def gamma_of(A: float, kappa: float) -> float:
    return math.sqrt(8.0 * kappa * A / 9.0)


def features(caps) -> np.ndarray:
    """Raw inputs (H, viscosity ratio, cos theta, gamma) of each capillary."""
    out = []
    for c in caps:
        p = c.params
        out.append([c.tube_h, p.nu_l / p.nu_g, math.cos(math.radians(c.theta_deg)), gamma_of(p.A, p.kappa)])
    return np.asarray(out, dtype=np.float64)


def normalize_x(f: np.ndarray) -> np.ndarray:
    f = np.asarray(f, dtype=np.float64)
    return np.stack([(f[:, 0] - 72.0) / 56.0, (np.log10(f[:, 1]) - 1.0), (f[:, 2] - 0.55) / 0.32,
                     (f[:, 3] - 0.0377) / 0.0094], axis=1).astype(np.float32)


def run_lb(caps, chunk: int = 1024, storage=None) -> Dict[str, np.ndarray]:
    """l(t_k) (and l_vol) of every capillary from the batched lattice Boltzmann sweep.

    storage None: FP32 populations in 32-node blocks, which give the same bits as the
    planar FP32 storage (the capillaries' own) and run the batch faster."""
    import torch
    from .lb import STORAGE_F32_BLOCKED, Batch
    if storage is None:
        storage = STORAGE_F32_BLOCKED
    ls, lv = [], []
    t0 = time.perf_counter()
    lu = 0
    for i in range(0, len(caps), chunk):
        part = caps[i:i + chunk]
        b = Batch(part, storage=storage)
        b.set_tile(128, 16)
        out = b.run_sampled(SAMPLE_STEPS)
        lu += b.fluid_nodes() * int(SAMPLE_STEPS[-1])
        ls.append(out[:, :, 0])
        lv.append(out[:, :, 1])
        b.close()
        del b
        torch.cuda.empty_cache()
    dt = time.perf_counter() - t0
    return {"l": np.concatenate(ls), "l_vol": np.concatenate(lv), "seconds": dt, "lattice_updates": lu}


def washburn(caps, l0: float = 10.0) -> np.ndarray:
    """Eq. (3) with theta_eq and l_eff = l + H/2, t0 from l(0) = l0."""
    out = []
    for c in caps:
        p = c.params
        g = gamma_of(p.A, p.kappa)
        H = float(c.tube_h)
        rate = g * H * math.cos(math.radians(c.theta_deg)) / (3.0 * p.nu_l)   # eta = rho nu_l, rho = 1
        leff0 = l0 + H / 2.0
        t0 = leff0 * leff0 / rate
        out.append(np.sqrt(rate * (SAMPLE_STEPS + t0)) - H / 2.0)
    return np.asarray(out)


class Surrogate:
    """Ensemble MLP on log l(t_k); normalisation fitted on the training set."""

    def __init__(self, members: int = 5, hidden: int = 256, seed: int = 0, max_batch: int = 4096):
        from .mlp import MLP
        self.net = MLP(4, hidden, len(SAMPLE_STEPS), members=members, max_batch=max_batch, seed=seed)
        self.mu = None
        self.sd = None

    def fit(self, feats, l, steps: int = 6000, lr: float = 3e-3, lr_min: float = 1e-5, wd: float = 1e-6):
        y = np.log(np.maximum(np.asarray(l, dtype=np.float64), 1e-3))
        self.mu = y.mean(0)
        self.sd = y.std(0) + 1e-6
        self.net.set_data(normalize_x(feats), ((y - self.mu) / self.sd).astype(np.float32))
        return self.net.train(steps, lr=lr, lr_min=lr_min, wd=wd)

    def predict(self, feats):
        """Mean l(t_k) and the ensemble's relative spread (std of log l)."""
        m, s = self.net.predict(normalize_x(feats))
        logl = self.mu + self.sd * m.astype(np.float64)
        return np.exp(logl), self.sd * s.astype(np.float64)

    def close(self):
        self.net.close()


def predict_with_fallback(sur: Surrogate, caps, threshold: float = 0.02):
    """Surrogate answers where its spread is at most `threshold`, the LB elsewhere."""
    l, spread = sur.predict(features(caps))
    bad = np.where(spread.max(1) > threshold)[0]
    if len(bad):
        lb = run_lb([caps[i] for i in bad])["l"]
        l = l.copy()
        l[bad] = lb
    return l, bad


def rms_rel(pred, ref) -> float:
    return float(np.sqrt(np.mean(((pred - ref) / ref) ** 2)))


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--n-train", type=int, default=4096)
    ap.add_argument("--n-test", type=int, default=512)
    ap.add_argument("--out", default="surrogate_data.npz")
    ap.add_argument("--report", default="surrogate_report.json")
    ap.add_argument("--data", default=None, help="reuse a generated dataset instead of running the LB")
    ap.add_argument("--steps", type=int, default=6000)
    args = ap.parse_args(argv)
    train_caps = surrogate_sweep(1, args.n_train)
    test_caps = surrogate_sweep(2, args.n_test)
    if args.data:
        d = np.load(args.data)
        l_train, l_test = d["l_train"], d["l_test"]
        gen = {"seconds": float(d["seconds"]), "lattice_updates": int(d["lattice_updates"])}
    else:
        r1 = run_lb(train_caps)
        r2 = run_lb(test_caps)
        l_train, l_test = r1["l"], r2["l"]
        gen = {"seconds": r1["seconds"] + r2["seconds"], "lattice_updates": r1["lattice_updates"] + r2["lattice_updates"]}
        np.savez_compressed(args.out, l_train=l_train.astype(np.float32), l_test=l_test.astype(np.float32),
                            x_train=features(train_caps), x_test=features(test_caps), t=SAMPLE_STEPS,
                            seconds=gen["seconds"], lattice_updates=gen["lattice_updates"])
    sur = Surrogate()
    t0 = time.perf_counter()
    losses = sur.fit(features(train_caps), l_train, steps=args.steps)
    t_train = time.perf_counter() - t0
    t0 = time.perf_counter()
    pred, spread = sur.predict(features(test_caps))
    t_pred = time.perf_counter() - t0
    rms = rms_rel(pred, l_test)
    fall = spread.max(1) > 0.02
    combined = np.where(fall[:, None], l_test, pred)   # the fallback answers with the LB itself
    wash = washburn(test_caps)
    report = {"rms_rel_surrogate": rms, "rms_rel_with_fallback": rms_rel(combined, l_test),
              "fallback_fraction": float(fall.mean()), "rms_rel_washburn": rms_rel(wash, l_test),
              "train_seconds": t_train, "predict_seconds_512": t_pred,
              "lb_seconds_per_run": gen["seconds"] / (args.n_train + args.n_test),
              "lb_lattice_updates": gen["lattice_updates"], "final_losses": [float(v) for v in losses]}
    with open(args.report, "w") as f:
        json.dump(report, f, indent=1)
    print(json.dumps(report))
    sur.close()


if __name__ == "__main__":
    main()
