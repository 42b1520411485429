"""Benchmark: lattice updates per second of the binary capillary, 16384 x 256 (H = 200).

One "step" is one time step of the whole LB update (stencils, equilibria,
collision, streaming, walls) over the 16384 x 256 binary capillary, with the
FP64 reductions (mass, sum of phi, l(t)) every 100 steps, as in a filling run.
The state (2 x 302 MB in FP32) is larger than L2, so no flush is needed between
steps.  MLUPS counts fluid nodes only (solid wall rows are not updated).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own replica of the capillary (one capillary
does not shard without a halo exchange; the value is the sum over ranks and the
time is the maximum over ranks).  --impl reference times the FP64 CPU oracle, as
it stands, on a bounded sample of the same workload (one time step of the
1024 x 64 crop per bench step, in one independent copy of the oracle per host
core) on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "MLUPS (fluid-node lattice updates per second), binary capillary 16384x256"
RED_EVERY = 100
# stored surrogate targets vs a fresh LB run of the same queries: FP32 rounding differences
# of one build or GPU against another, far below the surrogate's 2 % bar
DATASET_TOL = 1e-3


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        time.sleep(0.25)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash():
    """Hash of the step kernel's code (comments and blank space removed, so that a comment
    edit keeps a capture valid)."""
    import re
    h = hashlib.sha256()
    for f in ("lb_device.cuh", "lb_step_tma.cuh", "lb_ops_impl.cuh"):
        src = open(os.path.join(ROOT, "paper_0911_0459_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


# ring depth NS of the staged kernel per tile width: shallow (variant 2) and deep (variant 3)
STAGED_NS = {2: {64: 4, 128: 4, 256: 3}, 3: {64: 8, 128: 6, 256: 4}}


def step_kernel_label(variant, tx, ty, storage="FP32"):
    """The exact step-kernel instance of a lattice: variant, tile and ring depth."""
    if variant in STAGED_NS:
        return (f"step_tma_kernel<binary, {storage}, BX={tx}, NS={STAGED_NS[variant][tx]}> "
                f"(variant {variant}, tile {tx}x{ty})")
    if variant == 4:
        return f"moment_step_kernel<{storage}> (tile {tx}x{ty})"
    return f"step_kernel<binary, {storage}, BX={tx}> (variant {variant}, tile {tx}x{ty})"


def ncu_traffic(kind, variant, tile):
    """DRAM bytes per launch of the step kernel from the committed ncu capture, if that
    capture was taken on the current kernel source, the same kernel variant and the same
    tile as the timed launches; None otherwise."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        d = json.load(open(path))
        e = d[kind]
        if e.get("kernel_hash") != kernel_source_hash():
            return None
        if int(e["variant"]) != int(variant) or list(e["tile"]) != list(tile):
            return None
        return float(e["dram_bytes_per_launch_full_size"])
    except Exception:
        return None


# FP64 work per fluid-node update of the liquid-gas step kernel (ncu instruction counts of
# one launch on 16384 x 256: 129.2 M DFMA, 82.6 M DMUL, 184.4 M DADD over 3 305 472 fluid
# nodes): 120 FP64 instructions, 159 flops (an FMA counts two)
LG_FP64_INST_PER_LU = 120.0
LG_FP64_FLOPS_PER_LU = 159.0


def lg_fp64_roofline(torch, Lattice):
    """The liquid-gas FP64 capillary at 16384 x 256 against the measured FP64 FMA rate
    (lb_fp64_fma_rate): GB300's FP64 pipe, not HBM, bounds this path."""
    from paper_0911_0459_gb300 import lb as lbmod
    lat = Lattice.from_workload(W.config_lg_16384x256())
    tx, ty, _ = lat.autotune()
    lat.step(4)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(lat.stream)
    lat.step(64)
    b.record(lat.stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / 64
    fluid = lat.fluid_nodes
    rate = max(lbmod.fp64_fma_rate() for _ in range(2))
    achieved = fluid * LG_FP64_FLOPS_PER_LU / (ms * 1e-3) / 1e12
    pipe = fluid * LG_FP64_INST_PER_LU / (ms * 1e-3) / 1e12           # FP64 instructions per ns
    out = {"MLUPS": fluid / (ms * 1e-3) / 1e6, "ms_per_step": ms, "tile": [tx, ty], "kernel_variant": lat.kernel(),
           "fp64_peak_tflops_measured": rate, "fp64_tflops_achieved": achieved,
           "frac_of_fp64_peak": achieved / rate,
           "frac_of_fp64_pipe": pipe / (rate / 2.0),
           "GBps": fluid * 144 / (ms * 1e-3) / 1e9,
           "what": "liquid-gas FP64, 144 B/LU; FP64 flops per LU from ncu instruction counts (159: 39 DFMA, "
                   "25 DMUL, 56 DADD); frac_of_fp64_pipe counts every FP64 instruction as one FMA slot"}
    lat.close()
    return out


def fluid_nodes_of(cap):
    """Fluid nodes of a workload: every node but the tube's solid rows."""
    solid = cap.tube_len * (cap.ny - cap.tube_h) if cap.tube_len > 0 else 0
    return cap.nx * cap.ny - solid


# algorithmic bytes per fluid-node update and the name of each storage
STORAGES = {"f32b": (144.0, "FP32 populations in 32-node blocks", "SF32B"),
            "f32": (144.0, "FP32 populations in planes", "FP32"), "f16dev": (76.0, "FP16-deviation storage", "FP16dev"),
            "f16b": (76.0, "FP16-deviation storage in 32-node blocks", "SF16B"),
            "moments": (48.0, "FP32 moment storage", "SM32"), "moments_f16": (28.0, "FP16 moment storage", "SM16"),
            "gelim": (80.0, "FP32 f + phi storage (g eliminated)", "SG32")}


def bench_config(cap, world, storage="f32b"):
    """The `config` object of both arms' JSON lines (the same workload)."""
    return {"workload": "binary_16384x256: H=200 tube over x in [512, 16384), gas 128 cols, "
                        f"viscosity ratio 50 (0.83/0.0166), theta 45 deg, {STORAGES[storage][1]}",
            "nodes": cap.nx * cap.ny, "fluid_nodes": fluid_nodes_of(cap), "reductions_every": RED_EVERY,
            "l2": "no flush: state 2 x 302 MB > 129 MB L2", "parallelism": f"replicas x{world}"}


def _oracle_copy(arg):
    """One copy of the oracle on the 1024 x 64 crop (a spawned process): `warm` steps,
    then `steps` steps timed from the shared start time t_start (system-wide monotonic
    clock).  Returns (start, end, fluid nodes)."""
    steps, warm, t_start = arg
    import oracle
    o = oracle.Oracle(W.config_binary_crop_1024x64()).init_default()
    fluid = int((o.node_kinds() < 2).sum())
    o.step(warm)
    while time.monotonic() < t_start:
        time.sleep(0.001)
    t0 = time.monotonic()
    o.step(steps)
    return t0, time.monotonic(), fluid


def oracle_all_cores(steps, warm=0, lead=8.0):
    """The oracle as it stands, one independent copy per available host core, all
    timed from one start: aggregate MLUPS over the span from that start to the last
    copy's end.  Processes are spawned (a fork after CUDA initialisation can hang)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    t_start = time.monotonic() + lead
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_copy, [(steps, warm, t_start)] * cores)
    span = max(r[1] for r in res) - min(r[0] for r in res)
    lu = sum(r[2] for r in res) * steps
    return {"value": lu / span / 1e6, "cores": cores, "seconds": span}


def cpu_baseline(sample_steps=2000, copy_steps=500):
    """The FP64 oracle on the 1024 x 64 crop of the same capillary: one copy per host
    core (the baseline value) and a single thread.  Returns the timing and the
    single-thread oracle, whose state after the sample serves the precision report."""
    import oracle
    cap = W.config_binary_crop_1024x64()
    o = oracle.Oracle(cap).init_default()
    t0 = time.perf_counter()
    o.step(sample_steps)
    dt = time.perf_counter() - t0
    fluid = int((o.node_kinds() < 2).sum())
    one = {"value": fluid * sample_steps / dt / 1e6, "cores": 1, "seconds": dt,
           "sample": f"{sample_steps} steps of the 1024x64 crop, 1 thread"}
    try:
        allc = oracle_all_cores(copy_steps)
    except Exception as ex:  # no process pool: report the single thread
        return {"value": one["value"], "unit": "MLUPS", "cores": 1, "kind": "oracle",
                "sample": one["sample"] + f" (all-core run failed: {ex!r})", "seconds": dt}, o
    return {"value": allc["value"], "unit": "MLUPS", "cores": allc["cores"], "kind": "oracle",
            "sample": f"{allc['cores']} independent copies of the oracle (one per host core), "
                      f"{copy_steps} steps each of the 1024x64 crop (H=50, same parameters), FP64",
            "seconds": allc["seconds"], "single_thread": one}, o


def precision_report(Lattice, orc, steps):
    """Error of each storage against the FP64 oracle on the crop after `steps` steps."""
    from paper_0911_0459_gb300 import (STORAGE_F16_BLOCKED, STORAGE_F16DEV, STORAGE_F32, STORAGE_F32_BLOCKED,
                                       STORAGE_F32_GELIM, STORAGE_F64, STORAGE_MOMENTS, STORAGE_MOMENTS_F16)
    rho_o, _, _, phi_o = orc.fields()
    l_o = orc.filled_length()["l"]
    out = {"workload": "1024x64 crop of the large capillary, default initial state", "steps": steps}
    import dataclasses
    for name, st, table in (("f64", STORAGE_F64, 0), ("f32", STORAGE_F32, 0), ("f32_blocks", STORAGE_F32_BLOCKED, 0),
                            ("f16dev", STORAGE_F16DEV, 0), ("f16_blocks", STORAGE_F16_BLOCKED, 0),
                            ("moments_f32", STORAGE_MOMENTS, 0), ("moments_f16", STORAGE_MOMENTS_F16, 0),
                            ("f32_g_eliminated", STORAGE_F32_GELIM, 0), ("f32_nu_table_1e4", STORAGE_F32, 10000)):
        cap = W.config_binary_crop_1024x64(st)
        cap.params = dataclasses.replace(cap.params, nu_table=table)
        lat = Lattice.from_workload(cap)
        lat.step(steps)
        rho, _, _, phi = lat.fields()
        out[name] = {"max_abs_drho": float(np.abs(rho - rho_o).max()),
                     "max_abs_dphi": float(np.abs(phi - phi_o).max()),
                     "abs_dl": abs(lat.filled_length()["l"] - l_o)}
        lat.close()
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    r = oracle_all_cores(args.steps, warm=args.warmup)
    v, dt = r["value"], r["seconds"]
    line = {"metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": bench_config(W.config_binary_16384x256(), world),
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": r["cores"], "kind": "oracle",
                             "sample": "binary_16384x256 sampled as its 1024x64 crop (H=50, ratio 50, 45 deg): "
                                       f"{args.steps} steps (one per bench step) of the crop in each of "
                                       f"{r['cores']} independent oracle copies (one per host core), FP64"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_vs_sequential(torch, Lattice, steps, n=256, storage=None):
    """The seeded sweep of 256 uneven binary capillaries (H 16..128, tube 1024..8192,
    ratios 1..100, 30..80 degrees) in the given storage: one persistent CUDA-graph launch per
    sampled run for all capillaries against one lattice per capillary run in
    turn (same storage), both with l(t) sampled 4 times over `steps` steps."""
    from paper_0911_0459_gb300 import Batch, shard
    rank, world, _ = dist_env()
    caps_all = W.sweep(seed=0, n=n)
    # ranks split the sweep by estimated cost; no exchange on the data path
    caps = [caps_all[i] for i in shard.my_share(caps_all, rank, world)] if world > 1 else caps_all
    at = [steps // 4, steps // 2, 3 * steps // 4, steps]
    b = Batch(caps, storage=storage)
    tx, ty, _ = b.autotune(steps=2)
    b.run_sampled([2])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = b.run_sampled(at)
    t_batch = time.perf_counter() - t0
    fluid = b.fluid_nodes()
    b.close()
    del b
    torch.cuda.empty_cache()
    # one launch per run: each capillary alone in the same persistent kernel (a batch of
    # one, the batch's tile), launched in turn; creation is outside the timed region
    singles = [Batch([c], storage=storage) for c in caps]
    for s in singles:
        s.set_tile(tx, ty)
        s.run_sampled([2])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in singles:
        s.run_sampled(at)
    torch.cuda.synchronize()
    t_one = time.perf_counter() - t0
    for s in singles:
        s.close()
    del singles
    torch.cuda.empty_cache()
    t_seq = 0.0
    for c in caps:
        lat = Lattice.from_workload(c, storage=storage)
        lat.step(2)
        lat.filled_length()
        t0 = time.perf_counter()
        prev = 0
        for s in at:
            lat.step(s - prev)
            lat.filled_length()
            prev = s
        t_seq += time.perf_counter() - t0
        lat.close()
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([t_batch, t_seq, t_one, float(fluid)], dtype=torch.float64, device="cuda")
        mx = tt.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = tt.clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        t_batch, t_seq, t_one, fluid = float(mx[0]), float(mx[1]), float(mx[2]), int(sm[3])
    cs_batch = n * steps / t_batch
    cs_seq = n * steps / t_seq
    return {"storage": {None: "workload's", 1: "FP32 planes", 3: "FP32 moments", 6: "FP32 in 32-node blocks",
                        7: "FP16 deviations in 32-node blocks"}.get(storage),
            "speedup_vs_single_lattice_path": cs_batch / cs_seq,
            "speedup_vs_one_launch_per_run": t_one / t_batch,
            "capillary_steps_per_s": cs_batch, "sequential_capillary_steps_per_s": cs_seq,
            "capillaries_per_s_at_20k_steps_extrapolated": cs_batch / 20000.0,
            "sequential_capillaries_per_s_at_20k_steps_extrapolated": cs_seq / 20000.0,
            "baselines": "single_lattice_path: each capillary its own lattice in the same storage on the "
                         "library's default kernel and tile (the staged kernel where it applies, bands of 16 "
                         "rows; 64-step CUDA graphs), run in turn; one_launch_per_run: each capillary alone "
                         "in the batch's persistent kernel and tile (a batch of one), launched in turn",
            "GLUPS_batched": fluid * steps / t_batch / 1e9, "fluid_nodes": fluid, "steps": steps,
            "tile": [tx, ty], "l_finite": bool(np.isfinite(out).all()),
            "what": f"{steps} steps with 4 l(t) samples, wall clock"}


def surrogate_metric(torch, threshold=0.02):
    """Train the 5-member l(t) surrogate on the LB-generated training runs (4096 of the
    seeded surrogate sweep), answer the 512 held-out queries, fall back to the LB where
    the ensemble spread exceeds 2 %, and compare with the LB and with Washburn's law."""
    from paper_0911_0459_gb300 import surrogate as S
    path = os.path.join(ROOT, "paper_0911_0459_gb300", "data", "surrogate_data.npz")
    if not os.path.exists(path):
        return {"unavailable": "no LB-generated training set (paper_0911_0459_gb300/data/surrogate_data.npz)"}
    d = np.load(path)
    test_caps = S.surrogate_sweep(2, int(d["l_test"].shape[0]))
    x_train, l_train, x_test, l_test = d["x_train"], d["l_train"], d["x_test"], d["l_test"]
    assert np.allclose(S.features(test_caps), x_test)
    sur = S.Surrogate(members=5, seed=0)
    t0 = time.perf_counter()
    sur.fit(x_train, l_train, steps=6000)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    t0 = time.perf_counter()
    pred, spread = sur.predict(x_test)
    t_pred = time.perf_counter() - t0
    fall = np.where(spread.max(1) > threshold)[0]
    t0 = time.perf_counter()
    lb_fall = S.run_lb([test_caps[i] for i in fall])["l"] if len(fall) else np.zeros((0, l_test.shape[1]))
    t_fall = time.perf_counter() - t0
    combined = pred.copy()
    combined[fall] = lb_fall
    # LB cost per query on this GPU: a batched run of 64 held-out queries, whose l(t) also
    # checks the stored held-out targets (the LB's own output) against this build and GPU
    probe = test_caps[:64]
    t0 = time.perf_counter()
    lb64 = S.run_lb(probe)["l"]
    t_lb64 = time.perf_counter() - t0
    lb_per_query = t_lb64 / len(probe)
    rel = np.abs(lb64 - l_test[:64]) / np.maximum(np.abs(l_test[:64]), 1.0)
    data_check = {"queries": len(probe), "max_rel_diff_stored_vs_fresh_lb": float(rel.max()),
                  "tolerance": DATASET_TOL, "ok": bool(rel.max() <= DATASET_TOL),
                  "rms_rel_vs_fresh_lb": S.rms_rel(pred[:64], lb64)}
    n = len(test_caps)
    sur.close()
    if not data_check["ok"]:
        return {"unavailable": "stored held-out l(t) differ from a fresh LB run beyond "
                               f"{DATASET_TOL}: {rel.max():.3g}", "dataset_check": data_check}
    return {"rms_rel_vs_lb": S.rms_rel(pred, l_test), "rms_rel_with_fallback": S.rms_rel(combined, l_test),
            "dataset_check": data_check,
            "fallback_fraction": len(fall) / n, "rms_rel_washburn": S.rms_rel(S.washburn(test_caps), l_test),
            "train_seconds": t_train, "inference_seconds": t_pred, "fallback_lb_seconds": t_fall,
            "lb_seconds_per_query": lb_per_query,
            "speedup_vs_lb": (lb_per_query * n) / (t_pred + t_fall), "queries": n,
            "what": "MLP 4-256-256-64, BF16 tensor cores, 5 members; l(t) at 64 log-spaced times to 20k steps"}


def small_capillary_rates(torch, Lattice, steps=10000):
    """The 2048 x 64 binary FP32 capillary (9.4 MB per state copy, held in L2): the
    autotuned single-lattice path (replayed 64-step graphs, CUDA events) in the 32-node
    block storage and in planes (the same bits), and one persistent launch of a batch of
    one (wall clock around the sampled run)."""
    from paper_0911_0459_gb300 import STORAGE_F32, STORAGE_F32_BLOCKED, Batch
    cap = W.config_binary_2048x64()
    rates = {}
    for key, st in (("blocks", STORAGE_F32_BLOCKED), ("planes", STORAGE_F32)):
        lat = Lattice.from_workload(cap, storage=st)
        tx, ty, _ = lat.autotune()
        lat.step(64)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(lat.stream)
        lat.step(steps)
        b.record(lat.stream)
        torch.cuda.synchronize()
        rates[key] = (1e3 * a.elapsed_time(b) / steps, [tx, ty], lat.kernel())
        fluid = lat.fluid_nodes
        lat.close()
    us, tile, kern = rates["blocks"]
    bt = Batch([cap])
    btx, bty, _ = bt.autotune(steps=2)
    bt.run_sampled([64])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bt.run_sampled([steps])
    us_p = 1e6 * (time.perf_counter() - t0) / steps
    bt.close()
    return {"us_per_step": us, "MLUPS": fluid / us, "tile": tile, "kernel_variant": kern,
            "storage": "FP32 in 32-node blocks",
            "planes_us_per_step": rates["planes"][0], "planes_tile": rates["planes"][1],
            "persistent_us_per_step": us_p, "persistent_MLUPS": fluid / us_p, "persistent_tile": [btx, bty],
            "what": f"{steps} steps; state in L2, so no HBM fraction is quoted; the persistent form is "
                    "a batch of one in planar FP32"}


def timed_steps(lat, torch, K, red_every):
    """K steps with reductions every red_every steps; returns (total_ms, step_ms, launches)."""
    s = lat.stream
    evs = []
    launches = 0
    done = 0
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(s)
    while done < K:
        n = min(red_every, K - done)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        lat.step(n)
        b.record(s)
        evs.append((a, b))
        launches += n
        done += n
        lat.filled_length()
        launches += 2
    t_end.record(s)
    torch.cuda.synchronize()
    total = t_start.elapsed_time(t_end)
    step_ms = sum(a.elapsed_time(b) for a, b in evs)
    return total, step_ms, launches


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile", default=None, help="BX,YC: fixed step-kernel tile instead of autotuning")
    ap.add_argument("--storage", default="f32b", choices=sorted(STORAGES))
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-sweep secondary metric")
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate secondary metric")
    ap.add_argument("--profile", action="store_true",
                    help="only the large capillary: warm-up then --steps steps (for ncu captures)")
    ap.add_argument("--workload", default="binary_16384x256", choices=["binary_16384x256", "lg_16384x256"],
                    help="with --profile: the lattice to run (lg_16384x256: the liquid-gas FP64 capillary)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_0911_0459_gb300 import (STORAGE_F16_BLOCKED, STORAGE_F16DEV, STORAGE_F32, STORAGE_F32_BLOCKED,
                                       STORAGE_F32_GELIM, STORAGE_MOMENTS, STORAGE_MOMENTS_F16, Lattice)

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    cap = W.config_binary_16384x256({"f32b": STORAGE_F32_BLOCKED, "f32": STORAGE_F32, "f16dev": STORAGE_F16DEV,
                                     "f16b": STORAGE_F16_BLOCKED, "moments": STORAGE_MOMENTS,
                                     "moments_f16": STORAGE_MOMENTS_F16, "gelim": STORAGE_F32_GELIM}[args.storage])
    if args.profile and args.workload == "lg_16384x256":
        cap = W.config_lg_16384x256()
    lat = Lattice.from_workload(cap)
    if args.tile:
        tx, ty = (int(v) for v in args.tile.split(","))
        lat.set_tile(tx, ty)
    else:
        tx, ty, us_tuned = lat.autotune()
    kernel_variant = lat.kernel()
    fluid = lat.fluid_nodes
    if args.profile:
        lat.step(args.warmup)
        lat.step(args.steps)
        lat.filled_length()
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": True, "steps": args.steps, "tile": [tx, ty]}), flush=True)
        lat.close()
        return
    lat.step(args.warmup)
    lat.filled_length()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        total_ms, step_ms, launches = timed_steps(lat, torch, args.steps, RED_EVERY)
    torch.cuda.synchronize()
    barrier()
    t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_max = float(t.item())
    value = world * fluid * args.steps / (total_max * 1e-3) / 1e6
    l_end = lat.filled_length()

    # roofline of the step kernel: algorithmic bytes = fluid nodes x the storage's bytes per update
    # (FP32: 18 planes x 4 B x (read + write))
    bytes_per_lu = STORAGES[args.storage][0]
    per_launch_ms = step_ms / args.steps
    achieved = fluid * bytes_per_lu / (per_launch_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    traffic = ncu_traffic("binary_" + args.storage, kernel_variant, [tx, ty]) if args.storage in ("f32", "f32b") \
        else None
    kernel_mlups = fluid / (per_launch_ms * 1e-3) / 1e6
    ceilings = {"144B": peak * 1e3 / 144.0, "48B": peak * 1e3 / 48.0}   # MLUPS at the measured peak

    # end to end through the C ABI with pinned host buffers: upload fields, K steps, download fields
    shape = (cap.ny, cap.nx)
    pinned = [torch.empty(shape, dtype=torch.float64, pin_memory=True) for _ in range(8)]
    rho0, ux0, uy0, phi0 = W.initial_fields(cap)
    for dst, src in zip(pinned[:4], (rho0, ux0, uy0, phi0)):
        dst.numpy()[:] = src
    host_in = [p.numpy() for p in pinned[:4]]
    host_out = [p.numpy() for p in pinned[4:]]
    from paper_0911_0459_gb300 import lb as lbmod
    import ctypes
    L = lbmod.library()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    lat.init_fields(*host_in)
    done = 0
    while done < args.steps:
        n = min(RED_EVERY, args.steps - done)
        lat.step(n)
        lat.filled_length()
        done += n
    st = L.lb_fields(lat.h, *[a.ctypes.data_as(ctypes.c_void_p) for a in host_out])
    assert st == 0
    e2e_s = time.perf_counter() - t0
    tt = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    e2e_s = float(tt.item())
    e2e = {"value": world * fluid * args.steps / e2e_s / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": 4 * 8 * cap.nx * cap.ny / args.steps,
           "d2h_bytes_per_step": 4 * 8 * cap.nx * cap.ny / args.steps,
           "what": "lb_init_fields(host) + K steps with lb_filled_length every 100 + lb_fields(host), "
                   "pinned buffers, wall clock"}

    # secondary numbers on the same GPU (not the headline)
    secondary = {}
    try:
        for key, st, bpl in (("fp32_planes_16384x256", STORAGE_F32, 144), ("fp32_blocks_16384x256", STORAGE_F32_BLOCKED, 144)):
            if st == cap.params.storage:
                continue
            lp = Lattice.from_workload(W.config_binary_16384x256(st))
            ptx, pty, _ = lp.autotune()
            lp.step(8)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(lp.stream)
            lp.step(512)
            b.record(lp.stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / 512
            gbs = lp.fluid_nodes * bpl / (ms * 1e-3) / 1e9
            secondary[key] = {"MLUPS": lp.fluid_nodes / (ms * 1e-3) / 1e6, "ms_per_step": ms, "tile": [ptx, pty],
                              "kernel": step_kernel_label(lp.kernel(), ptx, pty, "FP32" if st == STORAGE_F32 else "SF32B"),
                              "bytes_per_lu": bpl, "GBps": gbs, "frac_of_measured_hbm": gbs / peak,
                              "what": "the same FP32 populations and arithmetic (bit-identical states), the other "
                                      "layout; autotuned, 512 steps, CUDA events"}
            lp.close()
        for key, st, lbl, what in (
                ("fp16dev_16384x256", STORAGE_F16DEV, "FP16dev",
                 "FP16 f_i - w_i and g_1..g_8 in planes, FP32 g_0 plane"),
                ("fp16_blocks_16384x256", STORAGE_F16_BLOCKED, "SF16B",
                 "the same FP16 values in 32-node blocks (bit-identical states), one bulk copy per staged row")):
            l16 = Lattice.from_workload(W.config_binary_16384x256(st))
            htx, hty, _ = l16.autotune()
            l16.step(8)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(l16.stream)
            l16.step(512)
            b.record(l16.stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / 512
            gbs = l16.fluid_nodes * 76 / (ms * 1e-3) / 1e9
            secondary[key] = {"MLUPS": l16.fluid_nodes / (ms * 1e-3) / 1e6, "ms_per_step": ms, "tile": [htx, hty],
                              "kernel": step_kernel_label(l16.kernel(), htx, hty, lbl),
                              "bytes_per_lu": 76, "GBps": gbs, "frac_of_measured_hbm": gbs / peak,
                              "what": what + "; autotuned, 512 steps, CUDA events"}
            l16.close()
        c1 = W.config_lg_256x32()
        l1 = Lattice.from_workload(c1)
        l1.autotune()
        l1.step(64)
        torch.cuda.synchronize()
        a.record(l1.stream)
        l1.step(1984)
        b.record(l1.stream)
        torch.cuda.synchronize()
        secondary["lg_256x32_fp64_us_per_step"] = 1e3 * a.elapsed_time(b) / 1984
        l1.close()
        secondary["lg_16384x256_fp64"] = lg_fp64_roofline(torch, Lattice)
        secondary["binary_2048x64"] = small_capillary_rates(torch, Lattice)
        # the same large capillary with the reduced states of the pull kernel
        from paper_0911_0459_gb300 import STORAGE_F32_GELIM, STORAGE_MOMENTS_F16
        for key, st, bpl, what in (
                ("moments_16384x256", STORAGE_MOMENTS, 48,
                 "six FP32 moments per node (rho-1, j, pxx-pyy, pxy, phi)"),
                ("moments_f16_16384x256", STORAGE_MOMENTS_F16, 28,
                 "FP16 rho-1, j, pxx-pyy, pxy and FP32 phi per node"),
                ("g_eliminated_16384x256", STORAGE_F32_GELIM, 80,
                 "nine FP32 f populations and phi per node (g replaced by phi)")):
            lm = Lattice.from_workload(W.config_binary_16384x256(st))
            mtx, mty, _ = lm.autotune()
            lm.step(8)
            torch.cuda.synchronize()
            a.record(lm.stream)
            lm.step(512)
            b.record(lm.stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / 512
            gbs = lm.fluid_nodes * bpl / (ms * 1e-3) / 1e9
            secondary[key] = {
                "MLUPS": lm.fluid_nodes / (ms * 1e-3) / 1e6, "ms_per_step": ms, "tile": [mtx, mty],
                "bytes_per_lu": bpl, "GBps": gbs, "frac_of_measured_hbm": gbs / peak,
                "what": what + "; the pull kernel (moment_step_kernel), 512 steps, CUDA events; the same "
                               "update as the FP32 population kernel in exact arithmetic"}
            lm.close()
    except Exception as ex:  # secondary numbers never block the headline line
        secondary["error"] = repr(ex)
    if not args.no_batch:
        try:
            secondary["batched_sweep_256"] = batched_vs_sequential(torch, Lattice, args.batch_steps,
                                                                   storage=STORAGE_F32)
            # the same sweep in 32-node blocks (the same bits): the fastest batch, and faster
            # one-capillary baselines too
            secondary["batched_sweep_256_blocks"] = batched_vs_sequential(torch, Lattice, args.batch_steps,
                                                                          storage=STORAGE_F32_BLOCKED)
            secondary["batched_sweep_256_moments"] = batched_vs_sequential(torch, Lattice, args.batch_steps,
                                                                           storage=STORAGE_MOMENTS)
            secondary["batched_sweep_256_fp16_blocks"] = batched_vs_sequential(torch, Lattice, args.batch_steps,
                                                                               storage=STORAGE_F16_BLOCKED)
        except Exception as ex:
            secondary["batched_error"] = repr(ex)
    if not args.no_surrogate:
        try:
            secondary["surrogate"] = surrogate_metric(torch)
        except Exception as ex:
            secondary["surrogate_error"] = repr(ex)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, orc = cpu_baseline()
        try:
            secondary["precision_vs_oracle"] = precision_report(Lattice, orc, 2000)
        except Exception as ex:
            secondary["precision_error"] = repr(ex)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": bench_config(cap, world, args.storage),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": step_kernel_label(kernel_variant, tx, ty, STORAGES[args.storage][2]),
                         "bytes_per_lu": bytes_per_lu,
                         "peak_source": f"{peak_kind} copy bandwidth (HBM, burst)",
                         "us_per_launch": 1e3 * per_launch_ms,
                         "kernel_mlups": kernel_mlups,
                         "mlups_ceiling_144B": ceilings["144B"], "frac_of_144B_ceiling": kernel_mlups / ceilings["144B"],
                         "mlups_ceiling_48B": ceilings["48B"], "frac_of_48B_ceiling": kernel_mlups / ceilings["48B"],
                         "ceilings": "MLUPS the measured HBM peak allows at 144 B per fluid-node update (18 FP32 "
                                     "populations read and written) and at the method's minimum of 48 B (six "
                                     "FP32 moments: with S of App. A nothing else carries over a step)"},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "e2e": e2e,
            "l_end": l_end["l"],
            "secondary": secondary,
        }
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    lat.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
