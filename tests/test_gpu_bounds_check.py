"""The bounds-checked debug build (-DLB_CHECK) on every storage and step kernel (needs a GPU).

In that build every global load and store of the step kernels checks its index against
its buffer; an index outside would be counted and skipped.  Small lattices of every
model and storage run through every step kernel (the staged and the sliding-window
population kernels with both ring depths, on the planar storages and on the 32-node
block storages (FP32 and FP16) with aligned and unaligned rows, the pull kernel of the reduced states) and
through the batch bodies, in a child process that loads the checked library; every
counter must stay at zero, and the states must equal bit for bit those of the normal
build (the checks change nothing for accesses inside their buffers)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r'''
import hashlib, json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import workloads as W
from paper_0911_0459_gb300 import Batch, Lattice
out = {}

def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()[:16]

def lattice(name, cap, storage, variants, tiles):
    lat = Lattice.from_workload(cap, storage=storage)
    for v in variants:
        lat.set_kernel(v)
        for tx, ty in tiles:
            lat.set_tile(tx, min(ty, cap.ny))
            lat.step(5)
    lat.step(70)                 # a replayed graph as well
    d = lat.filled_length()
    out[name] = {"check": lat.check_report(), "state": digest(lat.save_state()[0]), "l": d["l"]}
    lat.close()

tiles = ((64, 3), (128, 8), (256, 16))
bp = W.binary_params(nu_l=0.5, nu_g=0.05)
cap8 = W.Capillary("c8", 200, 37, 64, 120, 5, 27, 12, 8, bp, theta_deg=50.0)     # nx % 8 == 0: staged fits
capw = W.Capillary("cw", 144, 30, 104, 90, 27, 20, 0, 0, bp, wall_grad=-0.1)      # tube through x = 0
capr = W.Capillary("cr", 203, 37, 61, 120, 5, 27, 12, 8, bp, wall_grad=-0.11)     # ragged nx
narrow = W.Capillary("nw", 20, 12, 6, 10, 2, 7, 2, 3, bp, wall_grad=-0.2)
for st in (0, 1, 2):             # FP64, FP32, FP16 deviations: sliding window, staged shallow and deep
    for nm, c in (("c8", cap8), ("cw", capw)):
        lattice(f"bin{st}_{nm}", c, st, (1, 2, 3), tiles)
    lattice(f"bin{st}_cr", capr, st, (1,), tiles)
cap96 = W.Capillary("c9", 96, 24, 24, 64, 3, 18, 8, 6, bp, theta_deg=45.0)       # nx % 32 == 0
tail = W.Capillary("ct", 513, 9, 100, 300, 1, 6, 20, 10, bp, wall_grad=-0.1)      # one-column last tile
for nm, c in (("c96", cap96), ("cw", capw), ("cr", capr), ("nw", narrow), ("ct", tail)):
    # FP32 and FP16 in 32-node blocks: aligned and unaligned rows, every kernel variant
    lattice(f"blk_{nm}", c, 6, (1, 2, 3), tiles)
    lattice(f"blk16_{nm}", c, 7, (1, 2, 3), tiles)
for st in (3, 4, 5):             # the pull kernel's reduced states
    for nm, c in (("c8", cap8), ("cw", capw), ("cr", capr), ("nw", narrow)):
        lattice(f"pull{st}_{nm}", c, st, (4,), tiles)
lg = W.config_lg_256x32()
for st in (0, 1):
    lattice(f"lg{st}", lg, st, (1, 2, 3), tiles)
# batch bodies: sliding window (ragged nx), staged (aligned nx), moments
caps = W.sweep(seed=3, n=6, steps=100)
for st, key in ((1, "batch_f32"), (2, "batch_f16"), (3, "batch_moments")):
    b = Batch(caps + [capr], storage=st)
    for v in ((1, 2, 3) if st != 3 else (4,)):
        if st != 3 and v > 1:
            continue         # the ragged lattice keeps this batch on the sliding-window body
        b.set_tile(128, 16)
        b.step(7)
    b.run_sampled([3, 9])
    out[key] = {"check": b.check_report(), "state": digest(b.save_state()[0])}
    b.close()
b = Batch(caps, storage=1)   # aligned rows: the staged body, both ring depths
for v in (2, 3):
    b.set_kernel(v)
    b.step(7)
out["batch_f32_staged"] = {"check": b.check_report(), "state": digest(b.save_state()[0])}
b.close()
for st, key in ((6, "batch_blk32"), (7, "batch_blk16")):   # block storages: staged at any nx
    b = Batch(caps + [capr], storage=st)
    for v in (1, 2, 3):
        b.set_kernel(v)
        b.set_tile(128, 16)
        b.step(7)
    b.run_sampled([3, 9])
    out[key] = {"check": b.check_report(), "state": digest(b.save_state()[0])}
    b.close()
print(json.dumps(out))
'''


def run(lib=None):
    env = dict(os.environ)
    env.pop("LB_GB300_LIBRARY", None)
    if lib:
        env["LB_GB300_LIBRARY"] = lib
    r = subprocess.run([sys.executable, "-c", RUN, ROOT], capture_output=True, text=True, env=env,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_no_access_leaves_its_buffer_and_the_checks_change_nothing():
    from paper_0911_0459_gb300 import build
    lib = build.build(variant="check")
    checked = run(lib)
    plain = run()
    for name, rec in checked.items():
        enabled, bad, first = rec["check"]
        assert enabled == 1, name
        assert bad == 0, (name, bad, first - 1)
        assert plain[name]["check"][0] == 0, name        # the normal build reports nothing
        assert rec["state"] == plain[name]["state"], name
