"""lb_filled_length_noalloc against lb_filled_length (needs a GPU).

The allocation-free entry point serves callers that cannot allocate device
memory (a framework that owns all device buffers, a loop that must not call
cudaMalloc); it keeps its partial sums in a static device array instead of
context memory.  This file is collected last so that a run stopping at the first
failure has already run every other test; it passes on its own in a fresh
process (where its first call resolves the scratch address) and after the rest.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0911_0459_gb300 import STORAGE_F32, STORAGE_F64, Lattice  # noqa: E402
from paper_0911_0459_gb300 import lb as lbmod  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MAX_BLOCKS = int(re.search(r"#define\s+LB_NOALLOC_MAX_BLOCKS\s+(\d+)",
                           open(os.path.join(ROOT, "include", "lb.h")).read()).group(1))
REL_TOL = 1e-12   # same kernels and summation order as lb_filled_length up to the block count


def noalloc_fn():
    fn = lbmod.library().lb_filled_length_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.POINTER(lbmod.LbGrid), C.POINTER(lbmod.LbWalls), C.POINTER(lbmod.LbParams),
                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    return fn


def device_state(lat, storage):
    """The lattice's stored state copied into caller-owned device tensors in the library layout."""
    f, g = lat.populations(rested=False)
    dt = torch.float64 if storage == STORAGE_F64 else torch.float32
    fd = torch.tensor(f, dtype=dt, device="cuda").contiguous()
    gd = torch.tensor(g, dtype=dt, device="cuda").contiguous() if g is not None else None
    return fd, gd


def call(lat, fd, gd, nblocks, out):
    fn = noalloc_fn()
    stream = torch.cuda.current_stream()
    st = fn(C.byref(lat.grid), C.byref(lat.walls), C.byref(lat.params), C.c_void_p(fd.data_ptr()),
            C.c_void_p(gd.data_ptr() if gd is not None else 0), None, int(nblocks),
            C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
    return st


def check(got, ref):
    for k, v in zip(("l", "l_vol", "mass", "phi_sum"), got):
        r = ref[k]
        assert abs(v - r) <= REL_TOL * max(1.0, abs(r)), (k, v, r)


def test_noalloc_matches_filled_length_on_two_calls_in_a_row():
    binary = W.Capillary("na", 300, 36, 60, 230, 4, 28, 20, 10, W.binary_params(nu_l=0.5, nu_g=0.05),
                         theta_deg=50.0)
    lg = W.config_lg_256x32()
    a = Lattice.from_workload(binary, storage=STORAGE_F32)
    a.step(137)
    b = Lattice.from_workload(lg)
    b.step(91)
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    # first call: the largest block count the scratch allows
    fa, ga = device_state(a, STORAGE_F32)
    assert call(a, fa, ga, MAX_BLOCKS, out) == lbmod.LB_OK
    torch.cuda.synchronize()
    check(out.cpu().numpy(), a.filled_length())
    # second call on another lattice with few blocks: stale partials of the first
    # call beyond its block count must not leak into the result
    fb, _ = device_state(b, STORAGE_F64)
    out2 = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    assert call(b, fb, None, 37, out2) == lbmod.LB_OK
    torch.cuda.synchronize()
    check(out2.cpu().numpy(), b.filled_length())
    # block counts beyond the scratch are refused
    assert call(a, fa, ga, MAX_BLOCKS + 1, out) == lbmod.LB_ERR_ARG
    assert call(a, fa, ga, 0, out) == lbmod.LB_ERR_ARG
    a.close()
    b.close()


def test_noalloc_reads_the_fp16_deviation_layout():
    """A caller-owned state in the FP16 layout the header documents: f_i - w_i rho0 in FP16
    with the bulk rest weights of the lattice's A (P0 = 1/3 + A/4), g_1..g_8 in FP16, g_0 in
    FP32.  The state is the lattice's own, rebuilt from its populations."""
    from paper_0911_0459_gb300 import STORAGE_F16DEV
    cap = W.Capillary("nh", 300, 36, 60, 230, 4, 28, 20, 10,
                      W.binary_params(nu_l=0.5, nu_g=0.05, A=0.035, kappa=0.035, storage=STORAGE_F16DEV),
                      theta_deg=50.0)
    lat = Lattice.from_workload(cap)
    lat.step(120)
    f, g = lat.populations(rested=False)
    P0 = 1.0 / 3.0 + 0.25 * cap.params.A
    w = np.array([1 - 5 * P0 / 3] + [P0 / 3] * 4 + [P0 / 12] * 4, dtype=np.float32)
    dev = (f.astype(np.float32) - w[:, None, None]).astype(np.float16)
    fd = torch.tensor(dev, device="cuda").contiguous()
    gd = torch.tensor(g[1:].astype(np.float16), device="cuda").contiguous()
    g0d = torch.tensor(g[0].astype(np.float32), device="cuda").contiguous()
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    fn = noalloc_fn()
    st = fn(C.byref(lat.grid), C.byref(lat.walls), C.byref(lat.params), C.c_void_p(fd.data_ptr()),
            C.c_void_p(gd.data_ptr()), C.c_void_p(g0d.data_ptr()), 64, C.c_void_p(out.data_ptr()),
            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == lbmod.LB_OK
    torch.cuda.synchronize()
    ref = lat.filled_length()
    for k, v in zip(("l", "l_vol", "mass", "phi_sum"), out.cpu().numpy()):
        assert abs(v - ref[k]) <= 1e-9 * max(1.0, abs(ref[k])), (k, v, ref[k])


def test_noalloc_wrapped_liquid_gas_tube_and_argument_errors():
    """A liquid-gas FP32 state whose tube starts at a nonzero offset and wraps through
    x = 0 (with a y offset) gives lb_filled_length's values; the header's argument errors
    (moment storage, binary without g, FP16 without g0) return LB_ERR_ARG with real
    device pointers too, and leave the output untouched."""
    from paper_0911_0459_gb300 import STORAGE_F16DEV, STORAGE_MOMENTS
    cap = W.Capillary("lw", 160, 24, 120, 100, 3, 18, 8, 10, W.lg_params(storage=STORAGE_F32), wall_grad=-0.1)
    lat = Lattice.from_workload(cap)
    lat.step(57)
    fd, _ = device_state(lat, STORAGE_F32)
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    assert call(lat, fd, None, 96, out) == lbmod.LB_OK
    torch.cuda.synchronize()
    check(out.cpu().numpy(), lat.filled_length())
    lat.close()
    binary = W.Capillary("nb", 300, 36, 60, 230, 4, 28, 20, 10, W.binary_params(), theta_deg=50.0)
    b = Lattice.from_workload(binary)
    fb, gb = device_state(b, STORAGE_F32)
    sentinel = torch.full((4,), 7.0, dtype=torch.float64, device="cuda")
    fn = noalloc_fn()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def status(params, g, g0):
        return fn(C.byref(b.grid), C.byref(b.walls), C.byref(params), C.c_void_p(fb.data_ptr()), g, g0, 64,
                  C.c_void_p(sentinel.data_ptr()), stream)
    pm = lbmod.LbParams.from_buffer_copy(b.params)
    pm.storage = STORAGE_MOMENTS
    assert status(pm, C.c_void_p(gb.data_ptr()), None) == lbmod.LB_ERR_ARG
    assert status(b.params, None, None) == lbmod.LB_ERR_ARG
    ph = lbmod.LbParams.from_buffer_copy(b.params)
    ph.storage = STORAGE_F16DEV
    assert status(ph, C.c_void_p(gb.data_ptr()), None) == lbmod.LB_ERR_ARG
    torch.cuda.synchronize()
    assert (sentinel.cpu().numpy() == 7.0).all()
    b.close()


@pytest.mark.parametrize("storage_name", ["STORAGE_F32_BLOCKED", "STORAGE_F16_BLOCKED"])
def test_noalloc_reads_the_block_layouts(storage_name):
    """A caller-owned state in a block storage's layout: the bytes lb_save_state writes,
    copied into a device buffer the caller owns, with g and g0 not passed (the layout
    places them).  The same values as lb_filled_length, up to the order of the partial sums."""
    from paper_0911_0459_gb300 import lb as L
    storage = getattr(L, storage_name)
    cap = W.Capillary("nb", 203, 36, 61, 130, 4, 28, 20, 10,
                      W.binary_params(nu_l=0.5, nu_g=0.05, storage=storage), theta_deg=50.0)
    lat = Lattice.from_workload(cap)
    lat.step(120)
    buf, _ = lat.save_state()
    fd = torch.tensor(np.frombuffer(buf.tobytes(), dtype=np.uint8), device="cuda")
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    fn = noalloc_fn()
    st = fn(C.byref(lat.grid), C.byref(lat.walls), C.byref(lat.params), C.c_void_p(fd.data_ptr()), None, None,
            97, C.c_void_p(out.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == lbmod.LB_OK
    torch.cuda.synchronize()
    check(out.cpu().numpy(), lat.filled_length())
    lat.close()
