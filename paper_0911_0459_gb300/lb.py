"""Python binding of include/lb.h (argument marshalling only).

Every step of the method runs in the CUDA library _lib/liblbgb300.so; this
module converts arrays and structs and checks status codes.  Device memory comes
from PyTorch's caching allocator through the lb_alloc callbacks and work is
issued on the current PyTorch CUDA stream.  There is no CPU fallback: if the
library has not been built, importing a Lattice raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# LB_GB300_LIBRARY selects another build of the same library (the bounds-checked one)
LIB_PATH = os.environ.get("LB_GB300_LIBRARY") or os.path.join(_PKG, "_lib", "liblbgb300.so")

LB_OK, LB_ERR_ARG, LB_ERR_CUDA, LB_ERR_NONFINITE, LB_ERR_TIMEOUT, LB_ERR_STATE, LB_ERR_NOMEM = range(7)
STATUS_NAMES = ["LB_OK", "LB_ERR_ARG", "LB_ERR_CUDA", "LB_ERR_NONFINITE", "LB_ERR_TIMEOUT",
                "LB_ERR_STATE", "LB_ERR_NOMEM"]
MODEL_LIQUID_GAS, MODEL_BINARY = 0, 1
STORAGE_F64, STORAGE_F32, STORAGE_F16DEV, STORAGE_MOMENTS = 0, 1, 2, 3
STORAGE_MOMENTS_F16, STORAGE_F32_GELIM, STORAGE_F32_BLOCKED, STORAGE_F16_BLOCKED = 4, 5, 6, 7


class LbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class LbGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int)]


class LbWalls(C.Structure):
    _fields_ = [("tube_x0", C.c_int), ("tube_len", C.c_int), ("tube_y0", C.c_int), ("tube_h", C.c_int),
                ("gas_cols", C.c_int), ("wall_grad", C.c_double)]


class LbParams(C.Structure):
    _fields_ = [("model", C.c_int), ("storage", C.c_int),
                ("kappa", C.c_double), ("a", C.c_double), ("b", C.c_double), ("T", C.c_double),
                ("A", C.c_double), ("M", C.c_double), ("nu_l", C.c_double), ("nu_g", C.c_double),
                ("nu", C.c_double), ("lambda_scale", C.c_double),
                ("rho_l", C.c_double), ("rho_g", C.c_double), ("l0", C.c_int), ("nu_table", C.c_int)]


MALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class LbAlloc(C.Structure):
    _fields_ = [("malloc_fn", MALLOC_FN), ("free_fn", FREE_FN), ("user", C.c_void_p)]


_lib = None


def library():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build() "
                           "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    vp, dp = C.c_void_p, C.c_void_p
    sig = {
        "lb_create": (C.c_int, [C.POINTER(LbGrid), C.POINTER(LbWalls), C.POINTER(LbParams),
                                C.POINTER(LbAlloc), vp, C.POINTER(vp)]),
        "lb_destroy": (None, [vp]),
        "lb_init_fields": (C.c_int, [vp, dp, dp, dp, dp]),
        "lb_step": (C.c_int, [vp, C.c_long]),
        "lb_fields": (C.c_int, [vp, dp, dp, dp, dp]),
        "lb_filled_length": (C.c_int, [vp] + [C.POINTER(C.c_double)] * 4),
        "lb_get_populations": (C.c_int, [vp, dp, dp, C.c_int]),
        "lb_get_moments": (C.c_int, [vp, dp]),
        "lb_set_populations": (C.c_int, [vp, dp, dp]),
        "lb_sync": (C.c_int, [vp]),
        "lb_inject_wait_timeout": (C.c_int, [vp]),
        "lb_check_report": (C.c_int, [vp, C.POINTER(C.c_int), C.POINTER(C.c_ulonglong), C.POINTER(C.c_ulonglong)]),
        "lb_batch_check_report": (C.c_int, [vp, C.POINTER(C.c_int), C.POINTER(C.c_ulonglong),
                                            C.POINTER(C.c_ulonglong)]),
        "lb_state_bytes": (C.c_size_t, [vp]),
        "lb_save_state": (C.c_int, [vp, vp, C.c_size_t]),
        "lb_load_state": (C.c_int, [vp, vp, C.c_size_t, C.c_long]),
        "lb_time": (C.c_long, [vp]),
        "lb_fluid_nodes": (C.c_long, [vp]),
        "lb_set_tile": (C.c_int, [vp, C.c_int, C.c_int]),
        "lb_set_kernel": (C.c_int, [vp, C.c_int]),
        "lb_get_kernel": (C.c_int, [vp, C.POINTER(C.c_int)]),
        "lb_get_tile": (C.c_int, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "lb_autotune": (C.c_int, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]),
        "lb_last_error": (C.c_char_p, [vp]),
        "lb_batch_create": (C.c_int, [C.c_int, C.POINTER(LbGrid), C.POINTER(LbWalls), C.POINTER(LbParams),
                                      C.POINTER(LbAlloc), vp, C.POINTER(vp)]),
        "lb_batch_destroy": (None, [vp]),
        "lb_batch_step": (C.c_int, [vp, C.c_long]),
        "lb_batch_lengths": (C.c_int, [vp, dp]),
        "lb_batch_run_sampled": (C.c_int, [vp, C.c_int, dp, dp]),
        "lb_batch_populations": (C.c_int, [vp, C.c_int, dp, dp, C.c_int]),
        "lb_batch_moments": (C.c_int, [vp, C.c_int, dp]),
        "lb_batch_set_tile": (C.c_int, [vp, C.c_int, C.c_int]),
        "lb_batch_autotune": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                        C.POINTER(C.c_double)]),
        "lb_batch_set_barrier": (C.c_int, [vp, C.c_uint, C.c_double]),
        "lb_batch_set_kernel": (C.c_int, [vp, C.c_int]),
        "lb_batch_get_kernel": (C.c_int, [vp, C.POINTER(C.c_int)]),
        "lb_batch_time": (C.c_long, [vp]),
        "lb_batch_fluid_nodes": (C.c_long, [vp, C.c_int]),
        "lb_batch_last_error": (C.c_char_p, [vp]),
        "lb_batch_state_bytes": (C.c_size_t, [vp]),
        "lb_batch_save_state": (C.c_int, [vp, vp, C.c_size_t]),
        "lb_batch_load_state": (C.c_int, [vp, vp, C.c_size_t, C.c_long]),
        "lb_fp64_fma_rate": (C.c_int, [vp, C.POINTER(C.c_double)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def exported_symbols():
    return ["lb_create", "lb_destroy", "lb_init_fields", "lb_step", "lb_fields", "lb_filled_length",
            "lb_get_populations", "lb_set_populations", "lb_get_moments", "lb_sync", "lb_inject_wait_timeout",
            "lb_check_report", "lb_batch_check_report", "lb_time", "lb_fluid_nodes",
            "lb_set_tile", "lb_get_tile", "lb_autotune", "lb_last_error", "lb_set_kernel", "lb_get_kernel",
            "lb_batch_create", "lb_batch_destroy", "lb_batch_step", "lb_batch_lengths", "lb_batch_run_sampled",
            "lb_batch_populations", "lb_batch_moments", "lb_batch_set_tile", "lb_batch_autotune", "lb_batch_set_barrier",
            "lb_batch_set_kernel", "lb_batch_get_kernel", "lb_batch_time", "lb_batch_fluid_nodes", "lb_batch_last_error",
            "lb_state_bytes", "lb_save_state", "lb_load_state", "lb_batch_state_bytes", "lb_batch_save_state",
            "lb_batch_load_state", "lb_fp64_fma_rate"]


def fp64_fma_rate(stream=None):
    """The device's measured FP64 fused multiply-add rate in TFLOP/s (lb_fp64_fma_rate),
    on a torch stream (default: the current one)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    v = C.c_double()
    status = library().lb_fp64_fma_rate(C.c_void_p(st.cuda_stream), C.byref(v))
    if status != LB_OK:
        raise LbError(status, "lb_fp64_fma_rate failed")
    return v.value


class _TorchAllocator:
    """lb_alloc backed by torch's CUDA caching allocator."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device

        def _malloc(nbytes, stream, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream))
            except Exception:  # allocation failure is reported to the library as NULL
                return None

        def _free(ptr, stream, user):
            if ptr:
                torch.cuda.caching_allocator_delete(int(ptr))

        self._m = MALLOC_FN(_malloc)
        self._f = FREE_FN(_free)
        self.struct = LbAlloc(self._m, self._f, None)


def _check(status, ctx):
    if status != LB_OK:
        msg = library().lb_last_error(ctx).decode(errors="replace")
        raise LbError(status, msg)


def _host(a, shape):
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if out.shape != shape:
        raise ValueError(f"expected shape {shape}, got {out.shape}")
    return out


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Lattice:
    """One lattice on the current CUDA device, owned by the C library."""

    def __init__(self, nx, ny, *, model, storage, tube_x0=0, tube_len=0, tube_y0=0, tube_h=None,
                 gas_cols=0, wall_grad=0.0, kappa=0.04, a=9 / 49, b=2 / 21, T=0.56, A=0.04, M=0.1,
                 nu_l=1 / 6, nu_g=1 / 6, nu=1 / 6, lambda_scale=1.0, rho_l=4.54, rho_g=2.59, l0=10,
                 nu_table=0, stream=None, use_torch_allocator=True):
        import torch
        L = library()
        if tube_h is None:
            tube_h = ny
        self.nx, self.ny, self.model = int(nx), int(ny), int(model)
        self.grid = LbGrid(self.nx, self.ny)
        self.walls = LbWalls(int(tube_x0), int(tube_len), int(tube_y0), int(tube_h), int(gas_cols),
                             float(wall_grad))
        self.params = LbParams(int(model), int(storage), kappa, a, b, T, A, M, nu_l, nu_g, nu,
                               lambda_scale, rho_l, rho_g, int(l0), int(nu_table))
        dev = torch.cuda.current_device()
        self._torch_stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._alloc = _TorchAllocator(dev) if use_torch_allocator else None
        h = C.c_void_p()
        st = L.lb_create(C.byref(self.grid), C.byref(self.walls), C.byref(self.params),
                         C.byref(self._alloc.struct) if self._alloc else None,
                         C.c_void_p(self._torch_stream.cuda_stream), C.byref(h))
        if st != LB_OK:
            raise LbError(st, L.lb_last_error(None).decode(errors="replace"))
        self.h = h

    @classmethod
    def from_workload(cls, cap, storage=None, **kw):
        """Build from a workloads.Capillary description."""
        p = cap.params
        wg = cap.wall_gradient()
        return cls(cap.nx, cap.ny, model=p.model, storage=p.storage if storage is None else storage,
                   tube_x0=cap.tube_x0, tube_len=cap.tube_len, tube_y0=cap.tube_y0, tube_h=cap.tube_h,
                   gas_cols=cap.gas_cols, wall_grad=wg, kappa=p.kappa, a=p.a, b=p.b, T=p.T, A=p.A,
                   M=p.M, nu_l=p.nu_l, nu_g=p.nu_g, nu=p.nu, lambda_scale=p.lambda_scale,
                   rho_l=p.rho_l, rho_g=p.rho_g, l0=cap.l0, nu_table=p.nu_table, **kw)

    def close(self):
        if getattr(self, "h", None) is not None:
            library().lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.ny, self.nx)

    @property
    def stream(self):
        return self._torch_stream

    def init_fields(self, rho, ux, uy, phi=None):
        s = self.shape
        arrs = [_host(rho, s), _host(ux, s), _host(uy, s), None if phi is None else _host(phi, s)]
        _check(library().lb_init_fields(self.h, *[_p(a) for a in arrs]), self.h)
        return self

    def step(self, n=1):
        _check(library().lb_step(self.h, int(n)), self.h)
        return self

    def check_report(self):
        """Bounds-checked build: (enabled, bad accesses, first bad index + 1) since the last call."""
        e, b, f = C.c_int(), C.c_ulonglong(), C.c_ulonglong()
        _check(library().lb_check_report(self.h, C.byref(e), C.byref(b), C.byref(f)), self.h)
        return e.value, b.value, f.value

    def inject_wait_timeout(self):
        """Failure injection for tests: mark the device error word as a timed-out wait does."""
        _check(library().lb_inject_wait_timeout(self.h), self.h)

    def sync(self):
        _check(library().lb_sync(self.h), self.h)

    @property
    def time(self):
        return library().lb_time(self.h)

    @property
    def fluid_nodes(self):
        return library().lb_fluid_nodes(self.h)

    def fields(self):
        out = [np.empty(self.shape) for _ in range(4)]
        _check(library().lb_fields(self.h, *[_p(a) for a in out]), self.h)
        rho, ux, uy, phi = out
        return rho, ux, uy, (phi if self.model == MODEL_BINARY else None)

    def filled_length(self):
        v = [C.c_double() for _ in range(4)]
        _check(library().lb_filled_length(self.h, *[C.byref(x) for x in v]), self.h)
        return {"l": v[0].value, "l_vol": v[1].value, "mass": v[2].value, "phi_sum": v[3].value}

    def populations(self, rested=True):
        f = np.empty((9,) + self.shape)
        g = np.empty((9,) + self.shape) if self.model == MODEL_BINARY else None
        _check(library().lb_get_populations(self.h, _p(f), _p(g), int(bool(rested))), self.h)
        return f, g

    def moments(self):
        """(6, ny, nx): rho, jx, jy, pxx - pyy, pxy, phi of the stored state (before
        the boundary-node rest rule)."""
        m = np.empty((6,) + self.shape)
        _check(library().lb_get_moments(self.h, _p(m)), self.h)
        return m

    def save_state(self):
        """Checkpoint: (bytes of the stored state as a uint8 array, step count)."""
        L = library()
        buf = np.empty(L.lb_state_bytes(self.h), dtype=np.uint8)
        _check(L.lb_save_state(self.h, buf.ctypes.data_as(C.c_void_p), buf.nbytes), self.h)
        return buf, self.time

    def load_state(self, buf, time):
        """Resume from save_state's bytes (a lattice of the same description)."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(library().lb_load_state(self.h, buf.ctypes.data_as(C.c_void_p), buf.nbytes, int(time)), self.h)
        return self

    def save(self, path):
        """save_state to an .npz file, with the grid, model and storage that must match on load."""
        buf, t = self.save_state()
        np.savez(path, state=buf, time=t, nx=self.grid.nx, ny=self.grid.ny, model=self.params.model,
                 storage=self.params.storage)

    def load(self, path):
        d = np.load(path)
        if (int(d["nx"]), int(d["ny"]), int(d["model"]), int(d["storage"])) != \
                (self.grid.nx, self.grid.ny, self.params.model, self.params.storage):
            raise ValueError(f"{path}: checkpoint of another grid, model or storage")
        return self.load_state(d["state"], int(d["time"]))

    def set_populations(self, f, g=None):
        s = (9,) + self.shape
        f = _host(f, s)
        g = None if g is None else _host(g, s)
        _check(library().lb_set_populations(self.h, _p(f), _p(g)), self.h)
        return self

    def set_tile(self, tx, ty):
        _check(library().lb_set_tile(self.h, int(tx), int(ty)), self.h)

    def set_kernel(self, variant):
        """0 automatic, 1 sliding-window kernel, 2 / 3 staged (bulk-copy) kernel with
        its shallow / deep ring."""
        _check(library().lb_set_kernel(self.h, int(variant)), self.h)

    def kernel(self):
        v = C.c_int()
        _check(library().lb_get_kernel(self.h, C.byref(v)), self.h)
        return v.value

    def tile(self):
        a, b = C.c_int(), C.c_int()
        _check(library().lb_get_tile(self.h, C.byref(a), C.byref(b)), self.h)
        return a.value, b.value

    def autotune(self):
        a, b, us = C.c_int(), C.c_int(), C.c_double()
        _check(library().lb_autotune(self.h, C.byref(a), C.byref(b), C.byref(us)), self.h)
        return a.value, b.value, us.value


def _structs_for(cap, storage=None):
    """lb_grid / lb_walls / lb_params for a workloads.Capillary description."""
    p = cap.params
    wg = cap.wall_gradient()
    grid = LbGrid(cap.nx, cap.ny)
    walls = LbWalls(cap.tube_x0, cap.tube_len, cap.tube_y0, cap.tube_h, cap.gas_cols, float(wg))
    params = LbParams(p.model, p.storage if storage is None else storage, p.kappa, p.a, p.b, p.T, p.A, p.M,
                      p.nu_l, p.nu_g, p.nu, p.lambda_scale, p.rho_l, p.rho_g, int(cap.l0),
                      int(p.nu_table))
    return grid, walls, params


def _bcheck(status, h):
    if status != LB_OK:
        raise LbError(status, library().lb_batch_last_error(h).decode(errors="replace"))


class Batch:
    """Many binary capillaries advanced together by one persistent kernel."""

    def __init__(self, caps, storage=None, stream=None, use_torch_allocator=True):
        import torch
        L = library()
        n = len(caps)
        structs = [_structs_for(c, storage) for c in caps]
        self.grids = (LbGrid * n)(*[s[0] for s in structs])
        self.walls = (LbWalls * n)(*[s[1] for s in structs])
        self.params = (LbParams * n)(*[s[2] for s in structs])
        self.caps = list(caps)
        self.n = n
        dev = torch.cuda.current_device()
        self._torch_stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._alloc = _TorchAllocator(dev) if use_torch_allocator else None
        h = C.c_void_p()
        st = L.lb_batch_create(n, self.grids, self.walls, self.params,
                               C.byref(self._alloc.struct) if self._alloc else None,
                               C.c_void_p(self._torch_stream.cuda_stream), C.byref(h))
        if st != LB_OK:
            raise LbError(st, L.lb_batch_last_error(None).decode(errors="replace"))
        self.h = h

    @property
    def stream(self):
        return self._torch_stream

    def check_report(self):
        """Bounds-checked build: (enabled, bad accesses, first bad index + 1) of the batch kernels."""
        e, b, f = C.c_int(), C.c_ulonglong(), C.c_ulonglong()
        L = library()
        st = L.lb_batch_check_report(self.h, C.byref(e), C.byref(b), C.byref(f))
        if st != LB_OK:
            raise LbError(st, L.lb_batch_last_error(self.h).decode(errors="replace"))
        return e.value, b.value, f.value

    def close(self):
        if getattr(self, "h", None) is not None:
            library().lb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n):
        _bcheck(library().lb_batch_step(self.h, int(n)), self.h)
        return self

    def lengths(self):
        out = np.empty((self.n, 4))
        _bcheck(library().lb_batch_lengths(self.h, _p(out)), self.h)
        return out

    def run_sampled(self, at):
        at = np.ascontiguousarray(np.asarray(at, dtype=np.int64))
        out = np.empty((self.n, len(at), 4))
        _bcheck(library().lb_batch_run_sampled(self.h, len(at), at.ctypes.data_as(C.c_void_p), _p(out)), self.h)
        return out

    def populations(self, i, rested=True):
        c = self.caps[i]
        f = np.empty((9, c.ny, c.nx))
        g = np.empty((9, c.ny, c.nx))
        _bcheck(library().lb_batch_populations(self.h, int(i), _p(f), _p(g), int(bool(rested))), self.h)
        return f, g

    def moments(self, i):
        """(6, ny, nx) moments of lattice i, as Lattice.moments."""
        c = self.caps[i]
        m = np.empty((6, c.ny, c.nx))
        _bcheck(library().lb_batch_moments(self.h, int(i), _p(m)), self.h)
        return m

    def save_state(self):
        """Checkpoint of every lattice: (bytes of the batch's state as a uint8 array, step count)."""
        L = library()
        buf = np.empty(L.lb_batch_state_bytes(self.h), dtype=np.uint8)
        _bcheck(L.lb_batch_save_state(self.h, buf.ctypes.data_as(C.c_void_p), buf.nbytes), self.h)
        return buf, self.time

    def load_state(self, buf, time):
        """Resume from save_state's bytes (a batch of the same lattices and storage)."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _bcheck(library().lb_batch_load_state(self.h, buf.ctypes.data_as(C.c_void_p), buf.nbytes, int(time)),
                self.h)
        return self

    def set_tile(self, tx, ty):
        _bcheck(library().lb_batch_set_tile(self.h, int(tx), int(ty)), self.h)

    def autotune(self, steps=4):
        a, b, ms = C.c_int(), C.c_int(), C.c_double()
        _bcheck(library().lb_batch_autotune(self.h, int(steps), C.byref(a), C.byref(b), C.byref(ms)), self.h)
        return a.value, b.value, ms.value

    def set_barrier(self, absent_blocks=0, limit_seconds=2.0):
        _bcheck(library().lb_batch_set_barrier(self.h, int(absent_blocks), float(limit_seconds)), self.h)

    def set_kernel(self, variant):
        """0 automatic, 1 sliding-window body, 2 / 3 staged body with its shallow /
        deep ring (every nx % 8 == 0)."""
        _bcheck(library().lb_batch_set_kernel(self.h, int(variant)), self.h)

    def kernel(self):
        v = C.c_int()
        _bcheck(library().lb_batch_get_kernel(self.h, C.byref(v)), self.h)
        return v.value

    @property
    def time(self):
        return library().lb_batch_time(self.h)

    def fluid_nodes(self, i=-1):
        return library().lb_batch_fluid_nodes(self.h, int(i))
