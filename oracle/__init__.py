"""FP64 CPU oracle for the free-energy MRT lattice Boltzmann method (TEST INFRASTRUCTURE).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  The product path (paper_0911_0459_gb300) never does, and this
package never imports the product.  The arithmetic lives in lb_oracle.c; this
file only marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OrcParams(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("model", C.c_int),
                ("tube_x0", C.c_int), ("tube_len", C.c_int), ("tube_y0", C.c_int),
                ("tube_h", C.c_int), ("wall_grad", C.c_double),
                ("kappa", C.c_double), ("a", C.c_double), ("b", C.c_double), ("T", C.c_double),
                ("A", C.c_double), ("M", C.c_double), ("nu_l", C.c_double), ("nu_g", C.c_double),
                ("nu", C.c_double), ("lambda_scale", C.c_double),
                ("rho_l", C.c_double), ("rho_g", C.c_double), ("nu_table", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        L.orc_create.argtypes = [C.POINTER(OrcParams), C.POINTER(C.c_void_p)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_destroy.restype = None
        for name in ("orc_init_fields", "orc_fields"):
            getattr(L, name).argtypes = [C.c_void_p] + [C.c_void_p] * 4
        L.orc_step.argtypes = [C.c_void_p, C.c_long]
        L.orc_get_populations.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_set_populations.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.orc_node_kinds.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_stencils.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_equilibria.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_filled_length.argtypes = [C.c_void_p] + [C.POINTER(C.c_double)] * 4
        L.orc_matrices.argtypes = [dp, dp]
        L.orc_matrices.restype = None
        L.orc_feq.argtypes = [C.c_double] * 10 + [dp]
        L.orc_feq.restype = None
        L.orc_geq.argtypes = [C.c_double] * 5 + [dp]
        L.orc_geq.restype = None
        L.orc_collide.argtypes = [dp, dp, C.c_double, dp]
        L.orc_collide.restype = None
        L.orc_time.argtypes = [C.c_void_p]
        L.orc_time.restype = C.c_long
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape):
    if a is None:
        return None
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    assert out.shape == shape, (out.shape, shape)
    return out


def wall_gradient_of(cap) -> float:
    """The wall gradient of a workload: given directly, or from its contact angle."""
    if cap.wall_grad is not None:
        return float(cap.wall_grad)
    if cap.theta_deg is None:
        return 0.0
    from .analysis import binary_wall_gradient_for_angle, lg_wall_gradient_for_angle
    p = cap.params
    if p.model == 1:
        return binary_wall_gradient_for_angle(cap.theta_deg, p.A, p.kappa)
    return lg_wall_gradient_for_angle(cap.theta_deg, p)


class Oracle:
    """One FP64 lattice on the CPU.  Fields are (ny, nx) arrays; populations (9, ny, nx)."""

    def __init__(self, cap, wall_grad=None):
        p = cap.params
        self.cap = cap
        self.nx, self.ny = cap.nx, cap.ny
        self.model = p.model
        wg = wall_gradient_of(cap) if wall_grad is None else float(wall_grad)
        self.wall_grad = wg
        self.params = OrcParams(cap.nx, cap.ny, p.model, cap.tube_x0, cap.tube_len, cap.tube_y0,
                                cap.tube_h, wg, p.kappa, p.a, p.b, p.T, p.A, p.M, p.nu_l, p.nu_g,
                                p.nu, p.lambda_scale, p.rho_l, p.rho_g, int(getattr(p, "nu_table", 0)))
        h = C.c_void_p()
        rc = lib().orc_create(C.byref(self.params), C.byref(h))
        if rc != 0:
            raise ValueError(f"oracle: invalid geometry or parameters (code {rc})")
        self.h = h

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            _lib.orc_destroy(h)
            self.h = None

    @property
    def shape(self):
        return (self.ny, self.nx)

    def init_fields(self, rho, ux, uy, phi=None):
        s = self.shape
        args = [_f64(rho, s), _f64(ux, s), _f64(uy, s), _f64(phi, s)]
        rc = lib().orc_init_fields(self.h, *[_ptr(a) for a in args])
        if rc:
            raise RuntimeError(f"oracle init failed ({rc})")
        return self

    def init_default(self):
        import workloads
        return self.init_fields(*workloads.initial_fields(self.cap))

    def step(self, n=1):
        rc = lib().orc_step(self.h, int(n))
        if rc:
            raise RuntimeError(f"oracle step failed ({rc})")
        return self

    @property
    def time(self):
        return lib().orc_time(self.h)

    def fields(self):
        s = self.shape
        out = [np.zeros(s) for _ in range(4)]
        lib().orc_fields(self.h, *[_ptr(a) for a in out])
        rho, ux, uy, phi = out
        return rho, ux, uy, (phi if self.model == 1 else None)

    def populations(self):
        f = np.zeros((9,) + self.shape)
        g = np.zeros((9,) + self.shape)
        lib().orc_get_populations(self.h, _ptr(f), _ptr(g))
        return f, (g if self.model == 1 else None)

    def set_populations(self, f, g=None, apply_rest=True):
        sh = (9,) + self.shape
        f = _f64(f, sh)
        g = _f64(g, sh) if g is not None else None
        lib().orc_set_populations(self.h, _ptr(f), _ptr(g), int(bool(apply_rest)))
        return self

    def node_kinds(self):
        k = np.zeros(self.shape, dtype=np.uint8)
        lib().orc_node_kinds(self.h, _ptr(k))
        return k

    def stencils(self, field, h=0.0):
        s = self.shape
        v = _f64(field, s)
        dx, dy, lap = np.zeros(s), np.zeros(s), np.zeros(s)
        rc = lib().orc_stencils(self.h, _ptr(v), float(h), _ptr(dx), _ptr(dy), _ptr(lap))
        if rc:
            raise RuntimeError(f"oracle stencil failed ({rc})")
        return dx, dy, lap

    def equilibria(self):
        feq = np.zeros((9,) + self.shape)
        geq = np.zeros((9,) + self.shape)
        om = np.zeros(self.shape)
        lib().orc_equilibria(self.h, _ptr(feq), _ptr(geq), _ptr(om))
        return feq, (geq if self.model == 1 else None), om

    def filled_length(self):
        vals = [C.c_double() for _ in range(4)]
        lib().orc_filled_length(self.h, *[C.byref(v) for v in vals])
        l, lvol, mass, phisum = (v.value for v in vals)
        return {"l": l, "l_vol": lvol, "mass": mass, "phi_sum": phisum}


def matrices():
    M = np.zeros(81)
    Mi = np.zeros(81)
    lib().orc_matrices(M, Mi)
    return M.reshape(9, 9), Mi.reshape(9, 9)


def feq(rho, ux, uy, P0, kappa, gpx, gpy, grx, gry, lam):
    out = np.zeros(9)
    lib().orc_feq(rho, ux, uy, P0, kappa, gpx, gpy, grx, gry, lam, out)
    return out


def geq(phi, ux, uy, mu, mob):
    out = np.zeros(9)
    lib().orc_geq(phi, ux, uy, mu, mob, out)
    return out


def collide(f, fe, omega):
    out = np.zeros(9)
    lib().orc_collide(np.ascontiguousarray(f, dtype=np.float64),
                      np.ascontiguousarray(fe, dtype=np.float64), float(omega), out)
    return out
