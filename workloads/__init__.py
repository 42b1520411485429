"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds geometry descriptions, parameter sets and initial macroscopic
fields only.  It contains none of the lattice Boltzmann arithmetic (no
equilibria, no stencils, no collision): both implementations turn the fields
produced here into populations with their own code.

Geometry (one convention for every workload).  The grid is nx x ny, periodic in
x and y.  A capillary occupies the columns [tube_x0, tube_x0 + tube_len) (taken
modulo nx); inside those columns the rows [tube_y0, tube_y0 + tube_h) (modulo
ny) are fluid and every other row is solid, so by the y-wrap one block of solid
forms both walls of the tube.  All other columns are fluid reservoirs, periodic
in y, as in the paper's capillary set-up (Sec. 2.2, Fig. 1b).  tube_len = 0
means no walls at all; tube_len = nx means a channel with walls along the whole
length.

Initial state (the paper's Sec. 2.2 starts the meniscus at l = 10): velocity
zero, liquid in x in [gas_cols, tube_x0 + l0) and gas elsewhere, with tanh
profiles of width 2 (liquid-gas) or sqrt(2) (binary, the phi^4 profile
tanh(x / sqrt(2 kappa / A)) with kappa = A) across both interfaces.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

LG, BINARY = 0, 1
STORAGE_F64, STORAGE_F32, STORAGE_F16DEV, STORAGE_MOMENTS = 0, 1, 2, 3
STORAGE_MOMENTS_F16, STORAGE_F32_GELIM, STORAGE_F32_BLOCKED, STORAGE_F16_BLOCKED = 4, 5, 6, 7


@dataclasses.dataclass
class Params:
    """Model parameters.  Values quoted from the paper where it gives them."""
    model: int = BINARY
    storage: int = STORAGE_F32
    # liquid-gas (van der Waals), Sec. 2: kappa = 0.02, a = 9/49, b = 2/21, T = 0.56
    kappa: float = 0.04
    a: float = 9.0 / 49.0
    b: float = 2.0 / 21.0
    T: float = 0.56
    # binary, Sec. 3.1: A = kappa = 0.04; mobility M is not valued in the paper
    A: float = 0.04
    M: float = 0.1
    nu_l: float = 1.0 / 6.0
    nu_g: float = 1.0 / 6.0
    # liquid-gas viscosity (tau = 1 <-> nu = 1/6); lambda = lambda_scale * local nu
    nu: float = 1.0 / 6.0
    lambda_scale: float = 1.0
    # densities used for the initial profile and for the liquid-gas l(t) threshold
    rho_l: float = 4.54
    rho_g: float = 2.59
    # binary: 0 = exact local viscosity; K >= 2 = the nearest of K viscosities evenly
    # spaced over [nu_g, nu_l] (the look-up table of App. A)
    nu_table: int = 0


def lg_params(**kw) -> Params:
    p = Params(model=LG, storage=STORAGE_F64, kappa=0.02, nu=1.0 / 6.0)
    return dataclasses.replace(p, **kw)


def binary_params(**kw) -> Params:
    p = Params(model=BINARY, storage=STORAGE_F32, kappa=0.04, A=0.04, M=0.1,
               rho_l=1.0, rho_g=1.0)
    return dataclasses.replace(p, **kw)


@dataclasses.dataclass
class Capillary:
    name: str
    nx: int
    ny: int
    tube_x0: int
    tube_len: int
    tube_y0: int
    tube_h: int
    gas_cols: int
    l0: int
    params: Params
    theta_deg: Optional[float] = None   # equilibrium contact angle the wall is set for
    wall_grad: Optional[float] = None   # d_n rho|_b (liquid-gas) or d_n phi|_b (binary), if given directly
    steps: int = 2000

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    def wall_gradient(self) -> float:
        """The wall gradient this workload gives the library: wall_grad when set, else (binary
        model) the one that makes theta_deg the equilibrium angle, else 0."""
        if self.wall_grad is not None:
            return float(self.wall_grad)
        if self.theta_deg is None:
            return 0.0
        if self.params.model != BINARY:
            raise ValueError("liquid-gas workloads must give wall_grad directly")
        return binary_wall_gradient(self.theta_deg, self.params.A, self.params.kappa)


def binary_wall_gradient(theta_deg: float, A: float = 0.04, kappa: float = 0.04) -> float:
    """Input conversion: the wall gradient d_n phi|_b (inward normal) that sets the
    equilibrium contact angle theta of the phi^4 binary model (Sec. 3.2).

    Cahn's wall energy -h phi_s with h = -kappa d_n phi|_b and Young's law give
    cos(theta) = ((1 + W)^1.5 - (1 - W)^1.5) / 2, W = h / sqrt(kappa A / 2); W is
    found by bisection on [-1, 1], where the right-hand side increases.
    """
    c = math.cos(math.radians(theta_deg))

    def cos_of(w):
        return 0.5 * ((1.0 + w) ** 1.5 - (1.0 - w) ** 1.5)
    lo, hi = -1.0, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if cos_of(mid) < c:
            lo = mid
        else:
            hi = mid
    w = 0.5 * (lo + hi)
    return -w * math.sqrt(kappa * A / 2.0) / kappa


# ---------------------------------------------------------------------------
# The paper-shaped workloads.
# ---------------------------------------------------------------------------

def config_lg_256x32() -> Capillary:
    """Liquid-gas FP64 capillary, 256 x 32, tube over x in [64, 256), H = 24.

    Wall gradient d_n rho|_b = -0.144, which the paper uses for a 60 degree
    equilibrium angle (Sec. 2.2).  Gas buffer [0, 16) joins the tube outlet
    through the x-wrap; liquid reservoir [16, 64); l0 = 10; tau = 1.
    """
    return Capillary("lg_256x32", 256, 32, 64, 192, 4, 24, 16, 10,
                     lg_params(), theta_deg=60.0, wall_grad=-0.144, steps=2000)


def config_lg_16384x256() -> Capillary:
    """Liquid-gas FP64 capillary at the large capillary's size, 16384 x 256 (H = 200,
    tube over x in [512, 16384), gas 128 columns), with the 256 x 32 capillary's
    parameters: a lattice larger than L2 for the FP64 path's roofline."""
    return Capillary("lg_16384x256", 16384, 256, 512, 16384 - 512, 28, 200, 128, 10,
                     lg_params(), theta_deg=60.0, wall_grad=-0.144, steps=2000)


def config_binary_2048x64() -> Capillary:
    """Binary FP32 capillary, 2048 x 64, H = 50, viscosity ratio 10, 60 degrees."""
    return Capillary("binary_2048x64", 2048, 64, 256, 1792, 7, 50, 64, 10,
                     binary_params(nu_l=0.83, nu_g=0.083), theta_deg=60.0, steps=50000)


def config_binary_16384x256(storage: int = STORAGE_F32) -> Capillary:
    """Binary single large capillary, 16384 x 256, H = 200, ratio 50, 45 degrees."""
    return Capillary("binary_16384x256", 16384, 256, 512, 16384 - 512, 28, 200, 128, 10,
                     binary_params(nu_l=0.83, nu_g=0.0166, storage=storage),
                     theta_deg=45.0, steps=2000)


def config_binary_crop_1024x64(storage: int = STORAGE_F32) -> Capillary:
    """1024 x 64 crop of the large capillary (H = 50 band, same parameters)."""
    return Capillary("binary_crop_1024x64", 1024, 64, 256, 768, 7, 50, 64, 10,
                     binary_params(nu_l=0.83, nu_g=0.0166, storage=storage),
                     theta_deg=45.0, steps=2000)


RATIOS = (1, 5, 10, 50, 100)


def viscosities_for_ratio(ratio: float):
    """Liquid and gas kinematic viscosities for a viscosity ratio.

    nu_l = 0.83 (the paper's Fig. 4 value) for ratios up to 50; ratio 100 uses
    nu_l = 1.7 so that nu_g = 0.017 stays at the paper's most extreme gas
    viscosity (Fig. 5a squares).
    """
    if ratio >= 100:
        return 1.7, 1.7 / ratio
    return 0.83, 0.83 / ratio


def sweep(seed: int = 0, n: int = 256, steps: int = 20000,
          lengths=(1024, 8192), fixed_len: Optional[int] = None,
          vary_gamma: bool = False, liquid_cols: int = 128, align: int = 8) -> List[Capillary]:
    """Seeded sweep of uneven binary capillaries.

    H uniform in {16, 24, ..., 128}; tube length uniform over the multiples of
    `align` in [1024, 8192] (or fixed_len), so that with the default align every
    nx = 160 + L is a multiple of 8; ny = H + 8; liquid reservoir 128 columns and a gas buffer of
    32 columns in front of it; viscosity ratio uniform in {1, 5, 10, 50, 100};
    theta uniform in [30, 80] degrees.  With vary_gamma the surface tension is
    varied by drawing A = kappa uniformly in [0.03, 0.05].  liquid_cols widens
    the liquid reservoir (so that it does not run dry on long fills).
    """
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        H = int(rng.choice(np.arange(16, 129, 8)))
        if fixed_len:
            L = int(fixed_len)
        else:
            lo, hi = -(-lengths[0] // align), lengths[1] // align
            L = align * int(rng.integers(lo, hi + 1))
        ratio = float(rng.choice(RATIOS))
        theta = float(rng.uniform(30.0, 80.0))
        Ak = float(rng.uniform(0.03, 0.05)) if vary_gamma else 0.04
        nu_l, nu_g = viscosities_for_ratio(ratio)
        gas, liquid = 32, liquid_cols
        x0 = gas + liquid
        p = binary_params(nu_l=nu_l, nu_g=nu_g, A=Ak, kappa=Ak)
        out.append(Capillary(f"sweep{seed}_{k}", x0 + L, H + 8, x0, L, 4, H, gas, 10, p,
                             theta_deg=theta, steps=steps))
    return out


# ---------------------------------------------------------------------------
# Initial macroscopic fields.  Arrays are (ny, nx), row-major, x contiguous.
# ---------------------------------------------------------------------------

def solid_mask(cap: Capillary) -> np.ndarray:
    x = np.arange(cap.nx)
    y = np.arange(cap.ny)
    in_tube = ((x - cap.tube_x0) % cap.nx) < cap.tube_len
    in_band = ((y - cap.tube_y0) % cap.ny) < cap.tube_h
    return (~in_band)[:, None] & in_tube[None, :]


def liquid_fraction_profile(cap: Capillary) -> np.ndarray:
    """Smooth liquid indicator in [0, 1] along x (liquid in [gas_cols, x0 + l0))."""
    w = 2.0 if cap.params.model == LG else math.sqrt(2.0)
    x = np.arange(cap.nx, dtype=np.float64)
    xa = float(cap.gas_cols)
    xb = float(cap.tube_x0 + cap.l0)
    return 0.5 * (np.tanh((x - xa) / w) - np.tanh((x - xb) / w))


def initial_fields(cap: Capillary):
    """rho, ux, uy, phi (phi is None for the liquid-gas model); solid nodes hold 0."""
    chi = np.broadcast_to(liquid_fraction_profile(cap)[None, :], (cap.ny, cap.nx))
    solid = solid_mask(cap)
    p = cap.params
    ux = np.zeros((cap.ny, cap.nx))
    uy = np.zeros((cap.ny, cap.nx))
    if p.model == LG:
        rho = p.rho_g + (p.rho_l - p.rho_g) * chi
        phi = None
    else:
        rho = np.ones((cap.ny, cap.nx))
        phi = 2.0 * chi - 1.0
        phi = np.where(solid, 0.0, phi)
    rho = np.where(solid, 0.0, rho)
    return np.ascontiguousarray(rho), ux, uy, (None if phi is None else np.ascontiguousarray(phi))


# ---------------------------------------------------------------------------
# Small synthetic set-ups used by the physics tests.
# ---------------------------------------------------------------------------

def periodic_box(nx: int, ny: int, params: Params, name: str = "box") -> Capillary:
    """Fully periodic box without walls."""
    return Capillary(name, nx, ny, 0, 0, 0, ny, 0, 0, params)


def channel(nx: int, ny: int, h: int, params: Params, wall_grad: float = 0.0,
            name: str = "channel") -> Capillary:
    """Walls along the whole length: fluid rows [0, h), solid rows [h, ny)."""
    return Capillary(name, nx, ny, 0, nx, 0, h, 0, 0, params, wall_grad=wall_grad)


def slab_fields(nx: int, ny: int, x_a: float, x_b: float, width: float,
                lo: float, hi: float) -> np.ndarray:
    """Field equal to hi inside [x_a, x_b) and lo outside, tanh edges."""
    x = np.arange(nx, dtype=np.float64)
    s = 0.5 * (np.tanh((x - x_a) / width) - np.tanh((x - x_b) / width))
    return np.ascontiguousarray(np.broadcast_to(lo + (hi - lo) * s, (ny, nx)).copy())


def drop_fields(nx: int, ny: int, xc: float, yc: float, radius: float, width: float,
                inside: float, outside: float) -> np.ndarray:
    """Circular drop with a tanh edge (periodic distances)."""
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    dx = (x - xc + nx / 2) % nx - nx / 2
    dy = (y - yc + ny / 2) % ny - ny / 2
    r = np.sqrt(dx * dx + dy * dy)
    s = 0.5 * (1.0 - np.tanh((r - radius) / width))
    return np.ascontiguousarray(outside + (inside - outside) * s)


def random_state_fields(nx: int, ny: int, seed: int, model: int, amp_u: float = 0.02):
    """Smooth random fields for per-step parity checks (low-pass filtered noise)."""
    rng = np.random.default_rng(seed)

    def smooth(a):
        k = np.fft.rfft2(a)
        ky = np.fft.fftfreq(a.shape[0])[:, None]
        kx = np.fft.rfftfreq(a.shape[1])[None, :]
        k *= np.exp(-(kx ** 2 + ky ** 2) / (2 * 0.06 ** 2))
        out = np.fft.irfft2(k, s=a.shape)
        return out / (np.abs(out).max() + 1e-30)

    ux = amp_u * smooth(rng.standard_normal((ny, nx)))
    uy = amp_u * smooth(rng.standard_normal((ny, nx)))
    if model == LG:
        rho = 3.5 + 0.9 * smooth(rng.standard_normal((ny, nx)))
        phi = None
    else:
        rho = 1.0 + 0.02 * smooth(rng.standard_normal((ny, nx)))
        phi = np.clip(1.3 * smooth(rng.standard_normal((ny, nx))), -1.0, 1.0)
    return rho, ux, uy, phi


ALL_CONFIGS: Dict[str, callable] = {
    "lg_256x32": config_lg_256x32,
    "binary_2048x64": config_binary_2048x64,
    "binary_16384x256": config_binary_16384x256,
    "binary_crop_1024x64": config_binary_crop_1024x64,
}
