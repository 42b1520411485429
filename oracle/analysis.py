"""Continuum theory and measurement helpers used to pin the oracle (TEST INFRASTRUCTURE).

Everything here is derived from the paper's continuum model, not from the
lattice scheme:
  - van der Waals free energy psi(rho) = rho T ln(rho / (1 - b rho)) - a rho^2,
    whose pressure rho psi' - psi is the p0 of Sec. 2;
  - phi^4 free energy A(-phi^2/2 + phi^4/4), whose chemical potential and
    pressure are Eq. (chempot) and the p0 of Sec. 3.1;
  - Maxwell construction, Cahn's interface integral for the surface tension,
    and Cahn's wall free energy -h psi_s (h = -kappa d_n psi|_b) for Young's law
    (Eq. Young), which gives the contact angle for a prescribed wall gradient;
  - Washburn's law, Eqs. (1)-(3), and the Poiseuille mean velocity, Eq. (1).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize

# --------------------------------------------------------------- van der Waals


def vdw_psi(rho, a, b, T):
    return rho * T * np.log(rho / (1.0 - b * rho)) - a * rho * rho


def vdw_mu(rho, a, b, T):
    return T * np.log(rho / (1.0 - b * rho)) + T / (1.0 - b * rho) - 2.0 * a * rho


def vdw_p0(rho, a, b, T):
    """Bulk pressure of Sec. 2, p0 = rho T / (1 - b rho) - a rho^2."""
    return rho * T / (1.0 - b * rho) - a * rho * rho


def maxwell(a=9.0 / 49.0, b=2.0 / 21.0, T=0.56, guess=(2.59, 4.54)):
    """Coexisting gas and liquid densities (equal mu and equal p0)."""
    def eqs(v):
        g, l = v
        return [vdw_mu(g, a, b, T) - vdw_mu(l, a, b, T), vdw_p0(g, a, b, T) - vdw_p0(l, a, b, T)]
    g, l = optimize.fsolve(eqs, guess, xtol=1e-12)
    return float(g), float(l)


def _vdw_excess(a, b, T):
    rg, rl = maxwell(a, b, T)
    mu_c = vdw_mu(rg, a, b, T)
    psi_g = vdw_psi(rg, a, b, T)

    def W(r):
        return max(vdw_psi(r, a, b, T) - psi_g - mu_c * (r - rg), 0.0)
    return rg, rl, W


def vdw_surface_tension(kappa=0.02, a=9.0 / 49.0, b=2.0 / 21.0, T=0.56):
    """Cahn: gamma = int_{rho_g}^{rho_l} sqrt(2 kappa W(rho)) d rho."""
    rg, rl, W = _vdw_excess(a, b, T)
    val, _ = integrate.quad(lambda r: math.sqrt(2.0 * kappa * W(r)), rg, rl, epsabs=1e-13, limit=200)
    return val


def lg_contact_angle(wall_grad, kappa=0.02, a=9.0 / 49.0, b=2.0 / 21.0, T=0.56):
    """Equilibrium angle (degrees) for d_n rho|_b = wall_grad (inward normal)."""
    rg, rl, W = _vdw_excess(a, b, T)
    h = -kappa * wall_grad
    target = 0.5 * kappa * wall_grad * wall_grad

    def F(r):
        v, _ = integrate.quad(lambda q: math.sqrt(2.0 * kappa * W(q)), rg, r, epsabs=1e-13, limit=200)
        return v
    gamma = F(rl)
    if wall_grad == 0.0:
        return 90.0
    if h > 0:
        rs_g = optimize.brentq(lambda r: W(r) - target, rg + 1e-12, 0.5 * (rg + rl))
        rs_l = optimize.brentq(lambda r: W(r) - target, rl + 1e-12, 1.0 / b - 1e-6)
    else:
        rs_g = optimize.brentq(lambda r: W(r) - target, 1e-9, rg - 1e-12)
        rs_l = optimize.brentq(lambda r: W(r) - target, 0.5 * (rg + rl), rl - 1e-12)
    gsg = -h * rs_g + abs(F(rs_g))
    gsl = -h * rs_l + abs(F(rs_l) - gamma)
    c = (gsg - gsl) / gamma
    return math.degrees(math.acos(max(-1.0, min(1.0, c))))


def lg_wall_gradient_for_angle(theta_deg, params):
    return optimize.brentq(lambda g: lg_contact_angle(g, params.kappa, params.a, params.b, params.T) - theta_deg,
                           -0.6, 0.6)


# --------------------------------------------------------------------- binary


def binary_surface_tension(A=0.04, kappa=0.04):
    """gamma = sqrt(8 kappa A / 9) for the phi^4 free energy with bulk phi = +-1."""
    return math.sqrt(8.0 * kappa * A / 9.0)


def binary_cos_theta(wall_grad, A=0.04, kappa=0.04):
    """Young + Cahn for phi^4: cos theta = ((1+O)^1.5 - (1-O)^1.5)/2, O = h / sqrt(kappa A / 2)."""
    h = -kappa * wall_grad
    om = h / math.sqrt(kappa * A / 2.0)
    return 0.5 * ((1.0 + om) ** 1.5 - (1.0 - om) ** 1.5)


def binary_contact_angle(wall_grad, A=0.04, kappa=0.04):
    return math.degrees(math.acos(binary_cos_theta(wall_grad, A, kappa)))


def binary_wall_gradient_for_angle(theta_deg, A=0.04, kappa=0.04):
    c = math.cos(math.radians(theta_deg))
    lim = math.sqrt(A / (2.0 * kappa))  # Omega = 1
    return optimize.brentq(lambda g: binary_cos_theta(g, A, kappa) - c, -lim + 1e-12, lim - 1e-12,
                           xtol=1e-16, rtol=8.9e-16, maxiter=500)


def binary_profile(x, A=0.04, kappa=0.04):
    """Flat-interface profile phi = tanh(x / (sqrt(2) xi)), xi = sqrt(kappa / A)."""
    return np.tanh(np.asarray(x) / (math.sqrt(2.0) * math.sqrt(kappa / A)))


# --------------------------------------------------------------- measurement


def crossings_along_x(v, level=0.0):
    """For each row, x positions (linear interpolation) where v - level changes sign."""
    out = []
    for row in np.asarray(v) - level:
        s = np.sign(row)
        idx = np.where(s[:-1] * s[1:] < 0)[0]
        out.append([k + row[k] / (row[k] - row[k + 1]) for k in idx])
    return out


def fit_circle(xs, ys):
    """Algebraic least-squares circle fit: returns (xc, yc, R)."""
    xs = np.asarray(xs, float)
    ys = np.asarray(ys, float)
    Amat = np.column_stack([xs, ys, np.ones_like(xs)])
    rhs = -(xs ** 2 + ys ** 2)
    (D, E, F), *_ = np.linalg.lstsq(Amat, rhs, rcond=None)
    xc, yc = -D / 2.0, -E / 2.0
    return xc, yc, math.sqrt(xc * xc + yc * yc - F)


def washburn_length(t, gamma, H, theta_deg, eta, t0=0.0):
    """Eq. (3): l = (gamma H cos(theta) / (3 eta))^(1/2) (t + t0)^(1/2)."""
    return np.sqrt(gamma * H * math.cos(math.radians(theta_deg)) / (3.0 * eta) * (np.asarray(t) + t0))


def poiseuille_mean_velocity(H, eta, dpdx):
    """Eq. (1): v = -H^2 / (12 eta) dp/dx."""
    return -H * H / (12.0 * eta) * dpdx


def linear_fit(x, y):
    """Least squares y = m x + c; returns (m, c, R^2)."""
    x = np.asarray(x, float)
    y = np.asarray(y, float)
    m, c = np.polyfit(x, y, 1)
    pred = m * x + c
    ss_res = float(np.sum((y - pred) ** 2))
    ss_tot = float(np.sum((y - y.mean()) ** 2))
    return float(m), float(c), 1.0 - ss_res / ss_tot if ss_tot > 0 else 1.0
