"""Host-side analysis of the lattice model's outputs (numpy).

Fits and reference curves of the Theoretical analysis and Numerical Results
sections: the Washburn law (Eq. 1), the viscous front law with both
viscosities (Eq. 15 without inertia), the front-dynamics ODE (Eq. 15) and
its equal-density, equal-viscosity closed form (Eq. 16), the square-root law
of the precursor lead, Laplace's law for droplets, and the contact angle of
a sessile droplet from its density field (Model section, after Eq. 11).
"""
from __future__ import annotations

import math

import numpy as np


# ---- front laws ----------------------------------------------------------------

def washburn_slope(t, z, t_min: float = 0.0):
    """Least-squares slope and intercept of z^2 against t for t >= t_min
    (Eq. 1: z^2 - z0^2 = gamma H cos(theta) t / (3 mu))."""
    t, z = np.asarray(t, float), np.asarray(z, float)
    m = t >= t_min
    A = np.vstack([t[m], np.ones(m.sum())]).T
    (k, c), *_ = np.linalg.lstsq(A, z[m] ** 2, rcond=None)
    return float(k), float(c)


def washburn_prefactor(gamma: float, H: float, cos_theta: float, mu: float) -> float:
    """gamma H cos(theta) / (3 mu) of Eq. 1."""
    return gamma * H * cos_theta / (3.0 * mu)


def viscous_front_time(z, z0, L, H, gamma, cos_theta, mu_l, mu_g):
    """Time at which the front reaches z when inertia is neglected in Eq. 15:
    z' (mu_g (L - z) + mu_l z) = gamma H cos(theta) / 6, integrated from z0."""
    z = np.asarray(z, float)
    lhs = 0.5 * (mu_l - mu_g) * (z * z - z0 * z0) + mu_g * L * (z - z0)
    return 6.0 * lhs / (gamma * H * cos_theta)


def sqrt_prefactor(t, dz, t_min: float = 0.0) -> float:
    """a of dz = a t^(1/2) (least squares through the origin, t >= t_min):
    the precursor lead over the bulk front (Numerical Results section, Fig. 8)."""
    t, dz = np.asarray(t, float), np.asarray(dz, float)
    m = t >= t_min
    s = np.sqrt(t[m])
    return float((s * dz[m]).sum() / (s * s).sum())


def front_ode(t_end, dt, z0, zdot0, L, H, gamma, cos_theta, rho_l, rho_g, mu_l, mu_g):
    """RK4 integration of the front-dynamics equation (Eq. 15):
    (rho_g (L - z) + rho_l z) z'' + (rho_l - rho_g) z'^2
        = 2 gamma cos(theta) / H - 12 z' (mu_g (L - z) + mu_l z) / H^2.
    Returns (t, z) sampled every dt."""
    def acc(z, v):
        m = rho_g * (L - z) + rho_l * z
        f = 2.0 * gamma * cos_theta / H - 12.0 * v * (mu_g * (L - z) + mu_l * z) / (H * H)
        return (f - (rho_l - rho_g) * v * v) / m

    n = int(round(t_end / dt))
    ts = np.arange(n + 1) * dt
    zs = np.empty(n + 1)
    z, v = float(z0), float(zdot0)
    zs[0] = z
    for i in range(n):
        k1z, k1v = v, acc(z, v)
        k2z, k2v = v + 0.5 * dt * k1v, acc(z + 0.5 * dt * k1z, v + 0.5 * dt * k1v)
        k3z, k3v = v + 0.5 * dt * k2v, acc(z + 0.5 * dt * k2z, v + 0.5 * dt * k2v)
        k4z, k4v = v + dt * k3v, acc(z + dt * k3z, v + dt * k3v)
        z += dt / 6.0 * (k1z + 2 * k2z + 2 * k3z + k4z)
        v += dt / 6.0 * (k1v + 2 * k2v + 2 * k3v + k4v)
        zs[i + 1] = z
    return ts, zs


def front_equal_fluids(t, z0, L, H, gamma, cos_theta, rho, mu):
    """Eq. 16: z = (gamma H cos(theta) / (6 mu L)) t_d [exp(-t/t_d) + t/t_d - 1] + z0,
    t_d = rho H^2 / (12 mu)."""
    t = np.asarray(t, float)
    td = rho * H * H / (12.0 * mu)
    return gamma * H * cos_theta / (6.0 * mu * L) * td * (np.exp(-t / td) + t / td - 1.0) + z0


# ---- droplets ------------------------------------------------------------------

def laplace_gamma(inv_radius, dp):
    """Surface tension from Laplace's law dp = gamma / R (Numerical Results
    section): slope of dp against 1/R, intercept and R^2 of the fit."""
    x, y = np.asarray(inv_radius, float), np.asarray(dp, float)
    A = np.vstack([x, np.ones_like(x)]).T
    (g, c), res, *_ = np.linalg.lstsq(A, y, rcond=None)
    ss = ((y - y.mean()) ** 2).sum()
    r2 = 1.0 - (res[0] / ss if len(res) and ss > 0 else 0.0)
    return float(g), float(c), float(r2)


def interface_points(nA, nB, y_min: int = 0, y_max=None):
    """Points of the phi = (nA - nB)/(nA + nB) = 0 contour, linearly
    interpolated along rows and columns, rows y_min <= y < y_max."""
    nA, nB = np.asarray(nA, float), np.asarray(nB, float)
    tot = nA + nB
    phi = np.where(tot > 0, (nA - nB) / np.where(tot > 0, tot, 1.0), np.nan)
    ny, nx = phi.shape
    y_max = ny if y_max is None else y_max
    pts = []
    for y in range(y_min, y_max):
        row = phi[y]
        for x in range(nx - 1):
            a, b = row[x], row[x + 1]
            if np.isfinite(a) and np.isfinite(b) and (a >= 0) != (b >= 0):
                pts.append((x + a / (a - b), y))
    for x in range(nx):
        col = phi[:, x]
        for y in range(max(y_min, 0), min(y_max, ny) - 1):
            a, b = col[y], col[y + 1]
            if np.isfinite(a) and np.isfinite(b) and (a >= 0) != (b >= 0):
                pts.append((x, y + a / (a - b)))
    return np.array(pts, float).reshape(-1, 2)


def fit_circle(pts):
    """Algebraic least-squares circle (x - a)^2 + (y - b)^2 = R^2 -> (a, b, R)."""
    x, y = pts[:, 0], pts[:, 1]
    A = np.vstack([2 * x, 2 * y, np.ones_like(x)]).T
    rhs = x * x + y * y
    (a, b, c), *_ = np.linalg.lstsq(A, rhs, rcond=None)
    return float(a), float(b), float(math.sqrt(c + a * a + b * b))


def droplet_contact_angle(nA, nB, wall_y: float = 0.5, skip_rows: int = 3):
    """Contact angle (degrees, measured inside species A) of a sessile droplet
    on a wall whose surface is at y = wall_y: circle fit of the phi = 0
    contour above the first skip_rows fluid rows, cos(theta) = (wall_y - y_c) / R."""
    ny = np.asarray(nA).shape[0]
    pts = interface_points(nA, nB, y_min=int(math.ceil(wall_y)) + skip_rows, y_max=ny // 2)
    if len(pts) < 8:
        return float("nan"), None
    a, b, R = fit_circle(pts)
    c = max(-1.0, min(1.0, (wall_y - b) / R))
    return math.degrees(math.acos(c)), (a, b, R)
