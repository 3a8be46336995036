"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds geometry descriptions, initial density layouts and seeded
parameter draws only: none of the lattice Boltzmann arithmetic.  Both the
FP64 oracle and the GPU library receive what is built here and nothing else.

Geometry (Numerical Results section, Fig. 1): a periodic nx x ny lattice; two
plates of one solid row each (rows ``y_bot`` and ``y_top``) span the columns
``[cap_x0, cap_x1)`` and form the capillary, everything else is fluid
(reservoir, periodic top/bottom and east/west).  ``y_top = -1`` means no top
plate (sessile-droplet boxes).

Initial layout: sharp two-phase step, the liquid (species A) at
(rho_major, rho_minor) and the gas (species B) at (rho_minor, rho_major), at
rest; solid nodes carry no fluid.
"""
from __future__ import annotations

import math

import numpy as np

RHO_MAJOR = 2.0
RHO_MINOR = 0.04

# Nominal wall couplings (w-weighted units, negative = attracts species A).
G_AW_THETA60 = -0.2     # capillary of the 256x32 case
G_AW_WETTING = -0.5     # complete-wetting capillary (theta = 0)


def capillary_geometry(nx: int, ny: int, cap_x0: int, cap_x1: int, y_bot: int, y_top: int) -> dict:
    return dict(nx=int(nx), ny=int(ny), cap_x0=int(cap_x0), cap_x1=int(cap_x1),
                y_bot=int(y_bot), y_top=int(y_top))


def periodic_box(nx: int, ny: int) -> dict:
    """A wall-free fully periodic box."""
    return dict(nx=int(nx), ny=int(ny), cap_x0=0, cap_x1=0, y_bot=-1, y_top=-1)


def solid_mask(geom: dict) -> np.ndarray:
    """uint8 [ny, nx]: 1 on plate nodes (or the explicit mask)."""
    if geom.get("mask") is not None:
        return np.asarray(geom["mask"], dtype=np.uint8).reshape(geom["ny"], geom["nx"])
    ny, nx = geom["ny"], geom["nx"]
    m = np.zeros((ny, nx), dtype=np.uint8)
    x0, x1 = geom["cap_x0"], geom["cap_x1"]
    for y in (geom["y_bot"], geom["y_top"]):
        if 0 <= y < ny and x1 > x0:
            m[y, x0:x1] = 1
    return m


def slab_fields(geom: dict, x_lo: int, x_hi: int, rho_major: float = RHO_MAJOR,
                rho_minor: float = RHO_MINOR):
    """Liquid A on columns [x_lo, x_hi), gas B elsewhere; zero on solids."""
    ny, nx = geom["ny"], geom["nx"]
    xs = np.arange(nx)[None, :].repeat(ny, 0)
    liquid = (xs >= x_lo) & (xs < x_hi)
    nA = np.where(liquid, rho_major, rho_minor).astype(np.float64)
    nB = np.where(liquid, rho_minor, rho_major).astype(np.float64)
    s = solid_mask(geom).astype(bool)
    nA[s] = 0.0
    nB[s] = 0.0
    return nA, nB


def droplet_fields(geom: dict, cx: float, cy: float, r: float, rho_major: float = RHO_MAJOR,
                   rho_minor: float = RHO_MINOR):
    """Liquid A inside the disc |x - c| < r (periodic images ignored)."""
    ny, nx = geom["ny"], geom["nx"]
    ys, xs = np.mgrid[0:ny, 0:nx].astype(np.float64)
    inside = (xs - cx) ** 2 + (ys - cy) ** 2 < r * r
    nA = np.where(inside, rho_major, rho_minor).astype(np.float64)
    nB = np.where(inside, rho_minor, rho_major).astype(np.float64)
    s = solid_mask(geom).astype(bool)
    nA[s] = 0.0
    nB[s] = 0.0
    return nA, nB


def random_fields(geom: dict, seed: int, lo: float = 0.05, hi: float = 2.0):
    """Independent uniform densities in [lo, hi) per node and species (PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ny, nx = geom["ny"], geom["nx"]
    nA = rng.uniform(lo, hi, size=(ny, nx))
    nB = rng.uniform(lo, hi, size=(ny, nx))
    s = solid_mask(geom).astype(bool)
    nA[s] = 0.0
    nB[s] = 0.0
    return nA, nB


def params(G: float, tau_A: float, tau_B: float, G_Aw: float = 0.0, G_Bw: float = 0.0,
           body=(0.0, 0.0), rho_bulk: float = RHO_MAJOR) -> dict:
    return dict(G=float(G), tau_A=float(tau_A), tau_B=float(tau_B), G_Aw=float(G_Aw),
                G_Bw=float(G_Bw), body=(float(body[0]), float(body[1])), rho_bulk=float(rho_bulk))


def capillary_run(L_cap: int, H: int, G: float, tau_A: float, tau_B: float, G_Aw: float,
                  G_Bw: float = 0.0) -> dict:
    """Capillary in the right half of a 2 L_cap x (H + 2) box (Fig. 1).  The
    reservoir (left half, periodic top and bottom) holds gas on [0, L_cap/2)
    and liquid from L_cap/2 to the front at L_cap + L_cap/4, so the gas that
    the liquid displaces leaves the capillary through the periodic east side
    into the reservoir's gas, across a flat reservoir interface."""
    nx, ny = 2 * L_cap, H + 2
    geom = capillary_geometry(nx, ny, L_cap, 2 * L_cap, 0, H + 1)
    x_front = L_cap + L_cap // 4
    return dict(geom=geom, params=params(G, tau_A, tau_B, G_Aw, G_Bw), init=("slab", L_cap // 2, x_front))


def capillary_run_long_reservoir(L_cap: int, H: int, G: float, tau_A: float, tau_B: float, G_Aw: float,
                                 G_Bw: float = 0.0) -> dict:
    """Capillary of length L_cap at the right end of a 3 L_cap x (H + 2) box
    whose reservoir (the left two thirds, periodic top and bottom) holds gas
    on [0, L_cap/2) and liquid from L_cap/2 to the front at 2 L_cap + L_cap/4:
    enough liquid to fill the whole capillary, so that the front can travel
    its full length while the reservoir still feeds it."""
    nx, ny = 3 * L_cap, H + 2
    geom = capillary_geometry(nx, ny, 2 * L_cap, 3 * L_cap, 0, H + 1)
    return dict(geom=geom, params=params(G, tau_A, tau_B, G_Aw, G_Bw),
                init=("slab", L_cap // 2, 2 * L_cap + L_cap // 4))


# ---- the five workload families ------------------------------------------

def config_capillary_256x32() -> dict:
    """256x32 periodic in x; plates of length 128 centred ([64, 192)) at rows 0
    and 25 (H = 24); liquid A on x < 96; G = 1.4, tau_A = 1.0, tau_B = 0.6;
    wall-A coupling for a partially wetting capillary; 3000 steps, z(t) every 50."""
    geom = capillary_geometry(256, 32, 64, 192, 0, 25)
    return dict(name="capillary_256x32_fp64", geom=geom,
                params=params(1.4, 1.0, 0.6, G_AW_THETA60, 0.0),
                init=("slab", 0, 96), steps=3000, log_every=50)


def config_capillary_8192x160(tau_B: float = 0.55) -> dict:
    """8192x160, capillary length 6144 centred ([1024, 7168)), plates at rows 0
    and 129 (H = 128); liquid on x < 2560; G = 1.4; tau_A = 1.0, tau_B in
    {1.0, 0.55} (dynamic-viscosity ratio 1 or 10 at matched densities);
    complete-wetting wall coupling; 10^5 steps."""
    geom = capillary_geometry(8192, 160, 1024, 7168, 0, 129)
    return dict(name=f"capillary_8192x160_tauB{tau_B}", geom=geom,
                params=params(1.4, 1.0, tau_B, G_AW_WETTING, 0.0),
                init=("slab", 0, 2560), steps=100000, log_every=50)


def batch_uneven_capillaries(n: int = 512, seed: int = 3) -> list:
    """n independent capillaries: H ~ U{16..128}, L_cap ~ U{256..4096}, grid
    2 L_cap x (H + 2), plates in the right half; G ~ U[1.2, 1.6], tau_B ~
    U[0.55, 1.5], tau_A = 1; wall-A coupling ~ U[-0.5, 0.3] (wetting to
    non-wetting)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    H = rng.integers(16, 129, size=n)
    L = rng.integers(256, 4097, size=n)
    G = rng.uniform(1.2, 1.6, size=n)
    tB = rng.uniform(0.55, 1.5, size=n)
    gw = rng.uniform(-0.5, 0.3, size=n)
    return [capillary_run(int(L[r]), int(H[r]), float(G[r]), 1.0, float(tB[r]), float(gw[r]))
            for r in range(n)]


def batch_uneven_capillaries_stable(n: int = 512, seed: int = 3) -> list:
    """The uneven ensemble of batch_uneven_capillaries inside the band where
    the velocity-shift scheme stays finite for 2 10^4 steps and more: the
    same sizes (H ~ U{16..128}, L_cap ~ U{256..4096}, grid 2 L_cap x (H + 2)),
    G ~ U[1.0, 1.1], tau_A = 1, tau_B ~ U[1.0, 1.5] (gas up to 1.9 times more
    viscous), and a target contact angle theta ~ U[60, 105] degrees per run
    (the range that the stable couplings -0.5 <= G_Aw <= 0.3 reach at every G
    and tau_B of the band).
    The wall coupling G_Aw that gives theta is not drawn here: it comes from
    a measured calibration table (the params carry G_Aw = nan and the target
    under "theta_target")."""
    rng = np.random.Generator(np.random.PCG64(seed))
    H = rng.integers(16, 129, size=n)
    L = rng.integers(256, 4097, size=n)
    G = rng.uniform(1.0, 1.1, size=n)
    tB = rng.uniform(1.0, 1.5, size=n)
    th = rng.uniform(60.0, 105.0, size=n)
    runs = []
    for r in range(n):
        run = capillary_run(int(L[r]), int(H[r]), float(G[r]), 1.0, float(tB[r]), float("nan"))
        run["params"]["theta_target"] = float(th[r])
        runs.append(run)
    return runs


def batch_sessile_droplets(n: int = 1024, seed: int = 4, nx: int = 256, ny: int = 128,
                           radius: float = 40.0) -> list:
    """n sessile droplets on a wall at y = 0 of a periodic nx x ny box, radius
    40 centred at (nx/2, 0.5); couplings (G_Aw, G_Bw) on a jittered 32x32 grid
    of [-0.5, 0.5]^2; G = 1.4, tau_A = tau_B = 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    side = int(math.ceil(math.sqrt(n)))
    cell = 1.0 / side
    runs = []
    for r in range(n):
        gi, gj = r % side, r // side
        a = -0.5 + (gi + rng.uniform(0.0, 1.0)) * cell
        b = -0.5 + (gj + rng.uniform(0.0, 1.0)) * cell
        geom = dict(nx=nx, ny=ny, cap_x0=0, cap_x1=nx, y_bot=0, y_top=-1)
        runs.append(dict(geom=geom, params=params(1.4, 1.0, 1.0, a, b),
                         init=("droplet", nx / 2.0, 0.5, radius)))
    return runs


def fp16_shift(run: dict):
    """FP16-shifted storage offset rho_ref per species: the species' density in
    the phase that fills most of the run's fluid nodes (the median of its
    initial field), so that most stored values are small."""
    nA, nB = initial_fields(run)
    fluid = solid_mask(run["geom"]) == 0
    return float(np.median(nA[fluid])), float(np.median(nB[fluid]))


def initial_fields(run: dict):
    """Initial (nA, nB) of a run dict built by this module."""
    kind = run["init"][0]
    if kind == "slab":
        return slab_fields(run["geom"], run["init"][1], run["init"][2])
    if kind == "droplet":
        _, cx, cy, r = run["init"]
        return droplet_fields(run["geom"], cx, cy, r)
    if kind == "fields":
        return run["init"][1], run["init"][2]
    raise ValueError(kind)
