"""Contact-angle calibration, capillary prefactors and the surrogate loop.

The paper obtains the contact angle of a wall coupling only a posteriori,
from static droplets (Model section, after Eq. 11), and compares capillary
fronts with Washburn's law (Eq. 1) and the viscous front law (Eq. 15) and the
precursor lead with a square-root law (Numerical Results section, Fig. 8).
This module runs those measurements with the GPU lattice model (batched runs
through ``Lattice``), builds the surrogate's training set from them, and
drives the proposal loop in which every proposal is judged by the lattice
model itself (FP64), with bisection on the coupling as the fallback.
"""
from __future__ import annotations

import math

import numpy as np

from . import analysis as A
from .lbm import Lattice

RHO = (2.0, 0.04)


def droplet_run(G_Aw, G_Bw, G, tau_A, tau_B, nx=128, ny=80, radius=24.0):
    """Sessile droplet of species A on a wall at y = 0 (full width) of a
    periodic nx x ny box, a half disc centred on the wall."""
    geom = dict(nx=nx, ny=ny, cap_x0=0, cap_x1=nx, y_bot=0, y_top=-1)
    prm = dict(G=float(G), tau_A=float(tau_A), tau_B=float(tau_B), G_Aw=float(G_Aw), G_Bw=float(G_Bw))
    return dict(geom=geom, params=prm, init=("droplet", nx / 2.0, 0.5, float(radius)), rho=RHO)


def measure_angles(couplings, G, tau_A=1.0, tau_B=1.0, steps=8000, precision="f32", nx=128, ny=80, radius=24.0):
    """Equilibrium contact angles (degrees) of sessile droplets, one per
    (G_Aw, G_Bw) pair, advanced together in one batched handle."""
    runs = [droplet_run(a, b, G, tau_A, tau_B, nx, ny, radius) for a, b in couplings]
    out = np.full(len(runs), np.nan)
    with Lattice(runs, precision=precision, tile=(128, 16)) as lat:
        lat.step(steps)
        for i in range(len(runs)):
            nA, nB = lat.densities(i)
            if np.all(np.isfinite(nA)) and np.all(np.isfinite(nB)):
                out[i], _ = A.droplet_contact_angle(nA, nB, wall_y=0.5, skip_rows=3)
    return out


def angle_table(G_values, tau_B_values, couplings, tau_A=1.0, steps=8000, precision="f32"):
    """Contact angle theta(G, tau_B, G_Aw) of sessile droplets (G_Bw = 0) on
    the grid G_values x tau_B_values x couplings, all droplets advanced in
    one batched handle: the a-posteriori map from wall coupling to angle
    (Model section, after Eq. 11).  Returns an array [len(G)][len(tau_B)][len(G_Aw)]."""
    G_values, tau_B_values, couplings = (np.asarray(v, float) for v in (G_values, tau_B_values, couplings))
    runs = [droplet_run(a, 0.0, G, tau_A, tB) for G in G_values for tB in tau_B_values for a in couplings]
    out = np.full(len(runs), np.nan)
    with Lattice(runs, precision=precision, tile=(128, 16)) as lat:
        lat.step(steps)
        for i in range(len(runs)):
            nA, nB = lat.densities(i)
            if np.all(np.isfinite(nA)) and np.all(np.isfinite(nB)):
                out[i], _ = A.droplet_contact_angle(nA, nB, wall_y=0.5, skip_rows=3)
    return out.reshape(len(G_values), len(tau_B_values), len(couplings))


def coupling_for_angle(table, G_values, tau_B_values, couplings, G, tau_B, theta):
    """Wall coupling G_Aw (G_Bw = 0) that gives the angle theta at (G, tau_B):
    the angle is interpolated bilinearly in (G, tau_B) from the table, then
    inverted linearly in G_Aw (theta increases with G_Aw).  Angles outside the
    table's range give its end coupling."""
    G_values, tau_B_values, couplings = (np.asarray(v, float) for v in (G_values, tau_B_values, couplings))

    def frac(v, grid):
        i = int(np.clip(np.searchsorted(grid, v) - 1, 0, len(grid) - 2))
        return i, float(np.clip((v - grid[i]) / (grid[i + 1] - grid[i]), 0.0, 1.0))
    i, fg = frac(G, G_values)
    j, ft = frac(tau_B, tau_B_values)
    th = ((1 - fg) * (1 - ft) * table[i, j] + fg * (1 - ft) * table[i + 1, j] + (1 - fg) * ft * table[i, j + 1]
          + fg * ft * table[i + 1, j + 1])
    order = np.argsort(th)
    return float(np.interp(theta, th[order], couplings[order]))


def map_couplings(runs, G_values=(1.0, 1.05, 1.1), tau_B_values=(1.0, 1.25, 1.5),
                  couplings=(-0.5, -0.4, -0.3, -0.2, -0.1, 0.0, 0.1, 0.2, 0.3), steps=8000):
    """Fills G_Aw of every run that carries params["theta_target"] from a
    measured angle table; returns the table (G, tau_B, G_Aw grids and angles)."""
    table = angle_table(G_values, tau_B_values, couplings, steps=steps)
    for run in runs:
        p = run["params"]
        if "theta_target" in p:
            p["G_Aw"] = coupling_for_angle(table, G_values, tau_B_values, couplings, p["G"], p["tau_B"],
                                           p["theta_target"])
    return dict(G=list(G_values), tau_B=list(tau_B_values), G_Aw=list(couplings), theta=table.tolist())


def capillary_run(L_cap, H, G, tau_A, tau_B, G_Aw, G_Bw):
    """Capillary of length L_cap and height H in the right half of a
    2 L_cap x (H + 2) box; the reservoir holds gas and liquid (Fig. 1)."""
    nx, ny = 2 * L_cap, H + 2
    geom = dict(nx=nx, ny=ny, cap_x0=L_cap, cap_x1=2 * L_cap, y_bot=0, y_top=H + 1)
    prm = dict(G=float(G), tau_A=float(tau_A), tau_B=float(tau_B), G_Aw=float(G_Aw), G_Bw=float(G_Bw))
    return dict(geom=geom, params=prm, init=("slab", L_cap // 2, L_cap + L_cap // 4), rho=RHO)


def capillary_prefactors(samples, L_cap=256, steps=20000, log_every=100, precision="f32", t_min=2000.0):
    """For each (G_Aw, G_Bw, G, tau_A, tau_B, H): the Washburn prefactor
    gamma H cos(theta) / (3 mu_l) obtained from the viscous front law of
    Eq. 15 with both viscosities (twice the slope of
    phi = (mu_l - mu_g) z^2 / 2 + mu_g L z against t, t >= t_min, over mu_l),
    and the prefactor a of the precursor lead
    z_prec - z_bulk = a t^(1/2).  Viscosities mu_k = rho nu_k with the total
    bulk density rho and nu_k = (tau_k - 1/2)/3."""
    runs = [capillary_run(L_cap, int(s[5]), s[2], s[3], s[4], s[0], s[1]) for s in samples]
    kw = np.full(len(runs), np.nan)
    ap = np.full(len(runs), np.nan)
    with Lattice(runs, precision=precision, tile=(128, 16), log_every=log_every,
                 log_capacity=steps // log_every + 2) as lat:
        lat.step(steps)
        for i, s in enumerate(samples):
            lg = lat.log(i)
            t, zb = lg[:, 0], lg[:, 1]
            zp = 0.5 * (lg[:, 2] + lg[:, 3])
            ok = np.isfinite(zb).all() and np.isfinite(zp).all() and zb.max() < 0.9 * L_cap
            if not ok:
                continue
            rho = RHO[0] + RHO[1]
            mu_l = rho * (s[3] - 0.5) / 3.0
            mu_g = rho * (s[4] - 0.5) / 3.0
            phi = 0.5 * (mu_l - mu_g) * zb ** 2 + mu_g * L_cap * zb
            m = t >= t_min
            # slope of the straight line through phi(t) after the start-up
            # transient (its intercept absorbs the transient's lag)
            D = float(np.polyfit(t[m], phi[m], 1)[0])   # = gamma H cos(theta) / 6
            kw[i] = 2.0 * D / mu_l
            ap[i] = A.sqrt_prefactor(t, zp - zb, t_min)
    return kw, ap


def sample_parameters(n, seed, G=(1.0, 1.08), gA=(-0.6, 0.3), gB=(-0.3, 0.5), H=(16, 48), both=None):
    """Seeded draws of (G_Aw, G_Bw, G, tau_A, tau_B, H) inside the stable band
    of the velocity-shift scheme (tau_A = tau_B = 1); half the samples vary
    G_Aw with G_Bw = 0 and half the reverse (the paper's two wetting schemes).
    With both = (G_Aw, (lo, hi)) a third of the samples instead combine the
    two schemes: G_Aw fixed, G_Bw ~ U[lo, hi] (the strongly wetting angles
    that neither scheme reaches alone in the stable band)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X = np.zeros((n, 6))
    nA = n // 3 if both else n // 2
    nB = n // 3 if both else n - nA
    X[:nA, 0] = rng.uniform(*gA, size=nA)
    X[nA:nA + nB, 1] = rng.uniform(*gB, size=nB)
    if both:
        X[nA + nB:, 0] = both[0]
        X[nA + nB:, 1] = rng.uniform(*both[1], size=n - nA - nB)
    X[:, 2] = rng.uniform(*G, size=n)
    X[:, 3] = 1.0
    X[:, 4] = 1.0
    X[:, 5] = rng.integers(H[0], H[1] + 1, size=n)
    return X


def build_dataset(n, seed, droplet_steps=8000, capillary_steps=20000, L_cap=256, precision="f32"):
    """Inputs X (n, 6) and targets T (n, 3) = (cos theta, Washburn prefactor,
    precursor prefactor) measured by the lattice model; rows with a failed
    measurement are dropped."""
    X = sample_parameters(n, seed)
    ang = np.full(n, np.nan)
    for G in np.unique(np.round(X[:, 2], 6)):
        sel = np.where(np.round(X[:, 2], 6) == G)[0]
        ang[sel] = measure_angles([(X[i, 0], X[i, 1]) for i in sel], G, steps=droplet_steps, precision=precision)
    kw, ap = capillary_prefactors(X, L_cap=L_cap, steps=capillary_steps, precision=precision)
    T = np.stack([np.cos(np.radians(ang)), kw, ap], axis=1)
    ok = np.all(np.isfinite(T), axis=1)
    return X[ok], T[ok]


def bisection(targets_deg, fixed, lo=-0.6, hi=0.3, tol_deg=2.0, max_iter=12, precision="f64", steps=8000,
              family="A", other=0.0, droplet=None):
    """Plain lattice-model search: bisection on the varying coupling of a
    one-parameter family for each target angle, all targets advanced in
    lock-step batches.  Family "A": G_Aw varies, G_Bw = other (theta falls as
    G_Aw becomes more attractive); "B": G_Bw varies, G_Aw = other (theta
    falls as G_Bw becomes more repulsive).  droplet: size keywords of the
    judging droplets (measure_angles' defaults if None).  Returns
    (couplings, angles, runs per target)."""
    G, tau_A, tau_B, _ = fixed
    targets = np.asarray(targets_deg, float)
    a = np.full(len(targets), lo)
    b = np.full(len(targets), hi)
    best = np.full(len(targets), np.nan)
    best_ang = np.full(len(targets), np.nan)
    runs = np.zeros(len(targets), int)
    done = np.zeros(len(targets), bool)
    for _ in range(max_iter):
        idx = np.where(~done)[0]
        if len(idx) == 0:
            break
        mid = 0.5 * (a[idx] + b[idx])
        pairs = [(m, other) if family == "A" else (other, m) for m in mid]
        ang = measure_angles(pairs, G, tau_A, tau_B, steps=steps, precision=precision, **(droplet or {}))
        runs[idx] += 1
        for j, i in enumerate(idx):
            best[i], best_ang[i] = mid[j], ang[j]
            if abs(ang[j] - targets[i]) <= tol_deg:
                done[i] = True
            elif (ang[j] > targets[i]) == (family == "A"):
                b[i] = mid[j]       # A too non-wetting: more attraction (more negative G_Aw)
            else:
                a[i] = mid[j]       # B too non-wetting: more repulsion of B (larger G_Bw)
    return best, best_ang, runs


def propose_and_verify(surrogate, targets_deg, fixed, tol_deg=2.0, precision="f64", steps=8000, fallback_iter=10):
    """Surrogate proposals (family G_Bw = 0), each judged by one FP64 droplet
    run; targets missed by more than tol_deg fall back to bisection in a
    bracket around the proposal.  Returns (couplings, angles, runs per target)."""
    targets = np.asarray(targets_deg, float)
    prop = surrogate.propose(np.cos(np.radians(targets)), fixed, family="A")[:, 0]
    ang = measure_angles([(g, 0.0) for g in prop], fixed[0], fixed[1], fixed[2], steps=steps, precision=precision)
    runs = np.ones(len(targets), int)
    miss = np.where(~(np.abs(ang - targets) <= tol_deg))[0]
    if len(miss):
        lo = np.clip(prop[miss] - 0.1, -0.6, 0.3)
        hi = np.clip(prop[miss] + 0.1, -0.6, 0.3)
        for j, i in enumerate(miss):
            c, a2, r = bisection([targets[i]], fixed, lo=lo[j], hi=hi[j], tol_deg=tol_deg, max_iter=fallback_iter,
                                 precision=precision, steps=steps)
            prop[i], ang[i] = c[0], a2[0]
            runs[i] += r[0]
    return prop, ang, runs
