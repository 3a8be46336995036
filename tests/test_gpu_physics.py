"""The production path reproduces the paper's capillary-filling law at the
paper's own scale (capillary length L = 200, H = 40; Numerical Results
section, Fig. 3): equal-fluid filling follows Eq. 16 with gamma from
Laplace's law and theta from a sessile droplet, all three measured on the GPU
through the C ABI.  The precursor lead over the bulk front (Fig. 8) is
tracked and reported."""
import json
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
G = 1.0


def _lattice(*a, **k):
    from paper_0807_0602_gb300.build import build
    build()
    from paper_0807_0602_gb300.lbm import Lattice
    return Lattice(*a, **k)


def _gamma():
    inv_r, dp = [], []
    for R in (10, 14, 18, 22):
        geom = W.periodic_box(96, 96)
        nA, nB = W.droplet_fields(geom, 47.5, 47.5, R)
        with _lattice(dict(geom=geom, params=W.params(G, 1.0, 1.0), init=("fields", nA, nB)),
                      precision="f64") as lat:
            lat.step(6000)
            a, b = lat.densities()
        p = (a + b) / 3.0 + G * a * b / 3.0
        a_in, a_out = a[46:50, 46:50].mean(), a[:4, :4].mean()
        inv_r.append(1.0 / math.sqrt((a - a_out).sum() / (a_in - a_out) / math.pi))
        dp.append(p[46:50, 46:50].mean() - p[:4, :4].mean())
    A = np.vstack([inv_r, np.ones(4)]).T
    (g, c), res, *_ = np.linalg.lstsq(A, np.array(dp), rcond=None)
    return g, 1 - res[0] / ((np.array(dp) - np.mean(dp)) ** 2).sum()


def _theta(G_Aw):
    from paper_0807_0602_gb300 import calibrate as Cb
    return float(Cb.measure_angles([(G_Aw, 0.0)], G, precision="f64", steps=8000)[0])


def _front(L, H, G_Aw, steps, every=100):
    from paper_0807_0602_gb300 import calibrate as Cb
    run = Cb.capillary_run(L, H, G, 1.0, 1.0, G_Aw, 0.0)
    with _lattice(run, precision="f64", log_every=every, log_capacity=steps // every + 2) as lat:
        lat.step(steps)
        lg = lat.log()
    return lg[:, 0], lg[:, 1], 0.5 * (lg[:, 2] + lg[:, 3])


def test_filling_follows_eq16_at_the_papers_scale():
    gamma, r2_lap = _gamma()
    theta = _theta(-0.3)
    L, H = 200, 40
    t, z, _ = _front(L, H, -0.3, 15000)
    rho = 2.04
    mu = rho * 0.5 / 3.0
    td = rho * H * H / (12.0 * mu)
    f = td * (np.exp(-t / td) + t / td - 1.0)
    (A16, z0), res, *_ = np.linalg.lstsq(np.vstack([f, np.ones_like(f)]).T, z, rcond=None)
    r2_16 = 1 - res[0] / ((z - z.mean()) ** 2).sum()
    _, resw, *_ = np.linalg.lstsq(np.vstack([t, np.ones_like(t)]).T, z * z, rcond=None)
    r2_w = 1 - resw[0] / ((z * z - (z * z).mean()) ** 2).sum()
    pred = gamma * H * math.cos(math.radians(theta)) / (6.0 * mu * L)
    rep = dict(gamma=gamma, laplace_r2=r2_lap, theta_deg=theta, td=td, prefactor=A16, predicted=pred,
               ratio=A16 / pred, r2_eq16=r2_16, r2_washburn_form=r2_w, z_start=z[0], z_end=z[-1])
    print("eq16:", json.dumps({k: float(v) for k, v in rep.items()}))
    assert r2_lap > 0.999 and gamma > 0
    assert z[-1] > z[0] + 20.0
    assert r2_16 > 0.999 and r2_16 > r2_w
    assert 0.6 < rep["ratio"] < 1.2


def test_precursor_lead_under_strong_wetting():
    """Strong wetting (theta about 9 degrees): the wall-row front (n_A above
    rho_bulk / 3) leads the bulk front.  In this model the lead settles at
    about the meniscus offset (10 nodes for H = 40) instead of growing as
    t^(1/2) as in the paper's Fig. 8; the test checks the lead is tracked and
    positive while the reservoir feeds the capillary and reports its fit."""
    from paper_0807_0602_gb300 import analysis as A
    L, H = 200, 40
    t, zb, zp = _front(L, H, -1.0, 6000)
    lead = zp - zb
    m = (t >= 1000) & (zb > 0.0) & (zb < 0.8 * L)
    a = A.sqrt_prefactor(t[m], lead[m])
    rep = dict(sqrt_prefactor=a, points=int(m.sum()), lead=[float(v) for v in lead[::10]],
               bulk=[float(v) for v in zb[::10]])
    print("precursor:", json.dumps(rep))
    assert m.sum() >= 20
    assert np.all(lead[m] > 0.0)
    assert zb[m][-1] > zb[m][0] + 20.0


def _phase_viscosity(nA, nB, tau_A, tau_B):
    """Dynamic viscosity of a bulk phase: the species' partial viscosities
    n_k (tau_k - 1/2)/3 add."""
    return (nA * (tau_A - 0.5) + nB * (tau_B - 0.5)) / 3.0


def _viscous_front(tau_A, tau_B, steps, L=200, H=40, every=250):
    """FP64 capillary of the paper's size with a reservoir that can fill it;
    returns t, z of the bulk front (t >= 1000, z < 0.9 L), the phase densities
    and viscosities of liquid (at the inlet) and gas (ahead of the front)."""
    run = W.capillary_run_long_reservoir(L, H, G, tau_A, tau_B, -0.3, 0.0)
    with _lattice(run, precision="f64", log_every=every, log_capacity=steps // every + 2) as lat:
        lat.step(3000)            # phases settled; the front still far from the outlet
        nA, nB = lat.densities()
        lat.step(steps - 3000)
        lg = lat.log()
    mid = (H + 2) // 2
    liq = (nA[mid, 2 * L + 3], nB[mid, 2 * L + 3])
    gas = (nA[mid, 3 * L - 3], nB[mid, 3 * L - 3])
    t, z = lg[:, 0], lg[:, 1]
    m = (t >= 1000) & (z < 0.9 * L)
    return t[m], z[m], liq, gas, _phase_viscosity(*liq, tau_A, tau_B), _phase_viscosity(*gas, tau_A, tau_B)


def test_viscosity_ratio_front_law_and_the_front_ode_at_the_papers_scale():
    """Theoretical analysis, Eqs. 13-15, at L = 200, H = 40 (FP64, GPU):
    - gas 2.7 times more viscous than the liquid (tau_B = 2): the front speeds
      up as the gas column shortens; the viscous law of Eq. 15,
      F(z) = mu_g L z + (mu_l - mu_g) z^2 / 2 linear in t, fits better than a
      constant speed and than Washburn's z^2 ~ t (Eq. 1), and the speed-up
      lies between none and the one Eq. 15 predicts (the liquid's film along
      the walls ahead of the front lowers the gas column's resistance);
    - the front-dynamics equation (Eq. 15 with inertia, integrated by RK4 in
      analysis.front_ode, where the paper used Mathematica) with the measured
      phase densities and viscosities and one fitted driving constant
      gamma cos(theta) follows the lattice front to within 5 % of its travel
      (measured: 3.0 % of 128 lattice units; the ODE curves more than the
      lattice front, whose speed-up is 1.36 against Eq. 15's 1.65);
    - liquid 2.8 times more viscous (tau_A = 2): reported only.  Eq. 15
      predicts a slow-down to 0.77 of the early speed; the lattice front
      instead speeds up slightly (1.12 over 61 lattice units)."""
    from paper_0807_0602_gb300 import analysis as A
    L, H = 200, 40
    t, z, liq, gas, mu_l, mu_g = _viscous_front(1.0, 2.0, 60000)
    assert mu_g > 2.0 * mu_l and len(t) >= 40 and z[-1] > z[0] + L / 3.0
    M = np.vstack([t, np.ones_like(t)]).T
    a, b = 0.5 * (mu_l - mu_g), mu_g * L
    kF, cF = np.linalg.lstsq(M, b * z + a * z * z, rcond=None)[0]
    z15 = (-b + np.sqrt(b * b + 4 * a * (kF * t + cF))) / (2 * a)
    kz, cz = np.linalg.lstsq(M, z, rcond=None)[0]
    kw, cw = np.linalg.lstsq(M, z * z, rcond=None)[0]
    rms = lambda e: float(np.sqrt(np.mean(e * e)))
    rms15, rms_lin, rms_w = rms(z15 - z), rms(kz * t + cz - z), rms(np.sqrt(np.maximum(kw * t + cw, 0)) - z)
    q = len(t) // 4
    v = np.diff(z) / np.diff(t)
    up = v[-q:].mean() / v[:q].mean()
    up_pred = (b + 2 * a * z[: q + 1].mean()) / (b + 2 * a * z[-q - 1:].mean())
    # Eq. 15 with inertia from the first kept point; gamma cos(theta) = 6 kF / H
    rho_l, rho_g = liq[0] + liq[1], gas[0] + gas[1]
    k0 = max(1, q // 2)
    zdot0 = float(np.polyfit(t[:k0 + 1], z[:k0 + 1], 1)[0])
    dt = 5.0
    ts, zs = A.front_ode(t[-1] - t[0], dt, z[0], zdot0, L, H, 6.0 * kF / H, 1.0, rho_l, rho_g, mu_l, mu_g)
    z_ode = np.interp(t - t[0], ts, zs)
    dev = float(np.max(np.abs(z_ode - z)) / (z[-1] - z[0]))
    t2, z2, liq2, gas2, mu_l2, mu_g2 = _viscous_front(2.0, 1.0, 90000)
    q2 = len(t2) // 4
    v2 = np.diff(z2) / np.diff(t2)
    a2, b2 = 0.5 * (mu_l2 - mu_g2), mu_g2 * L
    rep = dict(mu_l=mu_l, mu_g=mu_g, rms_eq15=rms15, rms_linear=rms_lin, rms_washburn=rms_w, speedup=up,
               speedup_eq15=up_pred, gamma_cos_fit=6.0 * kF / H, ode_max_dev_of_travel=dev,
               travel=float(z[-1] - z[0]), viscous_liquid=dict(
                   mu_l=mu_l2, mu_g=mu_g2, travel=float(z2[-1] - z2[0]),
                   slowdown=float(v2[-q2:].mean() / v2[:q2].mean()),
                   slowdown_eq15=float((b2 + 2 * a2 * z2[: q2 + 1].mean()) / (b2 + 2 * a2 * z2[-q2 - 1:].mean()))))
    print("viscosity ratio:", json.dumps({k: (float(v) if not isinstance(v, dict) else v) for k, v in rep.items()}))
    assert kF > 0 and rms15 < rms_lin < rms_w
    assert 1.1 < up <= up_pred
    assert dev < 0.05
    assert len(t2) >= 40 and rep["viscous_liquid"]["travel"] > 20.0
