"""Host-side analysis: fits on constructed data and the front ODE against the
paper's closed form."""
import math

import numpy as np
import pytest

from paper_0807_0602_gb300 import analysis as A


def test_front_ode_reduces_to_eq16_for_equal_fluids():
    # Eq. 15 with rho_l = rho_g and mu_l = mu_g is z'' = 2 g cos / (rho L H) - z' / t_d,
    # whose solution from rest is Eq. 16
    L, H, gamma, ct, rho, mu = 200.0, 40.0, 0.02, math.cos(math.radians(40)), 1.0, 1.0 / 6.0
    t, z = A.front_ode(20000.0, 1.0, 30.0, 0.0, L, H, gamma, ct, rho, rho, mu, mu)
    ref = A.front_equal_fluids(t, 30.0, L, H, gamma, ct, rho, mu)
    assert np.max(np.abs(z - ref)) < 1e-9 * max(1.0, np.abs(ref).max())


def test_front_ode_tends_to_the_viscous_law():
    # late times: inertia negligible, z follows the viscous balance of Eq. 15
    L, H, gamma, ct = 400.0, 20.0, 0.05, 1.0
    rl, rg, ml, mg = 1.0, 0.3, 0.5, 0.05
    t, z = A.front_ode(4e5, 2.0, 10.0, 0.0, L, H, gamma, ct, rl, rg, ml, mg)
    tv = A.viscous_front_time(z, 10.0, L, H, gamma, ct, ml, mg)
    late = t > 2e5
    assert np.max(np.abs(tv[late] - t[late]) / t[late]) < 0.02


def test_washburn_and_sqrt_fits_recover_constructed_prefactors():
    t = np.linspace(0, 1e4, 201)
    z = np.sqrt(100.0 + 0.37 * t)
    k, c = A.washburn_slope(t, z)
    assert k == pytest.approx(0.37, rel=1e-12) and c == pytest.approx(100.0, rel=1e-10)
    assert A.sqrt_prefactor(t, 0.1 * np.sqrt(t)) == pytest.approx(0.1, rel=1e-12)
    assert A.washburn_prefactor(0.02, 40, 1.0, 1 / 6) == pytest.approx(0.02 * 40 / 0.5)


def test_laplace_fit():
    inv_r = 1.0 / np.array([10, 13, 16, 20.0])
    g, c, r2 = A.laplace_gamma(inv_r, 0.02 * inv_r + 1e-5)
    assert g == pytest.approx(0.02, rel=1e-10) and c == pytest.approx(1e-5, rel=1e-6) and r2 > 0.999999


@pytest.mark.parametrize("theta", [30.0, 60.0, 90.0, 120.0])
def test_droplet_angle_of_a_constructed_cap(theta):
    # a circular cap of radius 30 meeting the wall y = 0.5 at angle theta
    ny, nx, R = 96, 160, 30.0
    yc = 0.5 - R * math.cos(math.radians(theta))
    ys, xs = np.mgrid[0:ny, 0:nx].astype(float)
    d = np.hypot(xs - 80.0, ys - yc) - R
    phi = np.clip(-np.tanh(d / 2.0), -0.99, 0.99)
    nA, nB = (1 + phi), (1 - phi)
    nA[0], nB[0] = 0.0, 0.0
    ang, circ = A.droplet_contact_angle(nA, nB, wall_y=0.5, skip_rows=3)
    assert ang == pytest.approx(theta, abs=1.0)


@pytest.mark.parametrize("mu_l,mu_g", [(0.4, 1.05), (1.1, 0.43), (0.5, 0.5)])
def test_campaign_prefactor_recovers_the_viscous_law_of_eq15(mu_l, mu_g):
    """The surrogate campaign's Washburn prefactor fit: a front that follows
    Eq. 15's viscous law exactly, (mu_l - mu_g)(z^2 - z0^2)/2 + mu_g L (z - z0)
    = D t with D = gamma H cos(theta) / 6, plus a start-up lag that shifts t,
    gives back 2 D / mu_l (the Washburn prefactor gamma H cos(theta) / (3 mu_l)),
    whatever the viscosity ratio; records past 0.9 L are left out."""
    from paper_0807_0602_gb300.campaign import capillary_prefactor
    L, z0, D, lag = 2048.0, 400.0, 0.9, 700.0
    t = np.arange(0.0, 60000.0, 500.0)
    a = 0.5 * (mu_l - mu_g)
    b = mu_g * L
    c = -(a * z0 ** 2 + b * z0 + D * np.maximum(t - lag, 0.0))
    z = (-b + np.sqrt(b * b - 4 * a * c)) / (2 * a) if a != 0 else -c / b
    z = np.minimum(z, 0.95 * L)                   # a filled capillary stops at its end
    log = np.column_stack([t, z, z + 5.0, z + 5.0, np.ones_like(t), np.ones_like(t)])
    got = capillary_prefactor(log, L, mu_l, mu_g, t_min=2000.0)
    assert abs(got - 2.0 * D / mu_l) <= 1e-9 * (2.0 * D / mu_l)
    bad = log.copy()
    bad[10, 1] = np.nan                           # a diverged run gives no prefactor
    assert math.isnan(capillary_prefactor(bad, L, mu_l, mu_g, t_min=2000.0))


def test_coupling_for_angle_inverts_a_table_that_is_bilinear_in_g_and_tau_and_linear_in_the_coupling():
    """The calibration-table inversion used to map target angles to wall
    couplings: with theta(G, tau_B, G_Aw) = 80 + 40 G_Aw + 10 (G - 1) - 8 (tau_B - 1)
    (bilinear in G, tau_B and linear in the coupling, so interpolation is
    exact), a target angle anywhere inside the grid comes back as the exact
    coupling; angles beyond the table's range give its end couplings."""
    from paper_0807_0602_gb300.calibrate import coupling_for_angle
    Gs, taus, cps = np.array([1.0, 1.05, 1.1]), np.array([1.0, 1.25, 1.5]), np.linspace(-0.5, 0.3, 9)
    th = lambda G, t, a: 80.0 + 40.0 * a + 10.0 * (G - 1.0) - 8.0 * (t - 1.0)   # noqa: E731
    table = np.array([[[th(G, t, a) for a in cps] for t in taus] for G in Gs])
    rng = np.random.default_rng(5)
    for _ in range(50):
        G, t, a = rng.uniform(1.0, 1.1), rng.uniform(1.0, 1.5), rng.uniform(-0.5, 0.3)
        got = coupling_for_angle(table, Gs, taus, cps, G, t, th(G, t, a))
        assert abs(got - a) < 1e-12
    assert coupling_for_angle(table, Gs, taus, cps, 1.05, 1.2, 10.0) == -0.5
    assert coupling_for_angle(table, Gs, taus, cps, 1.05, 1.2, 170.0) == 0.3


@pytest.mark.parametrize("family,other", [("A", 0.0), ("B", -0.5)])
def test_bisection_walks_each_coupling_family_the_right_way(monkeypatch, family, other):
    """The lattice-model bisection on a one-parameter coupling family, with
    the droplet runs replaced by a monotone angle law (the angle falls as
    G_Aw falls in family A, and as G_Bw rises in family B at fixed G_Aw):
    every target inside the family's reach is met within the tolerance and
    the other coupling stays fixed."""
    from paper_0807_0602_gb300 import calibrate as Cb
    seen = []

    def fake(pairs, G, tau_A, tau_B, steps=0, precision="", **kw):
        seen.extend(pairs)
        return np.array([80.0 + 60.0 * a - 70.0 * b for a, b in pairs])
    monkeypatch.setattr(Cb, "measure_angles", fake)
    lo, hi = (-0.5, 0.3) if family == "A" else (0.0, 0.6)
    law = (lambda g: 80.0 + 60.0 * g) if family == "A" else (lambda g: 80.0 + 60.0 * other - 70.0 * g)
    targets = np.array([law(lo) + f * (law(hi) - law(lo)) for f in (0.1, 0.35, 0.6, 0.9)])
    c, ang, runs = Cb.bisection(targets, (1.0, 1.0, 1.0, 64.0), lo=lo, hi=hi, tol_deg=0.5, max_iter=20,
                                family=family, other=other)
    assert np.all(np.abs(ang - targets) <= 0.5)
    assert np.all((c >= lo) & (c <= hi)) and np.all(runs >= 1)
    fixed_col = 1 if family == "A" else 0
    assert all(p[fixed_col] == other for p in seen)
