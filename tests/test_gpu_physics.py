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
