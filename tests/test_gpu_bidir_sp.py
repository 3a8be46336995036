"""The species-packed bidirectional march (LBM_KERNEL_BIDIR_SP) through the
C ABI.

Species A and B share one packed FP32 instruction per operation of the
collision; every lane rounds as the scalar operation in the canonical order,
so the populations must equal the default kernel's bit for bit (FP32 and
FP16S storage); the default kernel is checked against the FP64 oracle in
tests/test_gpu_parity.py, and so is this one on the full 8192x160 workload.
The cases cover strip edges, grids narrower than a strip, periodic wrap,
plates and masks, uneven batches, graph chunks, tall and one-row tiles and
the density-ratio species model (free alpha_k, m_k: the packed coefficients
of the generalised equilibria).
"""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_0807_0602_gb300.lbm import Lattice

pytestmark = pytest.mark.gpu

SP = 12
IND = 11


def _mask_case():
    nx, ny = 45, 24
    m = np.zeros((ny, nx), np.uint8)
    m[0, 5:40] = 1
    m[12, 0:3] = 1
    m[12, 43:45] = 1
    m[7, 20] = 1
    m[15:23, 10] = 1
    m[23, 33:40] = 1
    geom = dict(nx=nx, ny=ny, cap_x0=0, cap_x1=0, y_bot=-1, y_top=-1, mask=m)
    nA, nB = W.random_fields(geom, 7, 0.2, 1.2)
    return geom, W.params(1.1, 1.0, 0.8, -0.2, 0.1), nA, nB


def _cases():
    out = {}
    g = W.capillary_geometry(300, 41, 60, 280, 0, 40)
    out["capillary300x41"] = (g, W.params(1.2, 1.0, 0.9, -0.1, 0.05), W.random_fields(g, 1, 0.2, 1.2))
    g = W.capillary_geometry(17, 9, 3, 14, 1, 7)
    out["odd17x9"] = (g, W.params(1.1, 1.2, 0.8, 0.1, -0.1), W.random_fields(g, 2, 0.2, 1.2))
    g = W.capillary_geometry(5, 4, 1, 4, 0, -1)
    out["tiny5x4"] = (g, W.params(1.0, 1.0, 0.7, -0.2, 0.0), W.random_fields(g, 3, 0.2, 1.2))
    g = W.capillary_geometry(251, 7, 0, 251, 0, 6)          # strips of 62 / 126 plus a few columns
    out["wide251x7"] = (g, W.params(1.0, 1.0, 1.0, -0.1, 0.1), W.random_fields(g, 4, 0.2, 1.2))
    g = W.capillary_geometry(1500, 300, 100, 1400, 20, 280)  # more units than CTAs: shares of many rows
    out["large1500x300"] = (g, W.params(1.0, 1.0, 0.8, -0.1, 0.0), W.random_fields(g, 6, 0.3, 1.1))
    geom, prm, nA, nB = _mask_case()
    out["mask45x24"] = (geom, prm, (nA, nB))
    return out


CASES = _cases()


@pytest.mark.parametrize("kv", [SP, IND])
@pytest.mark.parametrize("prec", ["f32", "f16s", "f64"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_packed_kernel_bit_identical_to_default_kernel(name, prec, kv):
    if kv == SP and prec == "f64":
        pytest.skip("FP32 arithmetic only")
    geom, prm, (nA, nB) = CASES[name]
    run = dict(geom=geom, params=prm, init=("fields", nA, nB))
    with Lattice(run, precision=prec, rho_ref=(1.0, 1.0)) as ref:
        ref.step(23)
        want = ref.populations()
        mass = ref.mass()
    for Wd, R, chunk in ((64, 4, -1), (128, 8, 5), (64, 1, 0), (128, 33, -1)):
        if prec == "f64" and Wd != 64:
            continue
        with Lattice(run, precision=prec, rho_ref=(1.0, 1.0), tile=(Wd, R), kernel=(kv, 4),
                     graph_chunk=chunk) as lat:
            assert lat.schedule == (Wd, R, kv, 4)
            lat.step(23)
            got = lat.populations()
            assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (Wd, R, chunk)
            assert np.array_equal(lat.mass(), mass)


@pytest.mark.parametrize("kv", [SP, IND])
@pytest.mark.parametrize("prec", ["f32", "f16s"])
def test_packed_kernel_bit_identical_with_free_alpha_and_mass(prec, kv):
    geom, prm, (nA, nB) = CASES["capillary300x41"]
    prm = dict(prm, alpha=(4.0 / 9.0, 0.8), mass=(1.0, 25.0 / 9.0))
    run = dict(geom=geom, params=prm, init=("fields", nA, nB))
    with Lattice(run, precision=prec, rho_ref=(1.0, 1.0)) as ref:
        ref.step(25)
        want = ref.populations()
    with Lattice(run, precision=prec, rho_ref=(1.0, 1.0), tile=(64, 4), kernel=(kv, 4)) as lat:
        lat.step(25)
        assert np.array_equal(lat.populations().view(np.uint8), want.view(np.uint8))


@pytest.mark.parametrize("n_runs", [5, 700])
def test_packed_kernel_batched_runs_equal_solo_runs(n_runs):
    """5 uneven capillaries and 700 small ones in one handle equal the same
    runs advanced alone (populations, fronts, velocities)."""
    rng = np.random.default_rng(n_runs)
    runs = []
    for j in range(n_runs):
        if n_runs == 5:
            L, H = ((40, 6), (100, 13), (65, 30), (7, 3), (260, 9))[j]
        else:
            L, H = int(rng.integers(6, 40)), int(rng.integers(3, 12))
        runs.append(W.capillary_run(L, H, 1.0 + 0.01 * (j % 5), 1.0, 0.8 + 0.05 * (j % 4), -0.05 * (j % 3)))
    with Lattice(runs, precision="f32", tile=(64, 4), kernel=(SP, 4)) as bat:
        bat.step(40)
        batched = [bat.populations(r) for r in range(len(runs))]
        zs = [bat.interface(r) for r in range(len(runs))]
        vel = [bat.velocity(r) for r in (0, len(runs) - 1)]
    for r in sorted({0, 1, len(runs) // 2, len(runs) - 1}):
        with Lattice(runs[r], precision="f32", tile=(128, 16)) as solo:
            solo.step(40)
            assert np.array_equal(solo.populations(), batched[r])
            assert np.array_equal(solo.interface(), zs[r])
            if r in (0, len(runs) - 1):
                ux, uy = solo.velocity()
                k = 0 if r == 0 else 1
                assert np.allclose(vel[k][0], ux, rtol=0, atol=1e-12)
                assert np.allclose(vel[k][1], uy, rtol=0, atol=1e-12)


def test_packed_kernel_full_size_capillary_8192x160():
    """The benchmark workload: the first steps within the FP32 bound of the
    FP64 oracle, and 200 steps (log on) bit-identical to the default kernel."""
    c = W.config_capillary_8192x160(tau_B=1.0)
    run = dict(geom=c["geom"], params=c["params"], init=c["init"])
    nA, nB = W.initial_fields(c)
    ref = oracle.OracleLattice(c["geom"], c["params"], nA, nB)
    ref.step(3)
    fluid = ref.solid() == 0
    rA, rB = ref.densities()
    with Lattice(run, precision="f32", tile=(64, 4), kernel=(SP, 4)) as lat:
        lat.step(3)
        gA, gB = lat.densities()
    for g, r in ((gA, rA), (gB, rB)):
        assert np.max(np.abs(g - r)[fluid]) / np.max(np.abs(r)) <= 1e-5
    outs = []
    for kw in (dict(), dict(tile=(64, 8), kernel=(SP, 4)), dict(tile=(128, 4), kernel=(SP, 4)),
               dict(tile=(64, 8), kernel=(IND, 4))):
        with Lattice(run, precision="f32", rho_ref=(0.04, 2.0), log_every=50, log_capacity=16, **kw) as lat:
            lat.step(200)
            outs.append((lat.populations(), lat.log(), lat.mass()))
    for o in outs[1:]:
        assert np.array_equal(outs[0][0].view(np.uint8), o[0].view(np.uint8))
        assert np.array_equal(outs[0][1], o[1]) and np.array_equal(outs[0][2], o[2])


def test_packed_kernel_rejected_where_it_does_not_apply():
    from paper_0807_0602_gb300 import _lib as L
    geom, prm, (nA, nB) = CASES["odd17x9"]
    run = dict(geom=geom, params=prm, init=("fields", nA, nB))
    with Lattice(run, precision="f64") as lat:          # FP32 arithmetic only
        with pytest.raises(L.LbmError):
            lat.schedule = (64, 4, SP, 4)
    with Lattice(run, precision="f32") as lat:
        for bad in ((256, 4, SP, 4), (32, 4, SP, 4), (64, 4, SP, 5)):
            with pytest.raises(L.LbmError):
                lat.schedule = bad
