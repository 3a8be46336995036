"""The persistent ring kernel (LBM_KERNEL_RING) through the C ABI.

It evaluates the same canonical order as every other FP32 / FP16S step
kernel (packed FP32 pairs round each component as the scalar operation), so
its populations must equal the default kernel's bit for bit; the default
kernel is in turn checked against the FP64 oracle within the FP32 bound
(tests/test_gpu_parity.py), and so is the ring kernel here on the full
8192x160 workload.  The cases cover the strip edges (odd widths, grids
narrower than one strip, a last strip of a few columns), periodic wrap in x
and y, plates, an explicit solid mask, uneven batches, every ring depth,
graph chunks and the density-ratio species model.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_0807_0602_gb300.lbm import Lattice

pytestmark = pytest.mark.gpu

RINGS = (10,)   # LBM_KERNEL_RING: two columns per consumer thread, packed FP32


def _mask_case():
    nx, ny = 45, 24
    m = np.zeros((ny, nx), np.uint8)
    m[0, 5:40] = 1
    m[12, 0:3] = 1                    # obstacle on the wrap columns
    m[12, 43:45] = 1
    m[7, 20] = 1                      # isolated solid node
    m[15:23, 10] = 1
    m[18, 10] = 0
    m[23, 33:40] = 1                  # next to the plate through the y wrap
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
    g = W.capillary_geometry(243, 7, 0, 243, 0, 6)          # 2 strips + 3 columns
    out["wide243x7"] = (g, W.params(1.0, 1.0, 1.0, -0.1, 0.1), W.random_fields(g, 4, 0.2, 1.2))
    g = W.periodic_box(121, 3)                             # one column past a strip
    out["box121x3"] = (g, W.params(0.9, 0.8, 1.3), W.random_fields(g, 5, 0.2, 1.2))
    geom, prm, nA, nB = _mask_case()
    out["mask45x24"] = (geom, prm, (nA, nB))
    return out


CASES = _cases()


@pytest.mark.parametrize("ring", RINGS)
@pytest.mark.parametrize("prec", ["f32", "f16s"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_ring_kernel_bit_identical_to_default_kernel(name, prec, ring):
    geom, prm, (nA, nB) = CASES[name]
    run = dict(geom=geom, params=prm, init=("fields", nA, nB))
    with Lattice(run, precision=prec, rho_ref=(1.0, 1.0)) as ref:
        ref.step(31)
        want = ref.populations()
        mass = ref.mass()
    for depth, chunk in ((3, -1), (4, 0), (5, 7)):
        with Lattice(run, precision=prec, rho_ref=(1.0, 1.0), tile=(128, 4), kernel=(ring, depth),
                     graph_chunk=chunk) as lat:
            assert lat.schedule == (128, 4, ring, depth)
            lat.step(31)
            got = lat.populations()
            assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (depth, chunk)
            assert np.array_equal(lat.mass(), mass)


@pytest.mark.parametrize("ring", RINGS)
@pytest.mark.parametrize("prec", ["f32", "f16s"])
def test_ring_kernel_bit_identical_with_free_alpha_and_mass(prec, ring):
    geom, prm, (nA, nB) = CASES["capillary300x41"]
    prm = dict(prm, alpha=(4.0 / 9.0, 0.8), mass=(1.0, 25.0 / 9.0))
    run = dict(geom=geom, params=prm, init=("fields", nA, nB))
    with Lattice(run, precision=prec, rho_ref=(1.0, 1.0)) as ref:
        ref.step(25)
        want = ref.populations()
    with Lattice(run, precision=prec, rho_ref=(1.0, 1.0), tile=(128, 4), kernel=(ring, 4)) as lat:
        lat.step(25)
        assert np.array_equal(lat.populations().view(np.uint8), want.view(np.uint8))


@pytest.mark.parametrize("ring", RINGS)
def test_ring_kernel_batched_runs_equal_solo_runs(ring):
    runs = []
    for j, (L, H) in enumerate(((40, 6), (100, 13), (65, 30), (7, 3), (260, 9))):
        runs.append(W.capillary_run(L, H, 1.0 + 0.05 * j, 1.0, 0.8 + 0.1 * j, -0.1 * j))
    with Lattice(runs, precision="f32", tile=(128, 4), kernel=(ring, 4)) as bat:
        bat.step(40)
        batched = [bat.populations(r) for r in range(len(runs))]
        zs = [bat.interface(r) for r in range(len(runs))]
    for r, run in enumerate(runs):
        with Lattice(run, precision="f32", tile=(128, 16)) as solo:
            solo.step(40)
            assert np.array_equal(solo.populations(), batched[r])
            assert np.array_equal(solo.interface(), zs[r])


@pytest.mark.parametrize("ring", RINGS)
@pytest.mark.parametrize("prec", ["f32", "f16s"])
def test_ring_kernel_full_size_capillary_8192x160(prec, ring):
    """The benchmark workload in the ring schedule: the first steps within
    the FP32 bound of the FP64 oracle (FP32), and 200 steps bit-identical to
    the default kernel (both precisions, log on)."""
    c = W.config_capillary_8192x160(tau_B=1.0)
    run = dict(geom=c["geom"], params=c["params"], init=c["init"])
    if prec == "f32":
        nA, nB = W.initial_fields(c)
        ref = oracle.OracleLattice(c["geom"], c["params"], nA, nB)
        ref.step(3)
        fluid = ref.solid() == 0
        rA, rB = ref.densities()
        with Lattice(run, precision="f32", tile=(128, 4), kernel=(ring, 4)) as lat:
            lat.step(3)
            gA, gB = lat.densities()
        for g, r in ((gA, rA), (gB, rB)):
            assert np.max(np.abs(g - r)[fluid]) / np.max(np.abs(r)) <= 1e-5
    outs = []
    for kw in (dict(), dict(tile=(128, 4), kernel=(ring, 4))):
        with Lattice(run, precision=prec, rho_ref=(0.04, 2.0), log_every=50, log_capacity=16, **kw) as lat:
            lat.step(200)
            outs.append((lat.populations(), lat.log(), lat.mass()))
    assert np.array_equal(outs[0][0].view(np.uint8), outs[1][0].view(np.uint8))
    assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][2], outs[1][2])


@pytest.mark.parametrize("ring", RINGS)
def test_ring_kernel_rejected_where_it_does_not_apply(ring):
    from paper_0807_0602_gb300 import _lib as L
    geom, prm, (nA, nB) = CASES["odd17x9"]
    run = dict(geom=geom, params=prm, init=("fields", nA, nB))
    with Lattice(run, precision="f64") as lat:          # FP64 keeps the register kernels
        with pytest.raises(L.LbmError):
            lat.schedule = (128, 4, ring, 4)
    with Lattice(run, precision="f32") as lat:
        for bad in ((64, 4, ring, 4), (128, 4, ring, 2), (128, 4, ring, 6)):
            with pytest.raises(L.LbmError):
                lat.schedule = bad
    g = W.periodic_box(3, 5)
    nA, nB = W.random_fields(g, 1, 0.2, 1.2)
    with Lattice(dict(geom=g, params=prm, init=("fields", nA, nB)), precision="f32") as lat:
        with pytest.raises(L.LbmError):
            lat.schedule = (128, 4, ring, 4)              # ghost windows need nx >= 4
