"""The bidirectional march compiled at run time for the handle's grid
(LBM_KERNEL_BIDIR_JIT) through the C ABI.

It is the source of LBM_KERNEL_BIDIR with the run's sizes as constants,
compiled with the same floating-point options, so its populations must equal
the default kernel's bit for bit in every precision (and, in FP64, the
oracle's, which tests/test_gpu_parity.py checks for the default kernel; the
full-size case here also checks the first steps against the oracle).  The
cases cover strip edges, grids narrower than a strip, periodic wrap, plates
and masks, tile heights from one row to taller than the grid, graph chunks,
the density-ratio species model and the 8192x160 workload with its log.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_0807_0602_gb300.lbm import Lattice

pytestmark = pytest.mark.gpu

JIT = 11


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
    g = W.capillary_geometry(251, 7, 0, 251, 0, 6)
    out["wide251x7"] = (g, W.params(1.0, 1.0, 1.0, -0.1, 0.1), W.random_fields(g, 4, 0.2, 1.2))
    geom, prm, nA, nB = _mask_case()
    out["mask45x24"] = (geom, prm, (nA, nB))
    return out


CASES = _cases()


@pytest.mark.parametrize("prec", ["f32", "f16s", "f64"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_compiled_kernel_bit_identical_to_default_kernel(name, prec):
    geom, prm, (nA, nB) = CASES[name]
    run = dict(geom=geom, params=prm, init=("fields", nA, nB))
    with Lattice(run, precision=prec, rho_ref=(1.0, 1.0)) as ref:
        ref.step(23)
        want = ref.populations()
        mass = ref.mass()
    for Wd, R, chunk in ((64, 4, -1), (128, 9, 5), (64, 1, 0), (128, 50, -1)):
        if prec == "f64" and Wd != 64:
            continue
        with Lattice(run, precision=prec, rho_ref=(1.0, 1.0), tile=(Wd, R), kernel=(JIT, 4),
                     graph_chunk=chunk) as lat:
            assert lat.schedule == (Wd, R, JIT, 4)
            lat.step(23)
            assert np.array_equal(lat.populations().view(np.uint8), want.view(np.uint8)), (Wd, R, chunk)
            assert np.array_equal(lat.mass(), mass)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_compiled_kernel_with_free_alpha_and_mass(prec):
    geom, prm, (nA, nB) = CASES["capillary300x41"]
    prm = dict(prm, alpha=(4.0 / 9.0, 0.8), mass=(1.0, 25.0 / 9.0))
    run = dict(geom=geom, params=prm, init=("fields", nA, nB))
    with Lattice(run, precision=prec) as ref:
        ref.step(25)
        want = ref.populations()
        uref = ref.velocity()
    with Lattice(run, precision=prec, tile=(64, 6), kernel=(JIT, 4)) as lat:
        lat.step(25)
        assert np.array_equal(lat.populations().view(np.uint8), want.view(np.uint8))
        u = lat.velocity()
        assert np.array_equal(u[0], uref[0]) and np.array_equal(u[1], uref[1])


def test_compiled_kernel_full_size_capillary_8192x160():
    """The benchmark workload: the first steps within the FP32 bound of the
    FP64 oracle, and 200 steps (log on) bit-identical to the default kernel
    at both strip widths."""
    c = W.config_capillary_8192x160(tau_B=1.0)
    run = dict(geom=c["geom"], params=c["params"], init=c["init"])
    nA, nB = W.initial_fields(c)
    ref = oracle.OracleLattice(c["geom"], c["params"], nA, nB)
    ref.step(3)
    fluid = ref.solid() == 0
    rA, rB = ref.densities()
    with Lattice(run, precision="f32", tile=(64, 18), kernel=(JIT, 4)) as lat:
        lat.step(3)
        gA, gB = lat.densities()
    for g, r in ((gA, rA), (gB, rB)):
        assert np.max(np.abs(g - r)[fluid]) / np.max(np.abs(r)) <= 1e-5
    outs = []
    for kw in (dict(), dict(tile=(64, 18), kernel=(JIT, 4)), dict(tile=(128, 9), kernel=(JIT, 4))):
        with Lattice(run, precision="f32", rho_ref=(0.04, 2.0), log_every=50, log_capacity=16, **kw) as lat:
            lat.step(200)
            outs.append((lat.populations(), lat.log(), lat.mass()))
    for o in outs[1:]:
        assert np.array_equal(outs[0][0].view(np.uint8), o[0].view(np.uint8))
        assert np.array_equal(outs[0][1], o[1]) and np.array_equal(outs[0][2], o[2])


def test_compiled_kernel_needs_a_single_run_and_a_bidirectional_tiling():
    from paper_0807_0602_gb300 import _lib as L
    runs = [W.capillary_run(40, 6, 1.0, 1.0, 1.0, -0.1), W.capillary_run(60, 9, 1.0, 1.0, 1.0, -0.1)]
    with Lattice(runs, precision="f32") as lat:            # a batch: one grid per kernel is not possible
        with pytest.raises(L.LbmError):
            lat.schedule = (64, 4, JIT, 4)
    geom, prm, (nA, nB) = CASES["odd17x9"]
    run = dict(geom=geom, params=prm, init=("fields", nA, nB))
    with Lattice(run, precision="f64") as lat:
        for bad in ((128, 4, JIT, 4), (256, 4, JIT, 4), (64, 4, JIT, 5)):
            with pytest.raises(L.LbmError):
                lat.schedule = bad
