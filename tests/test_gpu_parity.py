"""GPU path (through the C ABI) against the FP64 CPU oracle.

FP64 kernels are built without multiply-add contraction and follow the same
canonical order as the oracle, so they must agree to 1e-12 relative (in
practice bit for bit).  FP32 and FP16-shifted storage are compared with the
tolerances stated in each test.  Schedules (tilings, CUDA graphs, batching)
must not change a single bit.
"""
import os

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_0807_0602_gb300 import build as B
    B.build()
    oracle.build()


def Lattice(*a, **k):
    from paper_0807_0602_gb300.lbm import Lattice as _L
    return _L(*a, **k)


def rel_err(a, b, fluid):
    a, b = a[fluid], b[fluid]
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


CASES = {
    "box16x8": (W.periodic_box(16, 8), W.params(1.0, 0.8, 1.3), "random"),
    "capillary64x18": (W.capillary_geometry(64, 18, 16, 48, 0, 17), W.params(1.2, 1.0, 0.9, -0.1, 0.05), "slab"),
    "odd17x9": (W.capillary_geometry(17, 9, 3, 14, 1, 7), W.params(1.1, 1.2, 0.8, 0.1, -0.1), "random"),
    "tiny5x4": (W.capillary_geometry(5, 4, 1, 4, 0, 3), W.params(0.9, 1.0, 1.0, -0.2, 0.0), "random"),
    "row3x1": (W.periodic_box(3, 1), W.params(0.8, 1.0, 0.7), "random"),
    "wide300x5": (W.capillary_geometry(300, 5, 0, 300, 0, 4), W.params(1.0, 1.0, 1.0, -0.1, 0.1), "random"),
}


def _fields(geom, kind, seed=0):
    if kind == "random":
        return W.random_fields(geom, seed, 0.2, 1.2)
    return W.slab_fields(geom, 0, geom["nx"] // 3)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("steps", [1, 10, 100])
def test_fp64_matches_oracle(name, steps):
    geom, prm, kind = CASES[name]
    nA, nB = _fields(geom, kind)
    ref = oracle.OracleLattice(geom, prm, nA, nB)
    ref.step(steps)
    fluid = ref.solid() == 0
    with Lattice(dict(geom=geom, params=prm, init=("fields", nA, nB)), precision="f64") as lat:
        lat.step(steps)
        F = lat.populations()
        gA, gB = lat.densities()
        ux, uy = lat.velocity()
        M = lat.mass()
    Fr = ref.populations()
    assert np.max(np.abs(F - Fr)[:, :, fluid] / np.maximum(np.abs(Fr[:, :, fluid]), 1e-300)) <= 1e-12
    rA, rB = ref.densities()
    assert rel_err(gA, rA, fluid) <= 1e-12 and rel_err(gB, rB, fluid) <= 1e-12
    vx, vy = ref.velocity()
    scale = max(np.abs(vx).max(), np.abs(vy).max(), 1e-300)
    assert np.max(np.abs(ux - vx)) <= 1e-12 * scale and np.max(np.abs(uy - vy)) <= 1e-12 * scale
    Mr = ref.mass()
    assert np.all(np.abs(M - Mr) <= 1e-12 * Mr)


def test_fp64_fronts_and_log_match_oracle():
    geom = W.capillary_geometry(128, 26, 32, 96, 0, 25)
    prm = W.params(1.2, 1.0, 1.0, -0.15, 0.0)
    nA, nB = W.slab_fields(geom, 0, 48)
    ref = oracle.OracleLattice(geom, prm, nA, nB)
    with Lattice(dict(geom=geom, params=prm, init=("fields", nA, nB)), precision="f64", log_every=25,
                 log_capacity=64) as lat:
        want = []
        for k in range(8):
            want.append((ref.t, *ref.interface(), *ref.mass()))
            ref.step(25)
        want.append((ref.t, *ref.interface(), *ref.mass()))
        lat.step(200)
        log = lat.log()
        z = lat.interface()
    want = np.array(want)
    assert log.shape == want.shape
    assert np.array_equal(log[:, 0], want[:, 0])
    assert np.max(np.abs(log[:, 1:4] - want[:, 1:4])) <= 1e-10
    assert np.all(np.abs(log[:, 4:] - want[:, 4:]) <= 1e-12 * want[:, 4:])
    assert np.max(np.abs(z - ref.interface())) <= 1e-10


def test_fp64_capillary_256x32_3000_steps_matches_oracle():
    c = W.config_capillary_256x32()
    prm = dict(c["params"], tau_B=1.0)
    nA, nB = W.initial_fields(c)
    ref = oracle.OracleLattice(c["geom"], prm, nA, nB)
    ref.step(3000)
    with Lattice(dict(geom=c["geom"], params=prm, init=c["init"]), precision="f64") as lat:
        lat.step(3000)
        gA, gB = lat.densities()
        z = lat.interface()
    fluid = ref.solid() == 0
    rA, rB = ref.densities()
    assert rel_err(gA, rA, fluid) <= 1e-12 and rel_err(gB, rB, fluid) <= 1e-12
    assert np.max(np.abs(z - ref.interface())) <= 1e-10


def test_analytic_slab_and_droplet_init_equal_field_init():
    geom = W.capillary_geometry(50, 20, 10, 40, 0, 19)
    prm = W.params(1.0, 1.0, 1.0)
    for init, fields in ((("slab", 0, 17), W.slab_fields(geom, 0, 17)),
                         (("droplet", 25.0, 9.5, 6.3), W.droplet_fields(geom, 25.0, 9.5, 6.3))):
        with Lattice(dict(geom=geom, params=prm, init=init), precision="f64") as a, \
                Lattice(dict(geom=geom, params=prm, init=("fields", *fields)), precision="f64") as b:
            assert np.array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("prec", ["f64", "f32", "f16s"])
def test_results_independent_of_tiling_and_graphs(prec):
    geom = W.capillary_geometry(333, 37, 50, 300, 2, 30)
    prm = W.params(1.2, 1.0, 0.9, -0.1, 0.05)
    run = dict(geom=geom, params=prm, init=("slab", 0, 120))
    scheds = [((128, 16), 0, None), ((64, 1), -1, None), ((64, 3), 5, None), ((256, 37), 0, None),
              ((128, 100), 7, None)]
    if prec != "f16s":
        scheds += [((128, 16), 0, (1, 4)), ((64, 5), -1, (1, 3)), ((256, 8), 3, (1, 4)), ((64, 40), 0, (1, 4))]
    scheds += [((128, 16), 0, (2, 4)), ((64, 1), -1, (2, 4)), ((256, 7), 5, (2, 4)), ((64, 37), 0, (2, 4))]
    scheds += [((128, 16), 0, (2, 6)), ((64, 5), -1, (2, 8)), ((128, 3), 5, (2, 8))]
    if prec != "f64":   # FP64 at W = 256, depth 6 needs more than 227 KB of shared memory: rejected
        scheds += [((256, 3), 5, (2, 6))]
    scheds += [((64, 16), 0, (3, 4)), ((64, 1), -1, (3, 4)), ((64, 9), 5, (3, 4)), ((64, 37), 0, (3, 4))]
    if prec != "f64":   # the pipelined kernel takes W <= 64 in FP64
        scheds += [((128, 2), 0, (3, 4)), ((128, 9), 5, (3, 4))]
    scheds += [((128, 16), 0, (4, 4)), ((64, 1), -1, (4, 4)), ((256, 9), 5, (4, 4)), ((64, 37), 0, (4, 4))]
    scheds += [((128, 16), 0, (5, 4)), ((64, 1), -1, (5, 4)), ((256, 9), 5, (5, 4)), ((64, 37), 0, (5, 4))]
    scheds += [((128, 16), 0, (6, 4)), ((64, 1), -1, (6, 4)), ((128, 9), 5, (6, 4)), ((64, 37), 0, (6, 4))]
    if prec != "f64":   # FP64 at W = 256 exceeds that kernel's static shared memory and is rejected
        scheds += [((256, 9), 5, (6, 4))]
    scheds += [((64, 16), 0, (7, 4)), ((64, 1), -1, (7, 4)), ((64, 9), 5, (7, 4)), ((64, 37), 0, (7, 4))]
    if prec != "f64":   # the pair kernel takes W <= 64 in FP64
        scheds += [((128, 7), 5, (7, 4)), ((128, 37), 0, (7, 4))]
    scheds += [((32, 14), 0, (8, 4)), ((32, 6), -1, (8, 4)), ((64, 6), 5, (8, 4)), ((32, 30), 0, (8, 4)),
               ((64, 14), 7, (8, 4))]
    scheds += [((64, 8), 0, (9, 4)), ((64, 1), -1, (9, 4)), ((64, 7), 5, (9, 4)), ((64, 37), 0, (9, 4)),
               ((64, 2), 0, (9, 4))]
    if prec != "f64":   # the bidirectional kernel takes W = 64 in FP64
        scheds += [((128, 8), 0, (9, 4)), ((128, 5), 7, (9, 4))]
    outs = []
    for tile, chunk, kern in scheds:
        with Lattice(run, precision=prec, tile=tile, graph_chunk=chunk, rho_ref=(1.0, 1.0), kernel=kern) as lat:
            if kern is not None:
                assert lat.schedule == (tile[0], tile[1], kern[0], kern[1])
            lat.step(23)
            outs.append(lat.populations())
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint8), outs[0].view(np.uint8))


@pytest.mark.parametrize("name", ["capillary64x18", "odd17x9", "tiny5x4", "wide300x5", "box16x8"])
@pytest.mark.parametrize("tile", [(64, 3), (128, 16), (256, 40)])
@pytest.mark.parametrize("kernel", [2, 3, 4, 5, 6, 7, 8, 9])
def test_tma_pipelined_split_kernels_fp64_match_oracle(name, tile, kernel):
    geom, prm, kind = CASES[name]
    nA, nB = _fields(geom, kind)
    if kernel == 8:   # the tile kernel's shapes: W x (R + 2) threads
        tile = {(64, 3): (32, 6), (128, 16): (32, 14), (256, 40): (64, 14)}[tile]
    wmax = {3: 64, 6: 128, 7: 64, 9: 64}.get(kernel, 256)   # FP64 static shared memory bounds W
    if tile[0] > wmax:
        from paper_0807_0602_gb300 import _lib as L
        with pytest.raises(L.LbmError) as e:
            Lattice(dict(geom=geom, params=prm, init=("fields", nA, nB)), precision="f64", tile=tile,
                    kernel=(kernel, 4))
        assert e.value.code == L.LBM_EINVAL
        tile = (wmax, tile[1])
    ref = oracle.OracleLattice(geom, prm, nA, nB)
    ref.step(30)
    with Lattice(dict(geom=geom, params=prm, init=("fields", nA, nB)), precision="f64", tile=tile,
                 kernel=(kernel, 4)) as lat:
        lat.step(30)
        F = lat.populations()
    assert np.array_equal(F, ref.populations())


@pytest.mark.parametrize("kernel", [2, 7, 8])
def test_ghost_column_kernels_rejected_below_four_columns(kernel):
    from paper_0807_0602_gb300 import _lib as L
    geom, prm, kind = CASES["row3x1"]
    nA, nB = _fields(geom, kind)
    with Lattice(dict(geom=geom, params=prm, init=("fields", nA, nB)), precision="f32") as lat:
        with pytest.raises(L.LbmError) as e:
            lat.schedule = (32, 14, kernel, 4) if kernel == 8 else (64, 16, kernel, 4)
        assert e.value.code == L.LBM_EINVAL


@pytest.mark.parametrize("depth", [6, 8])
@pytest.mark.parametrize("name", ["capillary64x18", "odd17x9"])
def test_tma_ring_depths_fp64_match_oracle(name, depth):
    geom, prm, kind = CASES[name]
    nA, nB = _fields(geom, kind)
    ref = oracle.OracleLattice(geom, prm, nA, nB)
    ref.step(30)
    with Lattice(dict(geom=geom, params=prm, init=("fields", nA, nB)), precision="f64", tile=(64, 7),
                 kernel=(2, depth)) as lat:
        lat.step(30)
        F = lat.populations()
    assert np.array_equal(F, ref.populations())


def test_async_kernel_fp64_matches_oracle():
    geom, prm, kind = CASES["capillary64x18"]
    nA, nB = _fields(geom, kind)
    ref = oracle.OracleLattice(geom, prm, nA, nB)
    ref.step(50)
    with Lattice(dict(geom=geom, params=prm, init=("fields", nA, nB)), precision="f64", tile=(64, 5),
                 kernel=(1, 4)) as lat:
        lat.step(50)
        F = lat.populations()
    assert np.array_equal(F, ref.populations())


@pytest.mark.parametrize("sched", [((64, 8), None), ((128, 4), (6, 4)), ((64, 7), (2, 4)), ((64, 6), (7, 4)),
                                   ((32, 6), (8, 4)), ((64, 8), (9, 4)), ((128, 5), (3, 4)), ((64, 16), (4, 4)),
                                   ((128, 16), (5, 4)), ((64, 3), (1, 4))])
def test_batched_runs_equal_solo_runs(sched):
    runs = []
    for j, (L, H) in enumerate(((40, 6), (100, 13), (65, 30), (7, 3))):
        r = W.capillary_run(L, H, 1.0 + 0.05 * j, 1.0, 0.8 + 0.1 * j, -0.1 * j)
        runs.append(r)
    tile, kern = sched
    kw = dict(tile=tile) if kern is None else dict(tile=tile, kernel=kern)
    with Lattice(runs, precision="f32", **kw) as bat:
        bat.step(40)
        batched = [bat.populations(r) for r in range(len(runs))]
        zs = [bat.interface(r) for r in range(len(runs))]
        ms = [bat.mass(r) for r in range(len(runs))]
    for r, run in enumerate(runs):
        with Lattice(run, precision="f32", tile=(128, 16)) as solo:
            solo.step(40)
            assert np.array_equal(solo.populations(), batched[r])
            assert np.array_equal(solo.interface(), zs[r])
            assert np.array_equal(solo.mass(), ms[r])


def test_autotune_keeps_results():
    geom = W.capillary_geometry(512, 34, 128, 512, 0, 33)
    run = dict(geom=geom, params=W.params(1.2, 1.0, 1.0, -0.1), init=("slab", 0, 200))
    with Lattice(run, precision="f32", autotune=True) as a, Lattice(run, precision="f32") as b:
        a.step(120)               # too few steps to time every candidate: no tuning yet
        b.step(120)
        assert a.schedule == b.schedule
        a.step(1500)              # both passes of the tuner run on these real steps
        b.step(1500)
        assert a.t == b.t == 1620
        assert np.array_equal(a.populations(), b.populations())
        fin = a.tuning()          # the finalists, each a valid schedule with its time
        assert 2 <= len(fin) <= 4 and b.tuning() == []
        assert a.schedule in [f[0] for f in fin]
        assert all(np.isfinite(ms) and ms > 0 for _, ms in fin)
        for sched, _ in fin:      # re-selecting a finalist keeps the bits
            a.schedule = sched
            b.schedule = sched
            a.step(3)
            b.step(3)
            assert np.array_equal(a.populations(), b.populations())


def test_checkpoint_resume_is_bit_identical(tmp_path):
    geom = W.capillary_geometry(96, 20, 24, 72, 0, 19)
    run = dict(geom=geom, params=W.params(1.2, 1.0, 0.9, -0.1), init=("slab", 0, 40))
    path = os.path.join(tmp_path, "ck.bin")
    with Lattice(run, precision="f32", log_every=10, log_capacity=32) as a:
        a.step(50)
        a.save(path)
        a.step(50)
        want, want_log, want_u = a.populations(), a.log(), a.velocity()
    from paper_0807_0602_gb300.lbm import Lattice as _L
    b = _L.load(path)
    assert b.t == 50
    b.step(50)
    assert np.array_equal(b.populations(), want)
    assert np.array_equal(b.log(), want_log)
    assert np.array_equal(b.velocity()[0], want_u[0])
    b.close()


def test_fp32_close_to_oracle_after_100_steps():
    # Reading of "relative error on densities": the error is taken relative to
    # the density scale, max |n_gpu - n_ref| / max |n_ref| per species.  The
    # pointwise ratio at minor-phase nodes (n ~ 0.008 against 2.0) is
    # ill-conditioned in FP32 (rounding of the major species enters the minor
    # one through the cross force); it is recorded, with a looser bound.
    geom, prm, _ = CASES["capillary64x18"]
    nA, nB = W.slab_fields(geom, 0, 21)
    ref = oracle.OracleLattice(geom, prm, nA, nB)
    ref.step(100)
    with Lattice(dict(geom=geom, params=prm, init=("fields", nA, nB)), precision="f32") as lat:
        lat.step(100)
        gA, gB = lat.densities()
        z = lat.interface()
    fluid = ref.solid() == 0
    rA, rB = ref.densities()
    for g, r in ((gA, rA), (gB, rB)):
        assert np.max(np.abs(g - r)[fluid]) / np.max(np.abs(r)) <= 1e-5
        assert rel_err(g, r, fluid) <= 1e-3
    assert np.max(np.abs(z - ref.interface())) <= 0.05


def test_fp16s_storage_error_is_bounded():
    geom, prm, _ = CASES["capillary64x18"]
    nA, nB = W.slab_fields(geom, 0, 21)
    ref = oracle.OracleLattice(geom, prm, nA, nB)
    ref.step(100)
    fluid = ref.solid() == 0
    rA, rB = ref.densities()
    for rho_ref in ((0.0, 0.0), (1.0, 1.0)):
        with Lattice(dict(geom=geom, params=prm, init=("fields", nA, nB)), precision="f16s", rho_ref=rho_ref) as lat:
            lat.step(100)
            gA, gB = lat.densities()
            M = lat.mass()
        assert np.max(np.abs(gA - rA)[fluid]) < 2e-2 and np.max(np.abs(gB - rB)[fluid]) < 2e-2
        assert np.all(np.abs(M - ref.mass()) < 1e-2 * ref.mass())


def test_nonfinite_state_is_reported():
    from paper_0807_0602_gb300 import _lib as L
    geom = W.periodic_box(20, 6)
    nA, nB = W.random_fields(geom, 1, 0.2, 1.0)
    nA[3, 7] = np.nan
    with Lattice(dict(geom=geom, params=W.params(1.0, 1.0, 1.0), init=("fields", nA, nB)), precision="f32") as lat:
        lat.step(2)
        with pytest.raises(L.LbmError) as e:
            lat.mass()
        assert e.value.code == L.LBM_ENONFINITE
        assert lat.status() == L.LBM_ENONFINITE


def test_full_size_capillary_8192x160_first_steps_match_oracle():
    c = W.config_capillary_8192x160(tau_B=1.0)
    nA, nB = W.initial_fields(c)
    ref = oracle.OracleLattice(c["geom"], c["params"], nA, nB)
    ref.step(3)
    fluid = ref.solid() == 0
    rA, rB = ref.densities()
    with Lattice(dict(geom=c["geom"], params=c["params"], init=c["init"]), precision="f64") as lat:
        lat.step(3)
        gA, gB = lat.densities()
    assert rel_err(gA, rA, fluid) <= 1e-12 and rel_err(gB, rB, fluid) <= 1e-12
    for kern in (None, (1, 4), (2, 4), (4, 4)):
        with Lattice(dict(geom=c["geom"], params=c["params"], init=c["init"]), precision="f32", tile=(128, 16),
                     kernel=kern) as lat:
            lat.step(3)
            gA, gB = lat.densities()
        for g, r in ((gA, rA), (gB, rB)):
            assert np.max(np.abs(g - r)[fluid]) / np.max(np.abs(r)) <= 1e-5


def test_schedule_validation_rejects_unsupported_combinations():
    from paper_0807_0602_gb300 import _lib as L
    geom, prm, kind = CASES["capillary64x18"]
    nA, nB = _fields(geom, kind)
    with Lattice(dict(geom=geom, params=prm, init=("fields", nA, nB)), precision="f64") as lat:
        before = lat.schedule
        for bad in ((128, 4, 6, 3), (128, 4, 2, 5), (128, 4, 1, 6), (96, 4, 0, 4), (32, 4, 0, 4), (64, 7, 8, 4),
                    (256, 4, 6, 4), (128, 4, 7, 4), (128, 4, 9, 4), (64, 4, 9, 5), (128, 4, 10, 4)):
            with pytest.raises(L.LbmError) as e:
                lat.schedule = bad
            assert e.value.code == L.LBM_EINVAL
            assert lat.schedule == before


def _mask_case():
    """A 40x24 periodic box with an explicit solid mask: blocks touching the
    wrap columns 0 and nx - 1 and the wrap rows, a one-node obstacle, a thin
    wall with a gap, and a fluid pocket enclosed on three sides."""
    nx, ny = 40, 24
    m = np.zeros((ny, nx), np.uint8)
    m[0, :] = 1                       # bottom plate across the wrap
    m[5:9, 0:3] = 1                   # block on the west edge
    m[5:9, 37:40] = 1                 # its periodic neighbour on the east edge
    m[12, 20] = 1                     # isolated solid node
    m[15:23, 10] = 1                  # thin wall ...
    m[18, 10] = 0                     # ... with a gap
    m[14:20, 26] = 1                  # pocket: three sides
    m[14, 26:31] = 1
    m[19, 26:31] = 1
    m[23, 33:40] = 1                  # top row next to the bottom plate (wraps)
    geom = dict(nx=nx, ny=ny, cap_x0=0, cap_x1=0, y_bot=-1, y_top=-1, mask=m)
    nA, nB = W.random_fields(geom, 7, 0.2, 1.2)
    return geom, W.params(1.1, 1.0, 0.8, -0.2, 0.1), nA, nB


MASK_SCHEDULES = [(None, None), ((128, 16), (0, 4)), ((64, 3), (1, 4)), ((64, 7), (2, 4)), ((64, 5), (3, 4)),
                  ((128, 16), (4, 4)), ((128, 9), (5, 4)), ((64, 4), (6, 4)), ((64, 6), (7, 4)), ((32, 6), (8, 4)),
                  ((64, 8), (9, 4))]


def test_solid_mask_every_kernel_matches_oracle_fp64():
    geom, prm, nA, nB = _mask_case()
    ref = oracle.OracleLattice(geom, prm, nA, nB)
    ref.step(30)
    want = ref.populations()
    for tile, kern in MASK_SCHEDULES:
        kw = {} if kern is None else dict(tile=tile, kernel=kern)
        with Lattice(dict(geom=geom, params=prm, init=("fields", nA, nB)), precision="f64", **kw) as lat:
            lat.step(30)
            got = lat.populations()
            M = lat.mass()
        assert np.array_equal(got, want), (tile, kern)
        assert np.all(np.abs(M - ref.mass()) <= 1e-12 * ref.mass())


@pytest.mark.parametrize("prec", ["f32", "f16s"])
def test_solid_mask_schedules_bit_identical(prec):
    geom, prm, nA, nB = _mask_case()
    outs = []
    for tile, kern in MASK_SCHEDULES:
        if prec == "f16s" and kern is not None and kern[0] == 1:
            continue   # the cp.async kernel moves 4- or 8-byte elements only
        kw = {} if kern is None else dict(tile=tile, kernel=kern)
        with Lattice(dict(geom=geom, params=prm, init=("fields", nA, nB)), precision=prec, rho_ref=(1.0, 1.0),
                     **kw) as lat:
            lat.step(25)
            outs.append(lat.populations())
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint8), outs[0].view(np.uint8))


def test_fp64_mini_capillary_1e4_steps_matches_oracle():
    """FP64 GPU against the oracle after 10^4 steps on the 64x18 mini
    capillary (stable parameters): bit-equal populations, equal fronts."""
    geom = W.capillary_geometry(64, 18, 16, 48, 0, 17)
    prm = W.params(1.0, 1.0, 1.0, -0.2, 0.0)
    nA, nB = W.slab_fields(geom, 0, 24)
    ref = oracle.OracleLattice(geom, prm, nA, nB)
    ref.step(10000)
    with Lattice(dict(geom=geom, params=prm, init=("fields", nA, nB)), precision="f64") as lat:
        lat.step(10000)
        F = lat.populations()
        z = lat.interface()
    assert np.all(np.isfinite(F))
    assert np.array_equal(F, ref.populations())
    assert np.max(np.abs(np.asarray(z) - np.asarray(ref.interface()))) <= 1e-10


@pytest.mark.parametrize("prec", ["f32", "f16s"])
def test_repeated_runs_are_bit_identical(prec):
    """Two handles on the same input give the same bits (fixed reduction
    orders, order-free integer minima, no atomics on floating-point data);
    with the log on, so that the mass sums and front scans run too."""
    c = W.config_capillary_8192x160(tau_B=1.0)
    run = dict(geom=c["geom"], params=dict(c["params"], G=1.0, G_Aw=-0.3), init=c["init"])
    outs = []
    for _ in range(2):
        with Lattice(run, precision=prec, rho_ref=(0.04, 2.0), log_every=50, log_capacity=16) as lat:
            lat.step(300)
            outs.append((lat.populations(), lat.log(), lat.mass()))
    assert np.array_equal(outs[0][0].view(np.uint8), outs[1][0].view(np.uint8))
    assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][2], outs[1][2])
