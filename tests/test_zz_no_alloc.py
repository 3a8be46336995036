"""The allocation-free mass entry point agrees with lbm_mass.

lbm_mass_noalloc serves callers that cannot allocate device memory where
they need the mass sums (inside an allocator callback that must not re-enter
its allocator, in a process whose device memory another pool owns).  It
keeps its partial sums in one fixed device array shared by all calls, so
this file is collected last and the test runs two calls in a row on the same
array.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _geometry(geom):
    from paper_0807_0602_gb300 import _lib as L
    g = L.Geometry()
    g.nx, g.ny = geom["nx"], geom["ny"]
    g.cap_x0, g.cap_x1, g.y_bot, g.y_top = geom["cap_x0"], geom["cap_x1"], geom["y_bot"], geom["y_top"]
    return g


def _noalloc(lib, g, prec, base, pitch, rho_ref, out):
    import torch
    from paper_0807_0602_gb300.lbm import PRECISIONS
    stream = torch.cuda.current_stream()
    return lib.lbm_mass_noalloc(ctypes.byref(g), PRECISIONS[prec], ctypes.c_void_p(base), pitch, rho_ref,
                                ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("prec", ["f64", "f32", "f16s"])
def test_mass_without_allocation_matches_lbm_mass(prec):
    import torch
    from paper_0807_0602_gb300 import _lib as L
    from paper_0807_0602_gb300.build import build
    from paper_0807_0602_gb300.lbm import Lattice

    build()
    lib = L.load()
    geom = W.capillary_geometry(300, 41, 60, 280, 0, 40)
    run = dict(geom=geom, params=W.params(1.1, 1.0, 1.0, -0.1), init=("slab", 0, 110))
    rho_ref = (ctypes.c_double * 2)(1.0, 1.0)
    g = _geometry(geom)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    with Lattice(run, precision=prec, rho_ref=(1.0, 1.0)) as lat:
        for call in range(2):
            lat.step(7 + call)
            info = lat.run_info(0)
            assert _noalloc(lib, g, prec, info.base[info.current], info.pitch, rho_ref, out) == L.LBM_OK
            got = out.cpu().numpy()
            want = lat.mass()
            assert np.all(np.isfinite(got))
            assert np.allclose(got, want, rtol=1e-12, atol=0.0)


def test_tall_narrow_grid_loops_over_rows_in_the_final_tree():
    """60000 rows (more than the 256 threads of the final tree, close to the
    array's 65536 rows): two calls in a row agree with lbm_mass."""
    import torch
    from paper_0807_0602_gb300 import _lib as L
    from paper_0807_0602_gb300.build import build
    from paper_0807_0602_gb300.lbm import Lattice

    build()
    lib = L.load()
    geom = W.periodic_box(8, 60000)
    nA, nB = W.random_fields(geom, seed=11)
    run = dict(geom=geom, params=W.params(1.0, 1.0, 1.0, 0.0), init=("fields", nA, nB))
    g = _geometry(geom)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    with Lattice(run, precision="f32") as lat:
        for call in range(2):
            lat.step(3)
            info = lat.run_info(0)
            assert _noalloc(lib, g, "f32", info.base[info.current], info.pitch, None, out) == L.LBM_OK
            assert np.allclose(out.cpu().numpy(), lat.mass(), rtol=1e-12, atol=0.0)


def test_rejects_sizes_beyond_its_limits_before_launching():
    """Real device buffers as large as the rejected geometries claim: more
    rows than the static array holds, and a buffer past 32-bit element
    offsets."""
    import torch
    from paper_0807_0602_gb300 import _lib as L
    from paper_0807_0602_gb300.build import build

    build()
    lib = L.load()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    g = _geometry(W.capillary_geometry(4, 65537, 0, 4, 0, 10))
    buf = torch.empty(18 * 65537 * 64, dtype=torch.float32, device="cuda")
    assert _noalloc(lib, g, "f32", buf.data_ptr(), 64, None, out) == L.LBM_EINVAL
    del buf
    g = _geometry(W.capillary_geometry(4000, 30000, 0, 4, 0, 10))   # 18 * 30000 * 4000 >= 2^31 elements
    buf = torch.empty(18 * 30000 * 4000, dtype=torch.float16, device="cuda")
    assert _noalloc(lib, g, "f16s", buf.data_ptr(), 4000, None, out) == L.LBM_EINVAL
    del buf
    assert np.array_equal(out.cpu().numpy(), [0.0, 0.0])
