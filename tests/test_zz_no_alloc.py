"""The allocation-free mass entry point agrees with lbm_mass.

lbm_mass_noalloc serves callers that cannot allocate device memory where
they need the mass sums (during stream capture, inside an allocator
callback, in a process whose device memory another pool owns).  It keeps its
partial sums in one fixed device array shared by all calls, so this file is
collected last and the test runs two calls in a row on the same array.
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


@pytest.mark.parametrize("prec", ["f64", "f32", "f16s"])
def test_mass_without_allocation_matches_lbm_mass(prec):
    import torch
    from paper_0807_0602_gb300 import _lib as L
    from paper_0807_0602_gb300.build import build
    from paper_0807_0602_gb300.lbm import PRECISIONS, Lattice

    build()
    lib = L.load()
    geom = W.capillary_geometry(300, 41, 60, 280, 0, 40)
    run = dict(geom=geom, params=W.params(1.1, 1.0, 1.0, -0.1), init=("slab", 0, 110))
    rho_ref = (ctypes.c_double * 2)(1.0, 1.0)
    g = _geometry(geom)
    stream = torch.cuda.current_stream()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    with Lattice(run, precision=prec, rho_ref=(1.0, 1.0)) as lat:
        for call in range(2):
            lat.step(7 + call)
            info = lat.run_info(0)
            rc = lib.lbm_mass_noalloc(ctypes.byref(g), PRECISIONS[prec], ctypes.c_void_p(info.base[info.current]),
                                      info.pitch, rho_ref, ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(stream.cuda_stream))
            assert rc == L.LBM_OK
            got = out.cpu().numpy()
            want = lat.mass()
            assert np.all(np.isfinite(got))
            assert np.allclose(got, want, rtol=1e-12, atol=0.0)


def test_rejects_more_rows_than_the_static_array_holds():
    from paper_0807_0602_gb300 import _lib as L
    from paper_0807_0602_gb300.build import build

    build()
    lib = L.load()
    g = _geometry(W.capillary_geometry(4, 65537, 0, 4, 0, 10))
    dummy = ctypes.c_void_p(16)
    assert lib.lbm_mass_noalloc(ctypes.byref(g), L.LBM_F32, dummy, 64, None, dummy, None) == L.LBM_EINVAL
