"""The C-ABI library builds, loads and exports every symbol include/*.h declares.

No compute call runs here: argument validation happens before the library
touches a GPU, so rejected arguments can be checked on a machine without one.
"""
import ctypes
import glob
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    pat = re.compile(r"^\s*(?!typedef)(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*([a-z][a-z0-9_]*)\s*\(")
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        with open(hdr) as fh:
            for line in fh:
                m = pat.match(line)
                if m:
                    names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_0807_0602_gb300 import build as B
    from paper_0807_0602_gb300 import _lib
    B.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_create", "lbm_step", "lbm_densities", "lbm_interface_positions", "lbm_create_batch",
                     "lbm_mass", "lbm_get_log", "lbm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    from paper_0807_0602_gb300 import _lib, surrogate
    names = declared_functions()
    assert set(n for n in names if n.startswith("lbm_")) <= set(_lib.SIGNATURES)
    assert set(n for n in names if n.startswith("mlp_")) <= set(surrogate.MLP_SIGNATURES)
    assert set(names) <= set(_lib.SIGNATURES) | set(surrogate.MLP_SIGNATURES)


def _geom(nx=16, ny=8):
    from paper_0807_0602_gb300 import _lib as L
    g = L.Geometry()
    g.nx, g.ny = nx, ny
    g.cap_x0, g.cap_x1, g.y_bot, g.y_top = 4, 12, 0, 7
    g.init_kind = L.LBM_INIT_SLAB
    g.x_lo, g.x_hi = 0.0, 6.0
    g.rho_major, g.rho_minor = 2.0, 0.04
    return g


def _create(lib, g, G=1.0, wall=(0.0, 0.0), tA=1.0, tB=1.0, opt=None):
    h = ctypes.c_void_p()
    w = (ctypes.c_double * 2)(*wall)
    rc = lib.lbm_create(ctypes.byref(g), G, w, tA, tB, ctypes.byref(opt) if opt is not None else None,
                        ctypes.byref(h))
    return rc, h


def test_invalid_arguments_are_rejected_without_touching_the_gpu(lib):
    from paper_0807_0602_gb300 import _lib as L
    assert _create(lib, _geom(), tA=0.5)[0] == L.LBM_EINVAL          # tau must exceed 1/2
    assert _create(lib, _geom(), tB=0.3)[0] == L.LBM_EINVAL
    assert _create(lib, _geom(), G=math.nan)[0] == L.LBM_EINVAL
    assert _create(lib, _geom(), wall=(math.inf, 0.0))[0] == L.LBM_EINVAL
    assert _create(lib, _geom(nx=0))[0] == L.LBM_EINVAL
    g = _geom()
    g.cap_x1 = 17                                                    # plates past the grid
    assert _create(lib, g)[0] == L.LBM_EINVAL
    g = _geom()
    g.y_top = 8
    assert _create(lib, g)[0] == L.LBM_EINVAL
    g = _geom()
    g.init_kind = L.LBM_INIT_FIELDS                                  # fields missing
    assert _create(lib, g)[0] == L.LBM_EINVAL
    opt = L.Options()
    lib.lbm_default_options(ctypes.byref(opt))
    opt.precision = 7
    assert _create(lib, _geom(), opt=opt)[0] == L.LBM_EINVAL
    opt.precision = L.LBM_F32
    opt.tile_w = 100
    assert _create(lib, _geom(), opt=opt)[0] == L.LBM_EINVAL
    opt.tile_w = 128
    opt.log_every, opt.log_capacity = 10, 0
    assert _create(lib, _geom(), opt=opt)[0] == L.LBM_EINVAL
    opt.log_every = 0
    for alpha in (1.0, -0.1, math.nan):                              # Eqs. 3-5: 0 <= alpha < 1
        opt.alpha[1] = alpha
        assert _create(lib, _geom(), opt=opt)[0] == L.LBM_EINVAL
    opt.alpha[1] = 4.0 / 9.0
    for m in (0.0, -1.0, math.inf):                                  # rho_k = m_k n_k, m_k > 0
        opt.molecular_mass[0] = m
        assert _create(lib, _geom(), opt=opt)[0] == L.LBM_EINVAL


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_has_gpu(), reason="on a GPU machine the gpu tests check this with real buffers")
def test_mass_noalloc_rejects_sizes_beyond_its_limits_without_a_gpu(lib):
    """Host-side checks of the allocation-free mass sums: more rows than its
    static array holds, and buffers past 32-bit element offsets
    (18 ny pitch >= 2^31), are rejected before any CUDA call.  Run only where
    no GPU exists, so the placeholder pointer can never reach a kernel."""
    from paper_0807_0602_gb300 import _lib as L
    placeholder = ctypes.c_void_p(256)
    g = _geom(nx=4, ny=65537)
    g.cap_x0, g.cap_x1, g.y_bot, g.y_top = 0, 4, 0, 10
    assert lib.lbm_mass_noalloc(ctypes.byref(g), L.LBM_F32, placeholder, 64, None, placeholder, None) == L.LBM_EINVAL
    g = _geom(nx=3856, ny=65536)
    g.cap_x0, g.cap_x1, g.y_bot, g.y_top = 0, 4, 0, 10
    assert lib.lbm_mass_noalloc(ctypes.byref(g), L.LBM_F32, placeholder, 3856, None, placeholder,
                                None) == L.LBM_EINVAL
    g = _geom(nx=16, ny=8)
    g.solid_mask = ctypes.cast(ctypes.create_string_buffer(128), ctypes.POINTER(ctypes.c_uint8))
    assert lib.lbm_mass_noalloc(ctypes.byref(g), L.LBM_F32, placeholder, 64, None, placeholder, None) == L.LBM_EINVAL


def test_wait_selftest_rejects_out_of_range_budgets_without_launching(lib):
    from paper_0807_0602_gb300 import _lib as L
    assert lib.lbm_selftest_wait_timeout(10, None) == L.LBM_EINVAL
    assert lib.lbm_selftest_wait_timeout(5_000_000_000, None) == L.LBM_EINVAL


def test_null_handles_and_status_strings(lib):
    from paper_0807_0602_gb300 import _lib as L
    assert lib.lbm_step(None, 1) == L.LBM_EINVAL
    assert lib.lbm_time(None) == -1
    n = ctypes.c_int(7)
    assert lib.lbm_get_tuning(None, 0, None, None, ctypes.byref(n)) == L.LBM_EINVAL
    assert lib.lbm_selftest_fp64_rate(None, None) == L.LBM_EINVAL
    lib.lbm_destroy(None)
    for code in range(9):
        assert lib.lbm_error_string(code)
    assert lib.lbm_error_string(99) == b"unknown status"


def test_default_options(lib):
    from paper_0807_0602_gb300 import _lib as L
    opt = L.Options()
    lib.lbm_default_options(ctypes.byref(opt))
    assert opt.precision == L.LBM_F32 and opt.tile_w == 128 and opt.tile_h == 4 and opt.rho_bulk == 2.0
    assert list(opt.alpha) == [4.0 / 9.0] * 2 and list(opt.molecular_mass) == [1.0, 1.0]


def test_structure_layouts_match_header():
    from paper_0807_0602_gb300 import _lib as L
    # 8 int32 + pointer + 7 doubles + 2 pointers
    assert ctypes.sizeof(L.Geometry) == 8 * 4 + 8 + 7 * 8 + 2 * 8
    # 8 int32 + 5 doubles + 4 pointers + 4 doubles
    assert ctypes.sizeof(L.Options) == 8 * 4 + 5 * 8 + 4 * 8 + 4 * 8
    assert ctypes.sizeof(L.RunInfo) == 6 * 4 + 8 + 2 * 8


def test_checked_build_compiles_and_exports_the_same_symbols(lib):
    """The -DLBM_CHECKED variant (bounds checks in every step kernel) builds
    and exports the same ABI as the default library."""
    from paper_0807_0602_gb300 import build as B
    path = B.build(checked=True)
    checked = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(checked, n)]
    assert not missing, missing
    checked.lbm_error_string.restype = ctypes.c_char_p
    assert b"checked" in checked.lbm_error_string(8)
