"""Failure detection on the GPU without a fault: a bounded mbarrier wait that
can never complete runs out, the library reports LBM_ETIMEOUT, and the
context stays usable (a lattice steps correctly afterwards)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    from paper_0807_0602_gb300 import _lib as L
    from paper_0807_0602_gb300.build import build
    from paper_0807_0602_gb300.lbm import Lattice
    build()
    lib = L.load()
    assert lib.lbm_selftest_wait_timeout(2_000_000, None) == L.LBM_ETIMEOUT   # about 1 ms of SM clock
    geom = W.capillary_geometry(64, 18, 16, 48, 0, 17)
    run = dict(geom=geom, params=W.params(1.0, 1.0, 1.0, -0.2), init=("slab", 0, 24))
    with Lattice(run, precision="f64", kernel=(2, 4), tile=(64, 8)) as lat:
        lat.step(20)
        assert lat.status() == L.LBM_OK
        assert np.all(np.isfinite(lat.mass()))
