"""The checked build (-DLBM_CHECKED) on valid inputs: every step kernel and
the mass sums validate their tiles and rows first, find nothing outside the
run's buffers, and give the same bits as the default build (the kernel
compiled at run time for the grid is compiled with the same checks).

The checked library is loaded in a child process (LBM_CHECKED=1), so this
process keeps the default build.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np
import oracle
import workloads as W
from paper_0807_0602_gb300 import _lib as L
from paper_0807_0602_gb300.lbm import Lattice

assert L.load()._name.endswith("_checked.so"), L.load()._name
SCHEDULES = [(None, None), ((128, 16), (0, 4)), ((64, 3), (1, 4)), ((64, 7), (2, 4)), ((64, 5), (3, 4)),
             ((128, 16), (4, 4)), ((128, 9), (5, 4)), ((64, 4), (6, 4)), ((64, 6), (7, 4)), ((32, 6), (8, 4)),
             ((64, 8), (9, 4)), ((64, 5), (11, 4))]
cases = [(W.capillary_geometry(17, 9, 3, 14, 1, 7), W.params(1.1, 1.2, 0.8, 0.1, -0.1)),
         (W.capillary_geometry(300, 5, 0, 300, 0, 4), W.params(1.0, 1.0, 1.0, -0.1, 0.1)),
         (W.periodic_box(5, 4), dict(W.params(0.9, 1.0, 1.0), alpha=(4 / 9, 0.8), mass=(1.0, 2.0)))]
for geom, prm in cases:
    nA, nB = W.random_fields(geom, 3, 0.2, 1.2)
    ref = oracle.OracleLattice(geom, prm, nA, nB)
    ref.step(12)
    for tile, kern in SCHEDULES:
        kw = {} if kern is None else dict(tile=tile, kernel=kern)
        with Lattice(dict(geom=geom, params=prm, init=("fields", nA, nB)), precision="f64", **kw) as lat:
            lat.step(12)
            lat.sync()                    # raises LBM_EBOUNDS if a check fired
            M = lat.mass()
            assert np.array_equal(lat.populations(), ref.populations()), (geom, kern)
            assert np.all(np.abs(M - ref.mass()) <= 1e-12 * ref.mass())
# the ring kernel (FP32 and FP16S storage only): its segments pass the same
# checks, and it gives the default kernel's bits
for geom, prm in cases:
    nA, nB = W.random_fields(geom, 3, 0.2, 1.2)
    run = dict(geom=geom, params=prm, init=("fields", nA, nB))
    for prec in ("f32", "f16s"):
        outs = []
        for kw in (dict(), dict(tile=(128, 4), kernel=(10, 3))):
            with Lattice(run, precision=prec, rho_ref=(1.0, 1.0), **kw) as lat:
                lat.step(12)
                lat.sync()
                outs.append(lat.populations())
        assert np.array_equal(outs[0].view(np.uint8), outs[1].view(np.uint8)), (geom, prec)
print("checked build ok")
'''


def test_checked_build_finds_no_bounds_violation_and_matches_oracle():
    from paper_0807_0602_gb300 import build as B
    import oracle
    B.build(checked=True)
    oracle.build()
    env = dict(os.environ, LBM_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "checked build ok" in r.stdout
