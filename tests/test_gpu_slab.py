"""x-slab decomposition on the GPU library (lbm_get_columns /
lbm_set_columns): slabs of one capillary, each a lattice with two halo
columns per side, exchanging edge columns after every step, reproduce the
undivided run bit for bit (FP64: also the oracle's bits), for every kernel
that reads the halo columns through the ghost images.

All slabs live in one process on one GPU and are stepped one after another;
no kernel waits on another (the multi-rank exchange over torch.distributed
is tested on CPU ranks in tests/test_dist_slab.py)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _case():
    geom = W.capillary_geometry(300, 41, 60, 280, 0, 40)
    nA, nB = W.random_fields(geom, 9, 0.2, 1.2)
    return dict(geom=geom, params=W.params(1.2, 1.0, 0.9, -0.1, 0.05), init=("fields", nA, nB)), nA, nB


def _slabs(run, nA, nB, parts, **kw):
    from paper_0807_0602_gb300 import slab as SL
    return [SL.Slab(run, a, b, nA, nB, **kw) for a, b in SL.slab_bounds(run["geom"]["nx"], parts)]


@pytest.mark.parametrize("parts", [2, 3])
def test_fp64_slabs_equal_the_oracle(parts):
    from paper_0807_0602_gb300 import slab as SL
    run, nA, nB = _case()
    slabs = _slabs(run, nA, nB, parts, precision="f64")
    SL.step_local(slabs, 25)
    got = np.concatenate([s.owned(s.lat.populations()) for s in slabs], axis=-1)
    o = oracle.OracleLattice(run["geom"], run["params"], nA, nB)
    o.step(25)
    assert np.array_equal(got, o.populations())


@pytest.mark.parametrize("prec,kernel", [("f32", None), ("f32", (10, 4)), ("f32", (2, 4)), ("f16s", None),
                                         ("f16s", (10, 3))])
def test_slabs_equal_the_undivided_gpu_run(prec, kernel):
    from paper_0807_0602_gb300 import slab as SL
    from paper_0807_0602_gb300.lbm import Lattice
    run, nA, nB = _case()
    kw = dict(precision=prec, rho_ref=(1.0, 1.0))
    if kernel is not None:
        kw.update(tile=(128, 4) if kernel[0] == 10 else (64, 7), kernel=kernel)
    slabs = _slabs(run, nA, nB, 3, **kw)
    SL.step_local(slabs, 40)
    got = np.concatenate([s.owned(s.lat.populations()) for s in slabs], axis=-1)
    with Lattice(run, precision=prec, rho_ref=(1.0, 1.0)) as whole:
        whole.step(40)
        want = whole.populations()
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8))


def test_workload_8192x160_in_two_slabs():
    from paper_0807_0602_gb300 import slab as SL
    from paper_0807_0602_gb300.lbm import Lattice
    c = W.config_capillary_8192x160(tau_B=1.0)
    run = dict(geom=c["geom"], params=c["params"], init=c["init"])
    nA, nB = W.initial_fields(c)
    slabs = _slabs(run, nA, nB, 2, precision="f32")
    SL.step_local(slabs, 30)
    got = np.concatenate([s.owned(s.lat.populations()) for s in slabs], axis=-1)
    with Lattice(run, precision="f32") as whole:
        whole.step(30)
        want = whole.populations()
    assert np.array_equal(got, want)


def test_column_window_arguments_are_checked():
    from paper_0807_0602_gb300 import _lib as L
    from paper_0807_0602_gb300.lbm import Lattice
    run, _, _ = _case()
    with Lattice(run, precision="f32") as lat:
        buf = lat.get_columns(298, 2)
        for x0, n in ((299, 2), (-1, 2), (0, 0)):
            with pytest.raises(L.LbmError):
                lat.get_columns(x0, n)
        lat.set_columns(298, buf)   # a round trip leaves the state unchanged
        assert np.array_equal(lat.get_columns(298, 2).cpu().numpy(), buf.cpu().numpy())
