"""Host-side input generators: seeded, shaped as stated, zero on solids."""
import numpy as np

import workloads as W


def test_random_fields_are_seeded_and_zero_on_solids():
    geom = W.capillary_geometry(40, 12, 8, 32, 0, 11)
    a = W.random_fields(geom, 5, 0.2, 1.2)
    b = W.random_fields(geom, 5, 0.2, 1.2)
    c = W.random_fields(geom, 6, 0.2, 1.2)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[0], c[0])
    s = W.solid_mask(geom).astype(bool)
    assert s.sum() == 2 * 24
    for f in a:
        assert np.all(f[s] == 0.0) and np.all((f[~s] >= 0.2) & (f[~s] < 1.2))


def test_fp16_shift_is_the_majority_phase_density():
    c = W.config_capillary_8192x160(tau_B=1.0)
    run = dict(geom=c["geom"], params=c["params"], init=c["init"])
    assert W.fp16_shift(run) == (W.RHO_MINOR, W.RHO_MAJOR)          # gas fills most of the grid
    box = W.periodic_box(64, 64)
    drop = dict(geom=box, params=W.params(1.4, 1.0, 1.0), init=("droplet", 32.0, 32.0, 40.0))
    assert W.fp16_shift(drop) == (W.RHO_MAJOR, W.RHO_MINOR)         # a droplet larger than half the box


def test_uneven_batch_matches_its_stated_ranges():
    runs = W.batch_uneven_capillaries(64, seed=3)
    for r in runs:
        g, p = r["geom"], r["params"]
        H = g["y_top"] - g["y_bot"] - 1
        L = g["cap_x1"] - g["cap_x0"]
        assert 16 <= H <= 128 and 256 <= L <= 4096 and g["nx"] == 2 * L and g["ny"] == H + 2
        assert 1.2 <= p["G"] <= 1.6 and 0.55 <= p["tau_B"] <= 1.5 and p["tau_A"] == 1.0
    again = W.batch_uneven_capillaries(64, seed=3)
    assert [r["params"] for r in runs] == [r["params"] for r in again]
