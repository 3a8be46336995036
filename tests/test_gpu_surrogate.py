"""What the trained surrogate gains over the plain lattice search.

The network is trained on contact angles and capillary prefactors measured
by the lattice model (FP32 batches) with the project's device kernels; it
then proposes the wall coupling for target contact angles.  Every proposal is
judged by an FP64 sessile-droplet run; a miss falls back to bisection near
the proposal.  The baseline is the same FP64 bisection from the full
coupling range.  The surrogate must reach the 2 degree tolerance with fewer
lattice runs.
"""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_surrogate_needs_fewer_lattice_runs_than_bisection():
    from paper_0807_0602_gb300.build import build
    build()
    from paper_0807_0602_gb300 import calibrate as Cb
    from paper_0807_0602_gb300.surrogate import Surrogate

    X, T = Cb.build_dataset(96, seed=11, droplet_steps=6000, capillary_steps=12000, L_cap=192)
    assert len(X) >= 80
    sur = Surrogate(X, T, seed=1, max_batch=2048)
    losses = sur.fit(X, T, steps=1500, lr=3e-3, batch=96)
    assert losses[-50:].mean() < 0.1 * losses[:10].mean()
    fixed = (1.04, 1.0, 1.0, 32.0)
    targets = np.array([55.0, 65.0, 75.0, 85.0, 95.0, 105.0])
    c_s, a_s, runs_s = Cb.propose_and_verify(sur, targets, fixed, tol_deg=2.0, precision="f64", steps=6000)
    c_b, a_b, runs_b = Cb.bisection(targets, fixed, tol_deg=2.0, precision="f64", steps=6000)
    report = dict(targets=targets.tolist(), surrogate_angles=np.round(a_s, 2).tolist(),
                  surrogate_runs=runs_s.tolist(), bisection_angles=np.round(a_b, 2).tolist(),
                  bisection_runs=runs_b.tolist(),
                  first_proposal_within_2deg=float(np.mean(runs_s == 1)))
    print("surrogate gain:", json.dumps(report))
    assert np.all(np.abs(a_s - targets) <= 2.0)
    assert runs_s.sum() < runs_b.sum()
