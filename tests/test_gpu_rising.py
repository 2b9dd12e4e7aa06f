"""Rising-bubble observables on the GPU (Section 6.1): a walled 48 x 192 x 48 box,
D = 12, Eo 10, Mo 1e-3, t_ref 600, three reference times.  The bubble rises on
the box axis, its centroid rising steadily; the indicator-weighted mean velocity
is of the centroid's rate but above it (it weights the core, whose internal
circulation outruns the bubble); the indicator volume changes little (it
measures the bubble inside the interface's mid-level, which the interface's
relaxation and deformation move slightly)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2012_06144_gb300 import lbm

    return lbm


def test_small_rising_bubble_observables(lbm):
    from paper_2012_06144_gb300 import observables as O

    D, t_ref = 12.0, 600.0
    prob, phi0 = W.rising_bubble(48, 192, 48, D=D, Eo=10.0, Mo=1e-3, t_ref=t_ref)
    sim = lbm.Simulation.from_problem(prob)
    sim.init_phase(phi0)
    rec = O.track(sim, steps=int(3 * t_ref), every=50)
    sim.synchronize()
    t, c, v, vol, umax = rec.arrays()
    s = O.summary(prob, rec, D, window=1.0)
    print(s)
    assert np.all(np.isfinite(c)) and np.all(np.isfinite(v))
    assert s["centroid_rise"] > 0.3 * D
    assert np.abs(c[:, 0] - 24.0).max() < 1e-3 and np.abs(c[:, 2] - 24.0).max() < 1e-3  # stays on the axis
    assert v[-1, 1] > 0 and s["u_t"] > 0
    late = t >= t_ref
    dv = O.centroid_velocity(rec)[late][1:-1].mean()
    assert 1.0 <= v[late, 1][1:-1].mean() / dv < 1.4
    assert s["u_t"] == pytest.approx(O.centroid_velocity(rec)[-6:-1].mean(), rel=0.1)
    assert abs(s["light_volume_drift"]) < 0.05
    assert np.all(np.diff(c[:, 1])[len(t) // 6:] > 0)  # steady rise once under way
    assert 0 < s["C_D"] < 100 and np.isfinite(s["C_D_correlation_Re_Gr"])
