"""Green-Kubo electric conductivity (paper Sec. 4, Eqs. 3-4) on the GPU.

The sampled current flux is held to the oracle's sum over the ions of the same
state; the device's autocorrelation and conductivity are held to the oracle's
brute-force autocorrelation and trapezoidal integral of the GPU's own samples.
"""
import os

import numpy as np
import pytest

from oracle import Oracle
from paper_1507_07548_gb300 import workloads as W

ms2 = pytest.importorskip("paper_1507_07548_gb300.ms2")
pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def ionic():
    wl = W.ionic_solution(seed=3)
    z = np.load(os.path.join(GOLDEN, "ionic_N1040.npz"))
    wl.R, wl.q, wl.v, wl.Lang = z["R"], z["q"], z["v"], z["Lang"]
    return wl


def test_current_matches_oracle():
    wl = ionic()
    s = ms2.System.from_workload(wl)
    s.conductivity_setup(every=1, n_lags=8)
    s.step(1)
    R, q, v, L, _ = s.get_state()
    j = s.current()
    jo = Oracle.from_workload(wl).current(v)
    np.testing.assert_allclose(j, jo, rtol=1e-12, atol=1e-14 * np.abs(jo).max())
    assert np.abs(jo).max() > 0


def test_autocorrelation_and_conductivity_of_the_gpu_samples():
    wl = ionic()
    s = ms2.System.from_workload(wl)
    every, lags, n = 2, 16, 40
    s.conductivity_setup(every=every, n_lags=lags)
    samples = []
    for _ in range(n):
        s.step(every)
        samples.append(s.current())
    sigma, acf, ns = s.conductivity()
    assert ns == n
    want = Oracle.flux_acf(np.array(samples), lags)
    np.testing.assert_allclose(acf, want, rtol=1e-10, atol=1e-13 * abs(want[0]))
    sig_o = Oracle.conductivity(want, every * wl.dt, wl.L ** 3, wl.T)
    assert sigma == pytest.approx(sig_o, rel=1e-9)
    assert np.isfinite(sigma)


def test_fused_sampling_equals_per_phase_and_neutral_water_carries_no_current():
    z = np.load(os.path.join(GOLDEN, "water_N1000.npz"))
    wl = W.water_box(N=1000, rc=14.0, seed=2)
    wl.R, wl.q, wl.v, wl.Lang = z["R"], z["q"], z["v"], z["Lang"]
    a = ms2.System.from_workload(wl)
    b = ms2.System.from_workload(wl, fused_step=0)
    for s in (a, b):
        s.conductivity_setup(every=3, n_lags=10)
        s.step(60)
    assert a.fused_step() == 1
    ra, rb = a.conductivity(), b.conductivity()
    assert ra[2] == rb[2] == 20
    assert ra[0] == rb[0] == 0.0 and not ra[1].any()
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_sampling_systems_are_not_batched_and_setup_checks_arguments():
    wl = ionic()
    s = ms2.System.from_workload(wl)
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        s.conductivity_setup(every=0, n_lags=8)
    with pytest.raises(ms2.Ms2Error, match="ESTATE"):
        s.current()
    w = ms2.System.from_workload(W.water_box(N=216, rc=9.0, seed=9))
    w.conductivity_setup(every=5, n_lags=8)
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        ms2.Batch([w])
