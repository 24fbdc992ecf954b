"""Residence time and solvation number (paper Sec. 4, Eq. 7, Impey tolerance)
on the GPU, held to the oracle's brute-force correlation over the GPU's own
trajectory (the configurations at every sample)."""
import os

import numpy as np
import pytest

from oracle import Oracle
from paper_1507_07548_gb300 import workloads as W

ms2 = pytest.importorskip("paper_1507_07548_gb300.ms2")
pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def snap(wl, name):
    z = np.load(os.path.join(GOLDEN, name + ".npz"))
    wl.R, wl.q, wl.v, wl.Lang = z["R"], z["q"], z["v"], z["Lang"]
    return wl


@pytest.mark.parametrize("name,si,sj,r,t_star", [("ionic", 1, 0, 3.3, 2), ("water", 0, 0, 3.4, 1)])
def test_residence_matches_oracle_on_the_gpu_trajectory(name, si, sj, r, t_star):
    wl = snap(W.ionic_solution(seed=3), "ionic_N1040") if name == "ionic" else \
        snap(W.water_box(N=216, rc=9.0, seed=9), "water_N216")
    s = ms2.System.from_workload(wl)
    every, lags, n = 3, 12, 25
    s.residence_setup(si, sj, r, every, lags, t_star)
    assert s.fused_step() == 0            # residence sampling runs on the per-phase path
    traj = []
    for _ in range(n):
        s.step(every)
        traj.append(s.get_state()[0])
    corr, tau, nsol, ns = s.residence()
    assert ns == n
    co, no = Oracle.from_workload(wl).residence(np.array(traj), si, sj, r, t_star, lags)
    np.testing.assert_allclose(corr, co, rtol=1e-12, atol=1e-15)
    assert nsol == pytest.approx(no, rel=1e-14)
    assert corr[0] == 1.0 and nsol > 0
    assert tau == pytest.approx(np.trapezoid(co) * every * wl.dt, rel=1e-12)


def test_residence_setup_checks_arguments():
    s = ms2.System.from_workload(snap(W.water_box(N=216, rc=9.0, seed=9), "water_N216"))
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        s.residence_setup(0, 3, 3.4, 1, 8)
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        s.residence_setup(0, 0, 0.6 * s.L, 1, 8)
    with pytest.raises(ms2.Ms2Error, match="ESTATE"):
        s.residence()
