"""Failure detection on the GPU, in forms that fault nothing: an overlapping
configuration set from the host (non-finite forces -> MS2_EUNSTABLE), a grid
barrier made to wait for an arrival that never comes (its bounded wait runs
out -> MS2_ETIMEOUT), and a failing job in the server beside healthy ones."""
import os

import numpy as np
import pytest

from paper_1507_07548_gb300 import workloads as W

ms2 = pytest.importorskip("paper_1507_07548_gb300.ms2")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def water216():
    wl = W.water_box(N=216, rc=9.0, seed=9)
    z = np.load(os.path.join(GOLDEN, "water_N216.npz"))
    wl.R, wl.q, wl.v, wl.Lang = z["R"], z["q"], z["v"], z["Lang"]
    return wl


def test_overlapping_configuration_is_reported_unstable():
    wl = water216()
    s = ms2.System.from_workload(wl)
    ref = s.energy_virial()
    R = wl.R.copy()
    R[1] = R[0]                      # two molecules on one centre, same orientation
    q = wl.q.copy()
    q[1] = q[0]
    s.set_state(R, q, wl.v, wl.Lang)
    with pytest.raises(ms2.Ms2Error, match="EUNSTABLE"):
        s.energy_virial()
    s.set_state(wl.R, wl.q, wl.v, wl.Lang)   # a valid state makes the system usable again
    assert s.energy_virial() == ref


def test_barrier_wait_runs_out_and_is_reported():
    wl = water216()
    s = ms2.System.from_workload(wl)
    if s.fused_step() != 1:
        pytest.skip("no fused step kernel on this device")
    s.fault_inject_barrier(50e-6)
    s.step(3)
    with pytest.raises(ms2.Ms2Error, match="ETIMEOUT"):
        s.energy_virial()
    # the flag is cleared; a state set again steps exactly as a fresh system does
    s.set_state(wl.R, wl.q, wl.v, wl.Lang)
    s.step(5)
    f = ms2.System.from_workload(wl)
    f.step(5)
    for x, y in zip(s.get_state()[:4], f.get_state()[:4]):
        assert np.array_equal(x, y)
    assert s.energy_virial() == f.energy_virial()


def serve(jobs, failing=None, steps=200):
    """Jobs all eligible at once (arrival 0.3 s, after every submit), so the
    admission order and each job's path are fixed; `failing` is submitted last."""
    s = ms2.Server(1 << 30, 64)
    ids = [s.submit(m, c, T, rho, rc, e, steps, arrival=0.3, seed=300 + k, rdf_bins=40)
           for k, (m, c, T, rho, rc, e) in enumerate(jobs)]
    bad = None
    if failing is not None:
        m, c, T, rho, rc, e, R0, q0 = failing
        bad = s.submit(m, c, T, rho, rc, e, steps, arrival=0.3, seed=999, rdf_bins=40, R0=R0, q0=q0)
    s.drain(300.0)
    res = {r["job_id"]: r for r in s.poll(256)}
    s.close()
    return [res[i] for i in ids], (res[bad] if bad is not None else None)


def test_a_failing_job_leaves_the_others_untouched():
    rho = W.WATER_NUMBER_DENSITY
    jobs = [([W.water()], [216], 298.0, rho, 9.0, ms2.ELEC_RF),
            ([W.stockmayer()], [300], 300.0, 0.012, 12.0, ms2.ELEC_RF)] * 4   # 8 resident: the batch runs
    wl = W.water_box(N=216, rc=9.0, seed=9)
    R0, q0 = wl.R.copy(), wl.q.copy()
    R0[1], q0[1] = R0[0], q0[0]          # an overlapping start
    ref, _ = serve(jobs)
    got, bad = serve(jobs, failing=([W.water()], [216], 298.0, rho, 9.0, ms2.ELEC_RF, R0, q0))
    assert ms2.STATUS[bad["status"]] == "MS2_EUNSTABLE"
    for a, b in zip(got, ref):
        assert a["status"] == b["status"] == 0
        assert a["U"] == b["U"] and a["P"] == b["P"] and a["T"] == b["T"]
        assert np.array_equal(a["g"], b["g"])
