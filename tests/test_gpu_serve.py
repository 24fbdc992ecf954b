"""Serving (ms2_serve_*): queued jobs admitted by memory budget, advanced
together between chunks, retired with averages and RDF.

A job's result must be the same whether it runs alone or arrives while other
jobs are resident (continuous batching: it joins the running batch), budget
admission must bind, and Ewald jobs (batched with the other kinds) must
complete too.
"""
import time

import numpy as np
import pytest

from paper_1507_07548_gb300 import workloads as W

ms2 = pytest.importorskip("paper_1507_07548_gb300.ms2")
pytestmark = pytest.mark.gpu


def argon():
    return W.Model("argon", [W.Site((0.0, 0.0, 0.0), 39.948, 3.405, 119.8, lj=True)])


RHO_W = W.WATER_NUMBER_DENSITY
JOBS = [  # (models, counts, T, rho, cutoff, elec)
    ([W.water()], [216], 298.0, RHO_W, 9.0, ms2.ELEC_RF),
    ([W.stockmayer()], [300], 300.0, 0.012, 12.0, ms2.ELEC_RF),
    ([argon()], [500], 120.0, 0.020, 10.0, ms2.ELEC_NONE),
    ([W.water()], [343], 298.0, RHO_W, 10.0, ms2.ELEC_RF),
]


def run(jobs, steps=200, budget=1 << 30, slots=64, stagger=0.0):
    s = ms2.Server(budget, slots)
    ids = []
    for k, (m, c, T, rho, rc, e) in enumerate(jobs):
        ids.append(s.submit(m, c, T, rho, rc, e, steps, arrival=k * stagger, seed=100 + k, rdf_bins=60))
    s.drain(300.0)
    res = {r["job_id"]: r for r in s.poll(256)}
    s.close()
    return [res[i] for i in ids]


def test_serve_completes_jobs_with_outputs():
    res = run(JOBS)
    for r, (m, c, T, *_rest) in zip(res, JOBS):
        assert r["status"] == 0
        assert np.isfinite(r["U"]) and np.isfinite(r["P"])
        assert r["T"] == pytest.approx(T, rel=1e-3)
        assert r["g"] is not None and r["g"].shape[1] == 60 and r["g"].sum() > 0
        assert r["t_arrive"] <= r["t_admit"] <= r["t_done"]


def wait_for(server, got, jid, timeout=120.0):
    t0 = time.time()
    while jid not in got:
        for r in server.poll(64):
            got[r["job_id"]] = r
        if time.time() - t0 > timeout:
            raise TimeoutError("job %d did not finish" % jid)
        time.sleep(0.01)
    return got[jid]


def test_result_is_the_same_alone_and_in_the_mix():
    """The target job alone (a batch of one) and the same job joining a running
    batch of nine other jobs (water, Stockmayer, argon, an Ewald ionic solution)
    mid-stream: its averages and g(r) are bit for bit the same."""
    target = JOBS[0]
    alone = run([target], steps=300)[0]          # seed 100
    ion = W.ionic_solution(n_water=200, n_ion_pairs=4, rc=8.0, seed=5)
    others = [JOBS[1], JOBS[2], JOBS[3], JOBS[1], JOBS[3], JOBS[0], JOBS[3],
              (ion.models, [200, 4, 4], 298.0, RHO_W, 8.0, ms2.ELEC_EWALD)]
    s = ms2.Server(1 << 30, 64)
    got = {}
    oid = [s.submit(*job, 100000, seed=200 + k, rdf_bins=60) for k, job in enumerate(others)]
    # a short job among them: once it is done, the batch has been running
    first = s.submit(*JOBS[2], 200, seed=300, rdf_bins=60)
    wait_for(s, got, first)
    jid = s.submit(*target, 300, arrival=0.0, seed=100, rdf_bins=60)
    mine = wait_for(s, got, jid)
    assert not any(i in got for i in oid)         # the long jobs ran beside it throughout
    s.close()                                    # (and retire unfinished here)
    assert got[first]["status"] == 0 and got[first]["t_done"] <= mine["t_admit"]
    assert mine["status"] == 0
    assert mine["U"] == alone["U"] and mine["P"] == alone["P"] and mine["T"] == alone["T"]
    assert mine["U_err"] == alone["U_err"] and mine["P_err"] == alone["P_err"]
    assert np.array_equal(mine["g"], alone["g"])


def test_budget_admission_binds_and_rejects_oversized_jobs():
    small = ms2.Server(2 << 20, 8)
    with pytest.raises(ms2.Ms2Error, match="EBUDGET"):
        small.submit([W.water()], [4000], 298.0, RHO_W, 14.0, ms2.ELEC_RF, 100)
    small.close()
    # room for two of these jobs at a time (~1.30 MiB each by the admission
    # estimate, which counts the batch's candidate lists)
    job = ([W.water()], [216], 298.0, RHO_W, 9.0, ms2.ELEC_RF)
    s = ms2.Server(int(3.0 * (1 << 20)), 64)
    for k in range(4):
        s.submit(*job, 400, seed=10 + k)
    s.drain(300.0)
    res = sorted(s.poll(16), key=lambda r: r["t_admit"])
    s.close()
    assert len(res) == 4 and all(r["status"] == 0 for r in res)
    # the third admission waited for a retirement
    assert res[2]["t_admit"] >= min(res[0]["t_done"], res[1]["t_done"]) - 1e-6


def test_ewald_job_runs_in_the_batch():
    ion = W.ionic_solution(n_water=200, n_ion_pairs=4, rc=8.0, seed=5)
    res = run([JOBS[0], (ion.models, [200, 4, 4], 298.0, RHO_W, 8.0, ms2.ELEC_EWALD)], steps=100)
    assert all(r["status"] == 0 for r in res)
    assert res[1]["T"] == pytest.approx(298.0, rel=1e-3)
