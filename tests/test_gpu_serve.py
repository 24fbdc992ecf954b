"""Serving (ms2_serve_*): queued jobs admitted by memory budget, advanced
together between chunks, retired with averages and RDF.

A job's result must be the same whether it runs alone or arrives while other
jobs are resident (continuous batching), budget admission must bind, and Ewald
jobs (stepped on their own streams beside the batch) must complete too.
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


def test_result_is_the_same_alone_and_in_the_mix():
    target = JOBS[0]
    alone = run([target], steps=300)[0]          # seed 100
    # the same job (seed 100) arrives while two others are already resident,
    # and a fourth arrives after it
    s = ms2.Server(1 << 30, 64)
    for k, job in enumerate([JOBS[1], JOBS[2]]):
        s.submit(*job, 300, arrival=0.0, seed=200 + k, rdf_bins=60)
    jid = s.submit(*target, 300, arrival=0.05, seed=100, rdf_bins=60)
    s.submit(*JOBS[3], 300, arrival=0.06, seed=203, rdf_bins=60)
    s.drain(300.0)
    got = {x["job_id"]: x for x in s.poll(64)}[jid]
    s.close()
    assert got["t_admit"] >= got["t_arrive"]
    assert got["U"] == alone["U"] and got["P"] == alone["P"] and got["T"] == alone["T"]
    assert np.array_equal(got["g"], alone["g"])


def test_budget_admission_binds_and_rejects_oversized_jobs():
    small = ms2.Server(2 << 20, 8)
    with pytest.raises(ms2.Ms2Error, match="EBUDGET"):
        small.submit([W.water()], [4000], 298.0, RHO_W, 14.0, ms2.ELEC_RF, 100)
    small.close()
    # room for two of these jobs at a time (~1.15 MB each by the admission estimate)
    job = ([W.water()], [216], 298.0, RHO_W, 9.0, ms2.ELEC_RF)
    s = ms2.Server(int(2.6 * (1 << 20)), 64)
    for k in range(4):
        s.submit(*job, 400, seed=10 + k)
    s.drain(300.0)
    res = sorted(s.poll(16), key=lambda r: r["t_admit"])
    s.close()
    assert len(res) == 4 and all(r["status"] == 0 for r in res)
    # the third admission waited for a retirement
    assert res[2]["t_admit"] >= min(res[0]["t_done"], res[1]["t_done"]) - 1e-6


def test_ewald_job_runs_beside_the_batch():
    ion = W.ionic_solution(n_water=200, n_ion_pairs=4, rc=8.0, seed=5)
    res = run([JOBS[0], (ion.models, [200, 4, 4], 298.0, RHO_W, 8.0, ms2.ELEC_EWALD)], steps=100)
    assert all(r["status"] == 0 for r in res)
    assert res[1]["T"] == pytest.approx(298.0, rel=1e-3)
