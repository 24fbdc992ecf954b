"""Long-run statistical parity: GPU and FP64 oracle NVT trajectories of the same
liquid sample the same ensemble.

Both start from the 216-water liquid snapshot (reaction field, rc = 9 A, 298 K,
isokinetic leapfrog, dt = 2 fs) and run 2e4 steps.  The FP32 site-pair forces
make the two trajectories decorrelate within a few hundred steps, so they agree
only statistically: <U>, <P> and the coordination number from g(r) must agree
within 2 sigma of their Flyvbjerg-Petersen block-averaged standard errors
(combined in quadrature), and g(r) bin by bin within 3 sigma for nearly all
bins (Sec. "Property Calculations", Eq. 2; the NVT averages of Sec. "Massieu
potential derivatives").
"""
import os

import numpy as np
import pytest

from oracle import Oracle
from paper_1507_07548_gb300 import workloads as W

ms2 = pytest.importorskip("paper_1507_07548_gb300.ms2")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
EVERY, SAMPLES, BLOCKS = 10, 2000, 20   # 2e4 steps, one sample every 10, g(r) in 20 blocks
R_MAX, BINS = 9.0, 90


def blocked_error(x):
    """Standard error of the mean of a correlated series by Flyvbjerg-Petersen
    blocking: the largest estimate over the blocking levels that keep >= 16
    blocks (the plateau, where blocks are uncorrelated)."""
    x = np.asarray(x, float)
    best = 0.0
    while len(x) >= 16:
        n = len(x)
        best = max(best, np.sqrt(x.var(ddof=1) / n))
        x = 0.5 * (x[: n // 2 * 2 : 2] + x[1 : n // 2 * 2 : 2])
    return best


def workload():
    wl = W.water_box(N=216, rc=9.0, seed=9)
    z = np.load(os.path.join(GOLDEN, "water_N216.npz"))
    wl.R, wl.q, wl.v, wl.Lang = z["R"], z["q"], z["v"], z["Lang"]
    return wl


def gpu_run(wl):
    s = ms2.System.from_workload(wl)
    s.rdf_setup(R_MAX, BINS, every=EVERY)
    U, P, blocks = [], [], []
    prev = np.zeros((1, BINS), np.int64)
    for k in range(SAMPLES):
        s.step(EVERY)
        u, _, _, p = s.energy_virial()
        U.append(u)
        P.append(p)
        if (k + 1) % (SAMPLES // BLOCKS) == 0:
            c = s.rdf()[0]
            blocks.append(c - prev)
            prev = c
    s.close()
    return np.array(U), np.array(P), np.array(blocks)


def oracle_run(wl):
    o = Oracle.from_workload(wl)
    R, q, v, L = wl.R, wl.q, wl.v, wl.Lang
    U, P, blocks = [], [], []
    acc = None
    for k in range(SAMPLES):
        R, q, v, L, th, _ = o.run_leapfrog(R, q, v, L, wl.dt, EVERY, T0=wl.T)
        U.append(th[-1, 0])
        P.append(th[-1, 4])
        c = o.rdf_counts(R, q, R_MAX, BINS)
        acc = c if acc is None else acc + c
        if (k + 1) % (SAMPLES // BLOCKS) == 0:
            blocks.append(acc)
            acc = None
    return np.array(U), np.array(P), np.array(blocks)


def z_score(a, b):
    ea, eb = blocked_error(a), blocked_error(b)
    return abs(a.mean() - b.mean()) / np.hypot(ea, eb), ea, eb


def test_long_run_averages_agree_with_the_oracle():
    wl = workload()
    Ug, Pg, Bg = gpu_run(wl)
    Uo, Po, Bo = oracle_run(wl)
    zu, eu_g, eu_o = z_score(Ug, Uo)
    zp, ep_g, ep_o = z_score(Pg, Po)
    print("<U> gpu %.1f +- %.1f, oracle %.1f +- %.1f K (z %.2f); <P> gpu %.4f +- %.4f, oracle %.4f +- %.4f "
          "K/A^3 (z %.2f)" % (Ug.mean(), eu_g, Uo.mean(), eu_o, zu, Pg.mean(), ep_g, Po.mean(), ep_o, zp))
    # the errors are those of a decorrelated run, not of a frozen one
    assert 0 < eu_g < 2e-3 * abs(Ug.mean()) and 0 < eu_o < 2e-3 * abs(Uo.mean())
    assert zu <= 2.0 and zp <= 2.0
    # g(r) of the single LJ-site kind pair (O-O): per-block histograms, same samples per block
    hg, ho = Bg[:, 0, :].astype(float), Bo[:, 0, :].astype(float)
    mg, mo = hg.mean(0), ho.mean(0)
    sg, so = hg.std(0, ddof=1) / np.sqrt(BLOCKS), ho.std(0, ddof=1) / np.sqrt(BLOCKS)
    used = (mg + mo) > 0
    zb = np.abs(mg - mo)[used] / np.maximum(np.hypot(sg, so)[used], 1e-12)
    assert np.mean(zb <= 3.0) >= 0.95, np.sort(zb)[-10:]
    # coordination number up to the first minimum of g_OO (3.3 A): block series
    k1 = int(3.3 / (R_MAX / BINS))
    zc, _, _ = z_score(hg[:, :k1].sum(1), ho[:, :k1].sum(1))
    assert zc <= 2.0
