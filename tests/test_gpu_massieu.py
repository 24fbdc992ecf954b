"""Massieu potential derivatives (paper Sec. 2, Eq. 1) on the GPU.

The volume derivatives dU/dV and d2U/dV2 of a configuration are held to the
FP64 oracle; the eight residual derivatives the library forms from its
running moments are held to the oracle's estimators fed with the same
per-step samples; the fused and per-phase paths agree bit for bit.
"""
import os

import numpy as np
import pytest

from oracle import Oracle
from paper_1507_07548_gb300 import workloads as W

ms2 = pytest.importorskip("paper_1507_07548_gb300.ms2")
pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def snapshot(wl, name):
    z = np.load(os.path.join(GOLDEN, name + ".npz"))
    wl.R, wl.q, wl.v, wl.Lang = z["R"], z["q"], z["v"], z["Lang"]
    return wl


def water():
    return snapshot(W.water_box(N=1000, rc=14.0, seed=2), "water_N1000")


def lj32():
    wl = W.lj_fluid(N=500, rho=0.8, rc=3.5, seed=11)
    wl.R = wl.R + np.random.default_rng(4).normal(0, 0.03, wl.R.shape)
    wl.integrator = 1
    return wl


def lj64():
    return W.lj_fluid(N=256, rho=0.7, T=1.0, rc=3.5, seed=1)


# relative tolerances (dU/dV, d2U/dV2): the FP64 point-LJ path to rounding; the
# FP32 paths at the level of the molecular virial (dU/dV = -W/(3V) - P_LRC) and,
# for d2U/dV2, ~10x the errors measured on GB300 (7e-8 water, 2e-7 LJ)
CASES = [(water, dict(), 5e-6, 1e-6), (lj32, dict(), 1e-6, 2e-6), (lj64, dict(fp64=1), 1e-11, 1e-12)]


@pytest.mark.parametrize("make,kw,tol1,tol2", CASES, ids=["water_rf", "lj_fp32", "lj_fp64"])
def test_volume_derivatives_match_oracle(make, kw, tol1, tol2):
    wl = make()
    s = ms2.System.from_workload(wl, massieu=1, **kw)
    UV, UVV = s.volume_derivatives()
    o = Oracle.from_workload(wl)
    oUV, oUVV = o.volume_derivatives(wl.R, wl.q)
    assert UV == pytest.approx(oUV, rel=tol1)
    assert UVV == pytest.approx(oUVV, rel=tol2)


@pytest.mark.parametrize("make,kw", [(water, dict()), (lj64, dict(fp64=1))], ids=["water_rf", "lj_fp64"])
def test_massieu_estimators_from_the_gpu_samples(make, kw):
    wl = make()
    s = ms2.System.from_workload(wl, massieu=1, **kw)
    s.reset_averages()
    samples = []
    for _ in range(40):
        s.step(1)
        U = s.energy_virial()[0]
        samples.append((U,) + s.volume_derivatives())
    got, n = s.massieu()
    assert n == 40
    S = np.array(samples)
    U0, V0 = S[0, 0], S[0, 1]
    x, y, w = S[:, 0] - U0, S[:, 1] - V0, S[:, 2]
    acc = [len(S)] + [float(f.sum()) for f in (x, x ** 2, x ** 3, y, y ** 2, x * y, x * x * y, x * y * y, w, x * w)]
    o = Oracle.from_workload(wl)
    want = Oracle.massieu(np.array(acc), U0, V0, 1.0 / wl.T, wl.L ** 3, wl.N)
    for k, name in enumerate(ms2.System.MASSIEU_NAMES):
        assert got[name] == pytest.approx(want[k], rel=1e-8, abs=1e-12 * max(1.0, abs(want[k]))), name


def test_fused_massieu_run_equals_per_phase_kernels_bitwise():
    wl = water()
    a = ms2.System.from_workload(wl, massieu=1)
    b = ms2.System.from_workload(wl, massieu=1, fused_step=0)
    assert a.fused_step() == 1 and b.fused_step() == 0
    for s in (a, b):
        s.reset_averages()
        s.step(75)
    assert a.massieu() == b.massieu()
    assert a.volume_derivatives() == b.volume_derivatives()


def test_massieu_kernels_agree_with_the_plain_kernels():
    """The Massieu kernels keep every site-pair row scalar; the plain water
    kernels evaluate the two H rows together in packed FP32x2 arithmetic.  Both
    evaluate the same configuration to FP32 rounding: energies agree, forces and
    torques to well inside the oracle bar, on the fused and on the per-phase path."""
    wl = water()
    for fused in (1, 0):
        a = ms2.System.from_workload(wl, massieu=1, fused_step=fused)
        b = ms2.System.from_workload(wl, fused_step=fused)
        assert a.fused_step() == b.fused_step() == fused
        Fa, Ta = a.forces_torques()
        Fb, Tb = b.forces_torques()
        assert np.linalg.norm(Fa - Fb) <= 1e-6 * np.linalg.norm(Fb)
        assert np.linalg.norm(Ta - Tb) <= 1e-6 * np.linalg.norm(Tb)
        Ua, Ub = a.energy_virial()[0], b.energy_virial()[0]
        assert abs(Ua - Ub) <= 1e-12 * abs(Ub)


def test_massieu_option_rejects_ewald_and_dipoles():
    ion = W.ionic_solution(n_water=200, n_ion_pairs=4, rc=8.0, seed=5)
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        ms2.System.from_workload(ion, massieu=1)
    st = W.stockmayer_fluid(N=200, seed=4)
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        ms2.System.from_workload(st, massieu=1)
    s = ms2.System.from_workload(water())
    with pytest.raises(ms2.Ms2Error, match="ESTATE"):
        s.volume_derivatives()
