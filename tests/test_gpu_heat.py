"""Green-Kubo thermal conductivity (paper Sec. 4, Eqs. 5-6) on the GPU.

The sampled heat flux J_q is held to the oracle's pair sum of the same
configuration at the integer-time velocities, for each kind of interaction the
power pass handles: LJ centres (leapfrog and velocity Verlet), water with the
reaction field, Stockmayer dipoles and a water-argon mixture with partial molar
enthalpies.  The device autocorrelation and lambda are held to the oracle's
autocorrelation and trapezoidal integral of the GPU's own samples; fused and
per-phase sampling agree bit for bit and sampling leaves the trajectory as it is.
"""
import os

import numpy as np
import pytest

from oracle import Oracle
from paper_1507_07548_gb300 import workloads as W

ms2 = pytest.importorskip("paper_1507_07548_gb300.ms2")
pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# |J_gpu - J_oracle| / |J_oracle|: FP32 site-pair forces and powers, FP32 lane
# sums of d_kl P_kl, FP64 kinetic part and molecular sums (seen on GB300:
# 5e-7 .. 1.4e-6 over the five systems)
TOL_J = 5e-6


def snapshot(wl, name):
    z = np.load(os.path.join(GOLDEN, name + ".npz"))
    wl.R, wl.q, wl.v, wl.Lang = z["R"], z["q"], z["v"], z["Lang"]
    return wl


def water1000():
    return snapshot(W.water_box(N=1000, rc=14.0, seed=2), "water_N1000")


def stock():
    return snapshot(W.stockmayer_fluid(N=500, seed=4), "stockmayer_N500")


def lj_leapfrog():
    wl = W.lj_fluid(N=500, rho=0.8, rc=3.5, seed=11)
    wl.R = wl.R + np.random.default_rng(4).normal(0, 0.03, wl.R.shape)
    wl.integrator = 1
    return wl


def lj_verlet():
    wl = W.lj_fluid(N=864, rho=0.75, rc=3.0, seed=12)
    wl.R = wl.R + np.random.default_rng(5).normal(0, 0.03, wl.R.shape)
    return wl


def mixture():
    wl = W.water_argon(n_water=700, n_argon=300, seed=6)
    wl.dt = 0.5
    return wl


def integer_time_velocities(wl, o, s):
    """State after the last step and the oracle's velocities at its integer time."""
    R, q, v, L, _ = s.get_state()
    if wl.integrator == 0:
        return R, q, v, L
    F, tau, _ = o.forces(R, q)
    M = np.array([sum(st.mass for st in m.sites) for m in wl.models])[wl.species]
    kc = o.s.kconv
    return R, q, v + 0.5 * wl.dt * kc * F / M[:, None], L + 0.5 * wl.dt * kc * tau


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


CASES = [(water1000, [0.0]), (stock, [-2500.0]), (lj_leapfrog, [0.0]), (lj_verlet, [1.5]),
         (mixture, [-4000.0, 350.0])]
IDS = ["water1000", "stockmayer", "lj_leapfrog", "lj_verlet", "water_argon"]


@pytest.mark.parametrize("make,h", CASES, ids=IDS)
@pytest.mark.parametrize("fused", [1, 0], ids=["fused", "per_phase"])
def test_heat_flux_matches_oracle(make, h, fused):
    wl = make()
    s = ms2.System.from_workload(wl, fused_step=fused)
    s.heat_setup(every=1, n_lags=4, h=h)
    s.step(2)
    J = s.heat_flux()
    o = Oracle.from_workload(wl)
    R, q, v, L = integer_time_velocities(wl, o, s)
    Jo = o.heat_flux(R, q, v, L, h=h)
    assert np.linalg.norm(Jo) > 0
    assert rel(J, Jo) <= TOL_J, (J, Jo, rel(J, Jo))


def test_enthalpy_term_is_minus_h_times_the_species_momentum_sum():
    wl = mixture()
    a = ms2.System.from_workload(wl)
    b = ms2.System.from_workload(wl)
    a.heat_setup(every=1, n_lags=4, h=[0.0, 0.0])
    b.heat_setup(every=1, n_lags=4, h=[-4000.0, 350.0])
    a.step(1)
    b.step(1)
    # the integer-time velocities the device used: its own forces
    _, _, v, _, _ = a.get_state()
    F, _ = a.forces_torques()
    M = np.array([sum(st.mass for st in m.sites) for m in wl.models])[wl.species]
    v = v + 0.5 * wl.dt * Oracle.from_workload(wl).s.kconv * F / M[:, None]
    want = 4000.0 * v[wl.species == 0].sum(0) - 350.0 * v[wl.species == 1].sum(0)
    np.testing.assert_allclose(b.heat_flux() - a.heat_flux(), want, rtol=1e-9, atol=1e-9 * np.abs(want).max())


def test_autocorrelation_and_lambda_of_the_gpu_samples():
    wl = water1000()
    s = ms2.System.from_workload(wl)
    every, lags, n = 2, 12, 30
    s.heat_setup(every=every, n_lags=lags)
    samples = []
    for _ in range(n):
        s.step(every)
        samples.append(s.heat_flux())
    lam, acf, ns = s.thermal_conductivity()
    assert ns == n
    want = Oracle.flux_acf(np.array(samples), lags)
    np.testing.assert_allclose(acf, want, rtol=1e-10, atol=1e-13 * abs(want[0]))
    lam_o = Oracle.thermal_conductivity(want, every * wl.dt, wl.L ** 3, wl.T)
    assert lam == pytest.approx(lam_o, rel=1e-9)
    assert np.isfinite(lam) and acf[0] > 0


@pytest.mark.parametrize("make", [water1000, stock, lj_leapfrog], ids=["water1000", "stockmayer", "lj"])
def test_fused_sampling_equals_per_phase_and_leaves_the_trajectory(make):
    wl = make()
    a = ms2.System.from_workload(wl)
    b = ms2.System.from_workload(wl, fused_step=0)
    c = ms2.System.from_workload(wl)
    for s in (a, b):
        s.heat_setup(every=3, n_lags=10, h=[-100.0])
    assert a.fused_step() == 1 and b.fused_step() == 0
    # 120 steps = chunks of 50, 50, 20; samples at 3, 6, ..., the chunk ends on none
    # and on one (step 120)
    for s in (a, b, c):
        s.step(120)
    assert np.array_equal(a.heat_flux(), b.heat_flux())
    ra, rb = a.thermal_conductivity(), b.thermal_conductivity()
    assert ra[2] == rb[2] == 40
    assert ra[0] == rb[0] and np.array_equal(ra[1], rb[1])
    for x, y, z in zip(a.get_state(), b.get_state(), c.get_state()):
        assert np.array_equal(np.asarray(x), np.asarray(y))
        assert np.array_equal(np.asarray(x), np.asarray(z))
    assert a.energy_virial() == c.energy_virial()


def test_setup_checks_arguments_and_ewald_is_refused():
    s = ms2.System.from_workload(water1000())
    with pytest.raises(ms2.Ms2Error, match="ESTATE"):
        s.heat_flux()
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        s.heat_setup(every=0, n_lags=8)
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        s.heat_setup(every=1, n_lags=1)
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        s.heat_setup(every=1, n_lags=8, h=[float("nan")])
    wl = W.ionic_solution(seed=3)
    e = ms2.System.from_workload(snapshot(wl, "ionic_N1040"))
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        e.heat_setup(every=1, n_lags=8)


def test_heat_flux_ragged_system_fused():
    """1003 molecules (a ragged last block of the fused decomposition)."""
    wl = W.water_box(N=1003, rc=14.0, seed=21)
    wl.dt = 0.5
    s = ms2.System.from_workload(wl)
    s.heat_setup(every=1, n_lags=4, h=[100.0])
    assert s.fused_step() == 1
    s.step(2)
    o = Oracle.from_workload(wl)
    R, q, v, L = integer_time_velocities(wl, o, s)
    Jo = o.heat_flux(R, q, v, L, h=[100.0])
    assert rel(s.heat_flux(), Jo) <= TOL_J
