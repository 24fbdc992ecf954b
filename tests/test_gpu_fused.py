"""Fused step (ms2_options.fused_step): a chunk of leapfrog steps as one
cooperative kernel.  It runs the per-phase kernels' device functions on their
work decomposition, so its results must equal theirs bit for bit: state,
energies, running averages and RDF counts after several chunks.  The per-phase
path itself is held to the FP64 oracle in test_gpu_parity.py; this file adds
one direct oracle check of a fused step as well.
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


def water1000():
    return snapshot(W.water_box(N=1000, rc=14.0, seed=2), "water_N1000")


def water_ragged():
    wl = W.water_box(N=1003, rc=14.0, seed=21)  # unrelaxed lattice start: a short time step
    wl.dt = 0.5
    return wl


def water_large():
    wl = W.water_box(N=2744, rc=14.0, seed=22)  # 19 molecules per block; unrelaxed lattice start
    wl.dt = 0.5
    return wl


def water_tiny():
    wl = W.water_box(N=100, rc=7.0, seed=23)  # fewer molecules than blocks: blocks that own none
    wl.dt = 0.5
    return wl


def stock():
    return snapshot(W.stockmayer_fluid(N=500, seed=4), "stockmayer_N500")


def lj32():
    wl = W.lj_fluid(N=500, rho=0.8, rc=3.5, seed=11)
    wl.R = wl.R + np.random.default_rng(4).normal(0, 0.03, wl.R.shape)
    wl.integrator = 1
    return wl


def ionic():
    return snapshot(W.ionic_solution(seed=3), "ionic_N1040")


CASES = [water1000, water_ragged, water_large, water_tiny, stock, lj32, ionic]
IDS = ["water1000", "water1003", "water2744", "water100", "stockmayer", "lj", "ionic_ewald"]


def rms_rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("make", CASES, ids=IDS)
def test_fused_chunks_equal_per_phase_kernels_bitwise(make):
    wl = make()
    a = ms2.System.from_workload(wl)
    b = ms2.System.from_workload(wl, fused_step=0)
    assert a.fused_step() == 1 and b.fused_step() == 0
    for s in (a, b):
        s.rdf_setup(min(s.rc, 0.5 * s.L), 80, every=7)
        s.reset_averages()
    assert a.fused_step() == 1
    # 120 steps = chunks of 50, 50, 20 (graph_chunk); RDF samples at 7, 14, ...
    for s in (a, b):
        s.step(120)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(np.asarray(x), np.asarray(y))
    assert a.energy_virial() == b.energy_virial()
    ta, tb = a.energy_terms(), b.energy_terms()
    assert ta == tb
    assert a.averages() == b.averages()
    ca, ga, _ = a.rdf()
    cb, gb, _ = b.rdf()
    assert ca.sum() > 0
    assert np.array_equal(ca, cb) and np.array_equal(ga, gb)
    Fa, Ta = a.forces_torques()
    Fb, Tb = b.forces_torques()
    assert np.array_equal(Fa, Fb) and np.array_equal(Ta, Tb)
    assert np.array_equal(a.molecule_energies(), b.molecule_energies())


def test_smaller_system_created_later_leaves_the_larger_one_launchable():
    """A kernel's dynamic shared-memory limit is one setting shared by every
    system that launches it: a small system of the same model, created after a
    large one, must not lower the limit the large one's pair tile needs."""
    big = ms2.System.from_workload(water_large(), fused_step=0)
    small = ms2.System.from_workload(W.water_box(N=216, rc=9.0, seed=9), fused_step=0)
    F, tau = big.forces_torques()  # the per-phase pair kernel with the large tile
    big.step(2)
    small.step(2)
    ref = ms2.System.from_workload(water_large(), fused_step=0)
    Fr, taur = ref.forces_torques()
    ref.step(2)
    assert np.array_equal(F, Fr) and np.array_equal(tau, taur)
    for x, y in zip(big.get_state(), ref.get_state()):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_fused_step_matches_oracle():
    wl = water1000()
    s = ms2.System.from_workload(wl)
    assert s.fused_step() == 1
    s.step(1)
    R, q, v, L, st = s.get_state()
    assert st == 1
    o = Oracle.from_workload(wl)
    Ro, qo, vo, Lo, th, _ = o.run_leapfrog(wl.R, wl.q, wl.v, wl.Lang, wl.dt, 1, T0=wl.T)
    dR = Ro - wl.R
    assert np.abs((R - wl.R) - dR).max() <= 1e-6 * np.abs(dR).max()
    sgn = np.sign((q * qo).sum(1))[:, None]
    assert np.abs(q * sgn - qo).max() <= 1e-7
    assert rms_rel(v, vo) <= 1e-6
    assert rms_rel(L, Lo) <= 1e-5
    U, Wv, T, P = s.energy_virial()
    assert abs(U - th[-1, 0]) <= 1e-6 * abs(th[-1, 0])
    # the virial on the identical configuration (the stepped GPU state): it moves
    # ~1e-6 under position changes of 1e-8 A, the size of the one-step deviation
    Wo = o.forces(R, q)[2]["W_total"]
    assert abs(Wv - Wo) <= 1e-6 * abs(Wo)
    assert T == pytest.approx(2 * (th[-1, 2] + th[-1, 3]) / o.ndof(), rel=1e-9)


def test_fused_timing_reports_pair_phase():
    s = ms2.System.from_workload(water1000())
    s.enable_timing(True)
    s.step(3)
    pair, ew, step, rest = s.last_step_times()
    assert 0 < pair < step and ew == 0.0 and rest > 0


def test_largest_rdf_histogram_stays_fused_and_exact():
    wl = water1000()
    a = ms2.System.from_workload(wl)
    b = ms2.System.from_workload(wl, fused_step=0)
    for s in (a, b):
        s.rdf_setup(min(s.rc, 0.5 * s.L), 12288, every=3)  # the largest histogram (48 KB of counters)
    assert a.fused_step() == 1
    for s in (a, b):
        s.step(9)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(np.asarray(x), np.asarray(y))
    assert np.array_equal(a.rdf()[0], b.rdf()[0])


def test_fused_ewald_step_matches_oracle():
    """The ionic solution (Ewald, water + ions) as one fused launch: its
    reciprocal-space tasks run between grid barriers inside the step kernel."""
    wl = ionic()
    s = ms2.System.from_workload(wl)
    assert s.fused_step() == 1
    s.step(1)
    R, q, v, L, st = s.get_state()
    o = Oracle.from_workload(wl)
    Ro, qo, vo, Lo, th, _ = o.run_leapfrog(wl.R, wl.q, wl.v, wl.Lang, wl.dt, 1, T0=wl.T)
    dR = Ro - wl.R
    assert np.abs((R - wl.R) - dR).max() <= 1e-6 * np.abs(dR).max()
    assert rms_rel(v, vo) <= 1e-6
    U, Wv, T, P = s.energy_virial()
    assert abs(U - th[-1, 0]) <= 1e-6 * abs(th[-1, 0])
    F, tau = s.forces_torques()
    Fo, To, to = o.forces(R, q)
    # the virial on the identical configuration, to the FP32 floor of the
    # real-space terms of the ionic solution (test_gpu_parity.W_EWALD)
    assert abs(Wv - to["W_total"]) <= 1e-5 * abs(to["W_total"])
    assert rms_rel(F, Fo) <= 1e-5 and rms_rel(tau, To) <= 1e-5
    t = s.energy_terms()
    assert t["U_rec"] == pytest.approx(to["U_rec"], rel=1e-6)
