"""Batched systems (ms2_batch_*): one cooperative kernel per model kind steps all systems.

Checks: one batched step against the FP64 oracle (same tolerances as the
single-system path), bit-identical results for a system alone and inside a
mixed batch, RDF/average bookkeeping, and rejection of systems the batch kernel
does not take.
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
    return snapshot(W.water_box(N=216, rc=9.0, seed=9), "water_N216")


def stock():
    return snapshot(W.stockmayer_fluid(N=500, seed=4), "stockmayer_N500")


def ljf():
    wl = W.lj_fluid(N=500, rho=0.8, rc=3.5, seed=11)
    wl.R = wl.R + np.random.default_rng(4).normal(0, 0.03, wl.R.shape)
    wl.integrator = 1
    return wl


def rms_rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("make", [water, stock, ljf], ids=["water", "stockmayer", "lj"])
def test_one_batched_step_matches_oracle(make):
    wl = make()
    s = ms2.System.from_workload(wl)
    b = ms2.Batch([s])
    b.step(1)
    R, q, v, L, st = s.get_state()
    assert st == 1
    o = Oracle.from_workload(wl)
    Ro, qo, vo, Lo, th, _ = o.run_leapfrog(wl.R, wl.q, wl.v, wl.Lang, wl.dt, 1, T0=wl.T)
    dR = Ro - wl.R
    assert np.abs((R - wl.R) - dR).max() <= 1e-6 * np.abs(dR).max()
    assert rms_rel(v, vo) <= 1e-6
    if np.linalg.norm(Lo) > 0:
        sgn = np.sign((q * qo).sum(1))[:, None]
        assert np.abs(q * sgn - qo).max() <= 1e-7
        assert rms_rel(L, Lo) <= 1e-5
    U, Wv, T, P = s.energy_virial()
    assert abs(U - th[0, 0]) <= 1e-6 * abs(th[0, 0])
    Wo = o.forces(R, q)[2]["W_total"]  # the virial on the identical (stepped) configuration
    assert abs(Wv - Wo) <= 1e-6 * abs(Wo)
    F, tau = s.forces_torques()
    Fo, To, _ = o.forces(Ro, qo)
    assert rms_rel(F, Fo) <= 1e-5


def dilute_lj():
    wl = W.lj_fluid(N=1372, rho=0.3, rc=3.0, T=1.5, seed=17)
    wl.integrator = 1
    return wl


def dilute_water():
    return W.water_box(N=1000, rc=14.0, seed=19, density=0.5 * W.WATER_NUMBER_DENSITY)


@pytest.mark.parametrize("make", [dilute_lj, dilute_water], ids=["lj", "water"])
def test_candidate_lists_find_every_partner(make):
    """Dilute systems take candidate lists in a batch (the list within r_c + skin
    holds 5 % and 42 % of the molecules).  After 150 batched steps in two launches
    (list builds at each launch and whenever a molecule has moved half the skin,
    list scans in between), each molecule's partner count equals that of a full
    evaluation of the same state, and the forces are the oracle's."""
    wl = make()
    s = ms2.System.from_workload(wl)
    b = ms2.Batch([s])
    b.step(150)
    R, q, v, L, _ = s.get_state()
    c = ms2.System.from_workload(wl)
    c.set_state(R, q, v, L)
    assert np.array_equal(np.asarray(s.partner_counts()), np.asarray(c.partner_counts()))
    F, tau = s.forces_torques()
    Fo, To, _ = Oracle.from_workload(wl).forces(R, q)
    assert rms_rel(F, Fo) <= 1e-5
    if np.linalg.norm(To) > 0:
        assert rms_rel(tau, To) <= 1e-5
    b.close()


def test_system_alone_and_in_a_mixed_batch_is_bitwise_identical():
    alone = ms2.System.from_workload(water())
    b1 = ms2.Batch([alone])
    b1.step(30)
    ref = alone.get_state()[:4]
    mix = [ms2.System.from_workload(w) for w in (ljf(), water(), stock(), water())]
    b2 = ms2.Batch(mix)
    b2.step(30)
    got = mix[1].get_state()[:4]
    for a, c in zip(got, ref):
        assert np.array_equal(a, c)
    assert alone.energy_virial() == mix[1].energy_virial()


def test_large_system_alone_and_beside_small_ones_is_bitwise_identical():
    """A system above 2048 molecules runs in its kind's large-size group, with
    its own block shape: alone, beside small systems of its kind, and stepped in
    two chunks, its state comes out the same bit for bit."""
    def big():
        wl = W.water_box(N=2744, rc=12.0, seed=31)   # unrelaxed lattice start: a short time step
        wl.dt = 0.5
        return wl
    alone = ms2.System.from_workload(big())
    b1 = ms2.Batch([alone])
    b1.step(24)
    ref = alone.get_state()[:4]
    mix = [ms2.System.from_workload(w) for w in (water(), big(), ljf(), water())]
    b2 = ms2.Batch(mix)
    b2.step(10)
    b2.step(14)
    got = mix[1].get_state()[:4]
    for a, c in zip(got, ref):
        assert np.array_equal(a, c)
    assert alone.energy_virial() == mix[1].energy_virial()


def test_full_size_mix_sampled_systems_match_oracle():
    """The batch benchmark's workload at full size, launched as the benchmark
    launches it: the 512-system mix (point LJ, Stockmayer, water; N ~ U[256,
    2048], seeded lattice starts) in one batch, one step.  Sampled systems -- the
    smallest and the largest of each kind -- against the oracle's step from the
    same state, at the single-system tolerances, and their partner counts
    bit-exact against a full evaluation of the stepped state."""
    specs = W.system_mix(512, seed=4)
    systems = [ms2.System(sp["models"], sp["counts"], sp["T"], sp["cutoff"], sp["elec"], rho=sp["rho"],
                          seed=sp["seed"], dt=2.0) for sp in specs]
    pick = []
    for kind in W.MIX_STATES:
        idx = sorted((k for k, sp in enumerate(specs) if sp["name"] == kind), key=lambda k: specs[k]["counts"][0])
        pick += [idx[0], idx[-1]]
    start = {k: systems[k].get_state() for k in pick}
    b = ms2.Batch(systems)
    b.step(1)
    for k in pick:
        sp, s = specs[k], systems[k]
        R0, q0, v0, L0, _ = start[k]
        R, q, v, L, st = s.get_state()
        assert st == 1
        o = Oracle(sp["models"], np.zeros(s.N, np.int32), s.L, s.rc, elec=sp["elec"])
        Ro, qo, vo, Lo, th, _ = o.run_leapfrog(R0, q0, v0, L0, 2.0, 1, T0=sp["T"])
        dR = Ro - R0
        assert np.abs((R - R0) - dR).max() <= 1e-6 * np.abs(dR).max(), sp["name"]
        assert rms_rel(v, vo) <= 1e-6, sp["name"]
        if np.linalg.norm(Lo) > 0:
            sgn = np.sign((q * qo).sum(1))[:, None]
            assert np.abs(q * sgn - qo).max() <= 1e-7, sp["name"]
            assert rms_rel(L, Lo) <= 1e-5, sp["name"]
        U, Wv, T, P = s.energy_virial()
        assert abs(U - th[0, 0]) <= 1e-6 * abs(th[0, 0]), sp["name"]
        F, tau = s.forces_torques()
        Fo, To, to = o.forces(R, q)  # the identical (stepped) configuration
        assert abs(Wv - to["W_total"]) <= 1e-6 * abs(to["W_total"]), sp["name"]
        assert rms_rel(F, Fo) <= 1e-5, sp["name"]
        if np.linalg.norm(To) > 0:
            assert rms_rel(tau, To) <= 1e-5, sp["name"]
        c = ms2.System(sp["models"], sp["counts"], sp["T"], sp["cutoff"], sp["elec"], rho=sp["rho"],
                       seed=sp["seed"], dt=2.0)
        c.set_state(R, q, v, L)
        assert np.array_equal(np.asarray(s.partner_counts()), np.asarray(c.partner_counts())), sp["name"]
        c.close()
    b.close()
    for s in systems:
        s.close()


def test_batch_matches_single_system_stepping_closely():
    a = ms2.System.from_workload(water())
    b = ms2.System.from_workload(water())
    a.step(20)
    bb = ms2.Batch([b])
    bb.step(20)
    Ra, Rb = a.get_state()[0], b.get_state()[0]
    assert np.abs(Ra - Rb).max() < 1e-4
    Ua, Ub = a.energy_virial()[0], b.energy_virial()[0]
    assert abs(Ua - Ub) <= 1e-4 * abs(Ua)


def test_batch_rdf_and_averages_bookkeeping():
    s = ms2.System.from_workload(water())
    s.rdf_setup(min(9.0, 0.5 * s.L), 90, every=10)
    s.reset_averages()
    b = ms2.Batch([s, ms2.System.from_workload(stock())])
    b.step(100)
    c, g, ns = s.rdf()
    assert ns == 10
    assert c.sum() > 0
    tail = g[0, -20:]
    assert abs(tail.mean() - 1.0) < 0.1
    av = s.averages()
    assert av["n"] == 100
    assert av["T"] == pytest.approx(298.0, rel=1e-3)


def ionic():
    return snapshot(W.ionic_solution(seed=3), "ionic_N1040")


def test_one_batched_ewald_step_matches_oracle():
    """The ionic solution (water + ions, Ewald) in a batch: the reciprocal-space
    tasks run between grid barriers of the multi-system kernel."""
    wl = ionic()
    s = ms2.System.from_workload(wl)
    b = ms2.Batch([s])
    b.step(1)
    R, q, v, L, st = s.get_state()
    assert st == 1
    o = Oracle.from_workload(wl)
    Ro, qo, vo, Lo, th, _ = o.run_leapfrog(wl.R, wl.q, wl.v, wl.Lang, wl.dt, 1, T0=wl.T)
    dR = Ro - wl.R
    assert np.abs((R - wl.R) - dR).max() <= 1e-6 * np.abs(dR).max()
    assert rms_rel(v, vo) <= 1e-6
    U, Wv, T, P = s.energy_virial()
    assert abs(U - th[0, 0]) <= 1e-6 * abs(th[0, 0])
    F, tau = s.forces_torques()
    Fo, To, to = o.forces(R, q)                   # the identical (stepped) configuration
    assert rms_rel(F, Fo) <= 1e-5 and rms_rel(tau, To) <= 1e-5
    assert abs(Wv - to["W_total"]) <= 1e-5 * abs(to["W_total"])   # W_EWALD of test_gpu_parity
    t = s.energy_terms()
    assert t["U_rec"] == pytest.approx(to["U_rec"], rel=1e-6)
    b.close()


def test_ewald_system_alone_and_in_a_mixed_batch_is_bitwise_identical():
    alone = ms2.System.from_workload(ionic())
    b1 = ms2.Batch([alone])
    b1.step(12)
    ref = alone.get_state()[:4]
    small = W.ionic_solution(n_water=400, n_ion_pairs=8, rc=9.0, seed=7)
    mix = [ms2.System.from_workload(w) for w in (water(), small, ionic(), stock())]
    b2 = ms2.Batch(mix)
    b2.step(12)
    got = mix[2].get_state()[:4]
    for a, c in zip(got, ref):
        assert np.array_equal(a, c)
    assert alone.energy_virial() == mix[2].energy_virial()


def test_batch_rejects_verlet_and_other_ewald_systems():
    m = W.water()                     # a TIP4P-like 4-site water: no batch kind takes it under Ewald
    m.sites[0].charge = 0.0
    m.sites.append(W.Site((0.0, 0.0, m.sites[0].pos[2] + 0.15), 0.0, charge=-0.8476))
    ion4 = ms2.System([m, W.cation(), W.anion()], [100, 2, 2], 298.0, 7.0, ms2.ELEC_EWALD,
                      rho=W.WATER_NUMBER_DENSITY)
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        ms2.Batch([ion4])
    wl = W.lj_fluid(N=256, rho=0.7, rc=3.5)
    vv = ms2.System.from_workload(wl)
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        ms2.Batch([vv])
