"""GPU (libms2, through the C ABI) against the FP64 oracle on identical inputs.

Tolerances: FP64 path (point LJ, velocity Verlet) 1e-12 per evaluation and
1e-9 on positions after 100 steps; FP32 site-pair path: force and torque RMS
relative error <= 1e-5, energy and virial relative error <= 1e-6; integer
results (partner counts, RDF histograms) bit-exact up to pairs that lie within
FP32 rounding of a bin edge.
"""
import math
import os

import numpy as np
import pytest

from oracle import Oracle
from paper_1507_07548_gb300 import workloads as W

ms2 = pytest.importorskip("paper_1507_07548_gb300.ms2")
pytestmark = pytest.mark.gpu


def rms_rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# The molecular virial of the ionic solution at ambient pressure is ~1/100 of its
# LJ and real-space Coulomb parts (W = -2.0e5 K against +2.4e7 K of LJ virial and
# -1.8e7 K of site-lever terms).  Every FP32 constant of the Ewald terms carries
# its rounding remainder and close LJ pairs are double-float; what is left is the
# FP32 rounding of the erfc argument and of the arithmetic around erfcf/expf in
# the ~3.5e6 charged site pairs, ~7e-3 K rms per molecule by an FP32 emulation of
# the kernel, i.e. 0.1-0.6 K in W: measured 7e-7 on the snapshot and 2e-7 -
# 4.8e-6 on the states of the next five steps.  The Ewald cases are held to
# W_EWALD; every other case and every energy to 1e-6.
W_EWALD = 1e-5


def compare(s, o, R, q, tol_f=1e-5, tol_e=1e-6, tol_w=None):
    F, tau = s.forces_torques()
    t = s.energy_terms()
    Fo, To, to = o.forces(R, q)
    assert rms_rel(F, Fo) <= tol_f
    if np.linalg.norm(To) > 0:
        assert rms_rel(tau, To) <= tol_f
    assert abs(t["U_total"] - to["U_total"]) <= tol_e * abs(to["U_total"])
    tol_w = tol_e if tol_w is None else tol_w
    assert abs(t["W_total"] - to["W_total"]) <= tol_w * max(abs(to["W_total"]), 1e-300)
    assert t["n_pairs"] == to["n_pairs"]
    assert np.array_equal(s.partner_counts(), o.partner_counts(R))
    mg, mo = s.molecule_energies(), o.molecule_terms(R, q)
    scale = np.abs(mo).sum(0).max()
    assert np.abs(mg - mo).max() <= 1e-5 * scale
    return F, tau, t, to


# --------------------------------------------------------------- workloads
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def snapshot(wl, name):
    """Replace the lattice start by the oracle-equilibrated liquid snapshot
    (tests/golden/make_snapshots.py)."""
    z = np.load(os.path.join(GOLDEN, name + ".npz"))
    wl.R, wl.q, wl.v, wl.Lang = z["R"], z["q"], z["v"], z["Lang"]
    return wl


def lj_c0():
    return W.lj_fluid(N=256, rho=0.7, T=1.0, rc=3.5, seed=1)


def water_c1():
    return snapshot(W.water_box(N=1000, rc=14.0, seed=2), "water_N1000")


def ionic_c2():
    return snapshot(W.ionic_solution(seed=3), "ionic_N1040")


# ------------------------------------------------------------- LJ FP64 (C0)
def test_lj_fp64_single_evaluation():
    wl = lj_c0()
    wl.R = wl.R + np.random.default_rng(3).normal(0, 0.03, wl.R.shape)   # off the lattice: F != 0
    s = ms2.System.from_workload(wl, fp64=1)
    o = Oracle.from_workload(wl)
    F, tau = s.forces_torques()
    t = s.energy_terms()
    Fo, _, to = o.forces(wl.R, wl.q)
    assert np.abs(F - Fo).max() <= 1e-12 * np.abs(Fo).max()
    assert abs(t["U_total"] - to["U_total"]) <= 1e-12 * abs(to["U_total"])
    assert abs(t["W_total"] - to["W_total"]) <= 1e-12 * abs(to["W_total"])
    assert np.array_equal(s.partner_counts(), o.partner_counts(wl.R))


def test_lj_fp64_trajectory_100_steps():
    wl = lj_c0()
    s = ms2.System.from_workload(wl, fp64=1)
    s.step(100)
    R, q, v, L, st = s.get_state()
    assert st == 100
    o = Oracle.from_workload(wl)
    Ro, vo, th = o.run_vv(wl.R, wl.v, wl.dt, 100)
    assert np.abs(R - Ro).max() <= 1e-9
    assert np.abs(v - vo).max() <= 1e-9
    U, Wv, T, P = s.energy_virial()
    assert abs(U - th[-1, 0]) <= 1e-9 * abs(th[-1, 0])


# ------------------------------------------------------------ water (C1)
def test_water_rf_full_size_parity():
    wl = water_c1()
    s = ms2.System.from_workload(wl)
    o = Oracle.from_workload(wl)
    compare(s, o, wl.R, wl.q)


def test_water_rf_ragged_tiles():
    """N = 1003 liquid water (no multiple of any tile or block size), rc = 13 A."""
    wl = snapshot(W.water_box(N=1003, rc=13.0, seed=5), "water_N1003")
    s = ms2.System.from_workload(wl)
    compare(s, Oracle.from_workload(wl), wl.R, wl.q)


def test_site_offsets_match_oracle():
    wl = water_box_small()
    s = ms2.System.from_workload(wl)
    off = s.site_offsets()
    o = Oracle.from_workload(wl)
    pos = o.site_positions(wl.R, wl.q)[:, :3] - wl.R[:, None, :]
    assert np.abs(off[:, :3] - pos).max() <= 2e-7


def water_box_small():
    return snapshot(W.water_box(N=216, rc=9.0, seed=9), "water_N216")


def test_water_one_step_matches_oracle():
    wl = water_box_small()
    s = ms2.System.from_workload(wl)
    s.step(1)
    R, q, v, L, _ = s.get_state()
    o = Oracle.from_workload(wl)
    Ro, qo, vo, Lo, th, _ = o.run_leapfrog(wl.R, wl.q, wl.v, wl.Lang, wl.dt, 1, T0=wl.T)
    dR = Ro - wl.R
    assert np.abs((R - wl.R) - dR).max() <= 1e-6 * np.abs(dR).max()
    sgn = np.sign((q * qo).sum(1))[:, None]
    assert np.abs(q * sgn - qo).max() <= 1e-7
    assert rms_rel(v, vo) <= 1e-6
    assert rms_rel(L, Lo) <= 1e-5
    U, Wv, T, P = s.energy_virial()
    assert abs(U - th[0, 0]) <= 1e-6 * abs(th[0, 0])


def test_water_short_trajectory_stays_close():
    """20 NVT steps: trajectories diverge only by the FP32 force rounding."""
    wl = water_box_small()
    s = ms2.System.from_workload(wl)
    s.step(20)
    R, q, v, L, _ = s.get_state()
    o = Oracle.from_workload(wl)
    Ro, qo, vo, Lo, th, _ = o.run_leapfrog(wl.R, wl.q, wl.v, wl.Lang, wl.dt, 20, T0=wl.T)
    assert np.abs(R - Ro).max() <= 1e-4
    U, Wv, T, P = s.energy_virial()
    assert abs(U - th[-1, 0]) <= 1e-4 * abs(th[-1, 0])
    assert T == pytest.approx(th[-1, 2] * 2 / o.ndof() + th[-1, 3] * 2 / o.ndof(), rel=1e-4)


# ----------------------------------------------------------- ionic (C2)
def test_ionic_ewald_full_size_parity():
    wl = ionic_c2()
    s = ms2.System.from_workload(wl)
    o = Oracle.from_workload(wl)
    F, tau, t, to = compare(s, o, wl.R, wl.q, tol_w=W_EWALD)
    for k in ("U_rec", "U_self", "U_intra"):
        assert t[k] == pytest.approx(to[k], rel=1e-6)
    assert t["W_rec"] == pytest.approx(to["W_rec"], rel=1e-5, abs=1e-6 * abs(to["W_total"]))


def test_madelung_on_gpu():
    models = [W.ion(+1.0, 0.0, 0.0, 1.0, "p"), W.ion(-1.0, 0.0, 0.0, 1.0, "m")]
    for m in models:
        m.sites[0].lj = False
    g = np.stack(np.meshgrid(*[np.arange(4)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(float)
    sp = (g.sum(1) % 2).astype(np.int32)
    order = np.argsort(sp, kind="stable")
    R = g[order]
    s = ms2.System(models, [32, 32], 0.0, 1.99, ms2.ELEC_EWALD, box=4.0, reduced=1, lrc=0)
    s.ewald_params(3.0, 20, 20, 20)
    s.set_state(R, np.tile([1.0, 0, 0, 0], (64, 1)), np.zeros((64, 3)), np.zeros((64, 3)))
    U = s.energy_terms()["U_total"]
    assert U / -32.0 == pytest.approx(1.747564594633, rel=2e-6)


# ------------------------------------------------------- Stockmayer (C3)
def test_stockmayer_parity():
    wl = snapshot(W.stockmayer_fluid(N=500, seed=4), "stockmayer_N500")
    s = ms2.System.from_workload(wl)
    compare(s, Oracle.from_workload(wl), wl.R, wl.q)


def test_lj_fp32_leapfrog_parity():
    wl = W.lj_fluid(N=500, rho=0.8, rc=3.5, seed=11)
    wl.R = wl.R + np.random.default_rng(4).normal(0, 0.03, wl.R.shape)   # off the lattice: F != 0
    wl.integrator = 1
    s = ms2.System.from_workload(wl)
    compare(s, Oracle.from_workload(wl), wl.R, wl.q, tol_e=1e-6)


def test_generic_four_site_model_parity():
    """A 4-site water with a massless charge site (TIP4P-like geometry): no
    specialised kernel matches, the generic slot-pattern kernel runs."""
    m = W.water()
    h = m.sites[1].pos
    mpos = (0.0, 0.0, m.sites[0].pos[2] + 0.15)
    m.sites[0].charge = 0.0
    m.sites.append(W.Site(mpos, 0.0, charge=-0.8476))
    wl = water_box_small()
    wl.models = [m]
    s = ms2.System.from_workload(wl)
    compare(s, Oracle.from_workload(wl), wl.R, wl.q)


# -------------------------------------------------------------------- RDF
def rdf_compare(counts, ref, near):
    """Histograms equal except that pairs within rounding of an edge may cross it."""
    assert counts.sum() - ref.sum() in range(-int(near[-1]), int(near[-1]) + 1)
    cg, co = np.concatenate([[0], np.cumsum(counts.sum(0))]), np.concatenate([[0], np.cumsum(ref.sum(0))])
    assert np.all(np.abs(cg - co) <= near)


def test_rdf_counts_match_oracle():
    wl = water_c1()
    s = ms2.System.from_workload(wl)
    s.rdf_setup(14.0, 280)
    s.rdf_sample()
    c, g, ns = s.rdf()
    o = Oracle.from_workload(wl)
    ref = o.rdf_counts(wl.R, wl.q, 14.0, 280)
    near = o.rdf_edge_pairs(wl.R, wl.q, 14.0, 280, 2e-5)
    assert ns == 1 and c.shape == ref.shape
    rdf_compare(c, ref, near)


def test_rdf_mixture_rows_match_oracle():
    wl = ionic_c2()
    s = ms2.System.from_workload(wl)
    s.rdf_setup(14.0, 140)
    s.rdf_sample()
    c, g, _ = s.rdf()
    o = Oracle.from_workload(wl)
    ref = o.rdf_counts(wl.R, wl.q, 14.0, 140)
    near = o.rdf_edge_pairs(wl.R, wl.q, 14.0, 140, 2e-5)
    assert c.shape == ref.shape == (6, 140)
    for row in range(6):
        assert abs(int(c[row].sum()) - int(ref[row].sum())) <= near[-1]
    rdf_compare(c, ref, near)


# ------------------------------------------------- determinism, restart
def test_bitwise_repeatable():
    wl = water_box_small()
    out = []
    for _ in range(2):
        s = ms2.System.from_workload(wl)
        s.step(30)
        out.append(s.get_state()[:4])
        s.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_checkpoint_restart_is_bitwise():
    wl = water_box_small()
    s = ms2.System.from_workload(wl)
    s.step(25)
    ref = s.get_state()[:4]
    s2 = ms2.System.from_workload(wl)
    s2.step(10)
    R, q, v, L, _ = s2.get_state()
    s3 = ms2.System.from_workload(wl, set_state=False)
    s3.set_state(R, q, v, L)
    s3.step(15)
    for a, b in zip(s3.get_state()[:4], ref):
        assert np.array_equal(a, b)


# ------------------------------------------------------------ edge cases
def test_two_molecules_and_no_partners():
    m = W.water()
    s = ms2.System([m], [2], 298.0, 5.0, ms2.ELEC_RF, box=20.0)
    R = np.array([[1.0, 1.0, 1.0], [11.0, 11.0, 11.0]])
    s.set_state(R, np.tile([1.0, 0, 0, 0], (2, 1)), np.zeros((2, 3)), np.zeros((2, 3)))
    F, tau = s.forces_torques()
    assert np.all(F == 0) and np.all(tau == 0)
    assert s.energy_terms()["n_pairs"] == 0
    R[1] = [4.0, 1.0, 1.0]
    s.set_state(R)
    o = Oracle([m], np.zeros(2, np.int32), 20.0, 5.0, elec=1)
    compare(s, o, R, np.tile([1.0, 0, 0, 0], (2, 1)))


def test_invalid_arguments_are_rejected():
    m = W.water()
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        ms2.System([m], [100], 298.0, 20.0, ms2.ELEC_RF, box=30.0)      # rc >= L/2
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        ms2.System([W.cation()], [10], 298.0, 4.0, ms2.ELEC_RF, box=30.0)  # charged + RF
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        ms2.System([m], [10], 298.0, 4.0, ms2.ELEC_RF, box=30.0, rho=0.5)  # box/rho disagree
    s = ms2.System([m], [10], 298.0, 4.0, ms2.ELEC_RF, box=30.0)
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        s.ewald_params(0.3, 8, 8, 8)                                     # not an Ewald system


def test_ionic_ewald_anisotropic_k_range():
    """A k box of different extent per axis (|n| <= 5, 7, 9): the structure-factor
    columns, the nx runs and the generic force kernel, against the oracle."""
    wl = ionic_c2()
    wl.kmax = (5, 7, 9)
    s = ms2.System.from_workload(wl)
    o = Oracle.from_workload(wl)
    F, tau, t, to = compare(s, o, wl.R, wl.q, tol_w=W_EWALD)
    assert t["U_rec"] == pytest.approx(to["U_rec"], rel=1e-6)
    assert t["W_rec"] == pytest.approx(to["W_rec"], rel=1e-5, abs=1e-6 * abs(to["W_total"]))


def test_set_state_is_lazy_and_the_last_state_wins():
    """Two set_state calls in a row (alternating upload buffers): get_state returns
    the second state bit for bit, and stepping it equals a system created on it."""
    wl = water_c1()
    rng = np.random.default_rng(7)
    a = ms2.System.from_workload(wl)
    R2 = wl.R + rng.normal(0, 0.01, wl.R.shape)
    a.set_state(wl.R + 0.05, wl.q, wl.v, wl.Lang)
    a.set_state(R2, wl.q, wl.v, wl.Lang)
    R, q, v, L, _ = a.get_state()
    assert np.array_equal(R, R2) and np.array_equal(q, wl.q) and np.array_equal(v, wl.v)
    wl2 = water_c1()
    wl2.R = R2
    b = ms2.System.from_workload(wl2)
    assert a.energy_virial() == b.energy_virial()  # evaluated on demand
    for s in (a, b):
        s.step(7)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(np.asarray(x), np.asarray(y))
