"""Pins of the FP64 oracle against what the mathematics fixes (CPU only).

Each test ties one part of the oracle to something other than itself: a closed
form, a library routine, a limit, an invariant, or brute force.  A plausible
mistake in the oracle (a dropped term, a wrong sign, index or image, a transposed
operand) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial.transform import Rotation

from oracle import Oracle
from paper_1507_07548_gb300 import workloads as W

IDQ = np.array([1.0, 0.0, 0.0, 0.0])
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def qrot_space(q, axis, angle):
    """q' = (cos(a/2), sin(a/2) e) (x) q : rotate the body by `angle` about the space axis e."""
    e = np.asarray(axis, float) / np.linalg.norm(axis)
    p = np.concatenate([[math.cos(angle / 2)], math.sin(angle / 2) * e])
    w1, x1, y1, z1 = p
    w2, x2, y2, z2 = q
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def scipy_sites(model, R, q):
    """Site positions via scipy's rotation (scalar-last quaternion convention)."""
    rot = Rotation.from_quat([q[1], q[2], q[3], q[0]])
    return np.array([R + rot.apply(np.array(s.pos)) for s in model.sites])


# ---------------------------------------------------------------- rotation
def test_rotation_matches_scipy_and_is_proper():
    rng = np.random.default_rng(11)
    o = Oracle([W.water()], [0], 20.0, 5.0)
    for q in W.random_quaternions(20, rng):
        A = o.rotation(q)
        B = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        assert np.allclose(A, B, atol=1e-14)
        assert np.allclose(A @ A.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(A) - 1) < 1e-14


def test_site_positions_match_scipy():
    rng = np.random.default_rng(12)
    m = W.water()
    R = rng.uniform(0, 10, (5, 3))
    q = W.random_quaternions(5, rng)
    o = Oracle([m], np.zeros(5, np.int32), 20.0, 5.0)
    pos = o.site_positions(R, q)
    for i in range(5):
        assert np.allclose(pos[i, :3], scipy_sites(m, R[i], q[i]), atol=1e-13)


def test_model_body_frames_are_principal():
    for m in [W.water(), W.stockmayer(), W.lj_atom(), W.cation()]:
        P = np.array([s.pos for s in m.sites])
        mass = np.array([s.mass for s in m.sites])
        assert np.allclose((mass[:, None] * P).sum(0), 0, atol=1e-12)
        I = sum(mm * (np.dot(p, p) * np.eye(3) - np.outer(p, p)) for mm, p in zip(mass, P))
        assert np.allclose(I - np.diag(np.diag(I)), 0, atol=1e-12)


# ---------------------------------------------------------------- LJ dimer
@pytest.mark.parametrize("r", [0.95, 2 ** (1 / 6), 1.3, 2.0, 3.0])
def test_lj_dimer_closed_form(r):
    o = Oracle([W.lj_atom()], [0, 0], 20.0, 9.0, reduced=True, lrc=0)
    e = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    R = np.array([[5.0, 5.0, 5.0], 5.0 + r * e])
    F, tau, T = o.forces(R, np.tile(IDQ, (2, 1)))
    assert T["U_total"] == pytest.approx(4 * (r ** -12 - r ** -6), rel=1e-12, abs=1e-14)
    fmag = 24 * (2 * r ** -13 - r ** -7)          # -dU/dr along the separation
    assert np.allclose(F[1], fmag * e, atol=1e-12)
    assert np.allclose(F[0], -F[1], atol=1e-14)
    assert T["W_total"] == pytest.approx(fmag * r, rel=1e-12, abs=1e-12)
    if abs(r - 2 ** (1 / 6)) < 1e-12:
        assert T["U_total"] == pytest.approx(-1.0, rel=1e-13)
        assert np.abs(F).max() < 1e-12


# ------------------------------------------------------ partner search (a2)
@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_partner_counts_equal_bruteforce_images(seed):
    rng = np.random.default_rng(seed)
    N, L = 60, 7.0 + seed
    rc = 0.45 * L
    R = rng.uniform(-2 * L, 3 * L, (N, 3))   # unwrapped coordinates
    o = Oracle([W.lj_atom()], np.zeros(N, np.int32), L, rc, reduced=True)
    shifts = np.array([[a, b, c] for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]) * L
    Rw = R - L * np.floor(R / L)
    cnt = np.zeros(N, int)
    for i in range(N):
        for j in range(N):
            if i == j:
                continue
            d = np.sqrt((((Rw[j] - Rw[i])[None] + shifts) ** 2).sum(1)).min()
            assert abs(d - rc) > 1e-6
            cnt[i] += d < rc
    assert np.array_equal(o.partner_counts(R), cnt)


def test_lattice_threshold_is_exact_ceiling():
    for L, rc in [(31.07, 14.0), (7.1512, 3.5), (10.0, 4.9)]:
        o = Oracle([W.lj_atom()], [0], L, rc, reduced=True)
        T = (rc * 2.0 ** 32 / L) ** 2
        assert o.rc2_lattice() == math.ceil(T)


# ----------------------------------------- min image vs explicit images (a3)
@pytest.mark.parametrize("seed", [5, 6])
def test_water_rf_energy_equals_explicit_image_sum(seed):
    """Tiny box (rc < L/2): the oracle's energy equals a brute-force sum over
    the 27 periodic images of each partner molecule, site positions built with
    scipy's rotation."""
    rng = np.random.default_rng(seed)
    m = W.water()
    N, L, rc = 8, 9.0, 4.4
    R = rng.uniform(0, L, (N, 3))
    q = W.random_quaternions(N, rng)
    o = Oracle([m], np.zeros(N, np.int32), L, rc, elec=1, lrc=0)
    C = o.coulomb
    krf = 1 / (2 * rc ** 3)
    crf = 1 / rc + krf * rc * rc
    sites = [scipy_sites(m, R[i], q[i]) for i in range(N)]
    U = 0.0
    for i in range(N):
        for j in range(i + 1, N):
            for sh in np.array([[a, b, c] for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]) * L:
                dc = R[j] + sh - R[i]
                if np.linalg.norm(dc) >= rc:
                    continue
                for a, sa in enumerate(m.sites):
                    for b, sb in enumerate(m.sites):
                        r = np.linalg.norm(sites[j][b] + sh - sites[i][a])
                        if sa.lj and sb.lj:
                            U += 4 * sa.epsilon * ((sa.sigma / r) ** 12 - (sa.sigma / r) ** 6)
                        U += C * sa.charge * sb.charge * (1 / r + krf * r * r - crf)
    assert o.energy(R, q) == pytest.approx(U, rel=1e-12)


# ------------------------------------------------------- Newton's third law
def small_systems():
    rng = np.random.default_rng(21)
    wl = W.water_box(N=64, rc=6.0, seed=21)
    yield "water_rf", Oracle.from_workload(wl), wl.R, wl.q
    ion = W.ionic_solution(n_water=60, n_ion_pairs=2, rc=6.0, kmax=(6, 6, 6), alpha=0.5, seed=22)
    yield "ionic_ewald", Oracle.from_workload(ion), ion.R, ion.q
    st = W.stockmayer_fluid(N=64, rho=0.012, rc=8.0, seed=23)
    yield "stockmayer_rf", Oracle.from_workload(st), st.R, st.q
    lj = W.lj_fluid(N=108, rho=0.7, rc=2.5)
    yield "lj", Oracle.from_workload(lj), lj.R + rng.normal(0, 0.05, lj.R.shape), lj.q


@pytest.mark.parametrize("name,o,R,q", list(small_systems()), ids=lambda x: x if isinstance(x, str) else "")
def test_total_force_vanishes(name, o, R, q):
    F, tau, T = o.forces(R, q)
    assert np.abs(F.sum(0)).max() <= 1e-11 * np.abs(F).max() * len(F)


def test_isolated_cluster_conserves_angular_momentum():
    """All molecules within rc of each other, box much larger: sum(R x F + tau) = 0."""
    rng = np.random.default_rng(31)
    for models, sp, elec in [([W.water()], [0] * 6, 1), ([W.stockmayer()], [0] * 6, 1)]:
        R = 20.0 + rng.uniform(-3, 3, (6, 3))
        q = W.random_quaternions(6, rng)
        o = Oracle(models, np.array(sp, np.int32), 60.0, 25.0, elec=elec, lrc=0)
        F, tau, _ = o.forces(R, q)
        tot = np.cross(R, F).sum(0) + tau.sum(0)
        assert np.abs(tot).max() < 1e-10 * np.abs(tau).max() * 10


# ------------------------------------------------ finite differences of U
def fd_check(o, R, q, idx, h=1e-5, ang=1e-6):
    F, tau, _ = o.forces(R, q)
    for i in idx:
        for k in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[i, k] += h
            Rm[i, k] -= h
            fd = -(o.energy(Rp, q) - o.energy(Rm, q)) / (2 * h)
            assert fd == pytest.approx(F[i, k], rel=1e-6, abs=1e-6 * np.abs(F).max())
            e = np.eye(3)[k]
            qp, qm = q.copy(), q.copy()
            qp[i] = qrot_space(q[i], e, ang)
            qm[i] = qrot_space(q[i], e, -ang)
            if np.allclose(q[i], qp[i]):
                continue
            fdt = -(o.energy(R, qp) - o.energy(R, qm)) / (2 * ang)
            assert fdt == pytest.approx(tau[i, k], rel=1e-5, abs=1e-5 * np.abs(tau).max() + 1e-9)


@pytest.mark.parametrize("name,o,R,q", list(small_systems()), ids=lambda x: x if isinstance(x, str) else "")
def test_forces_torques_are_minus_gradient(name, o, R, q):
    fd_check(o, R, q, idx=[0, 5, 17])


@pytest.mark.parametrize("name,o,R,q", list(small_systems()), ids=lambda x: x if isinstance(x, str) else "")
def test_virial_is_minus_volume_derivative(name, o, R, q):
    """W = -dU/ds with centres and box edge scaled by s, orientations fixed."""
    s = o.s
    L0, h = s.L, 1e-6
    _, _, T = o.forces(R, q)

    def U(scale):
        s.L = L0 * scale
        try:
            t = o.forces(R * scale, q)[2]
        finally:
            s.L = L0
        return t["U_total"] - t["U_lrc"]

    fd = -(U(1 + h) - U(1 - h)) / (2 * h)
    assert fd == pytest.approx(T["W_total"], rel=1e-6, abs=1e-7 * abs(T["U_total"]))


@pytest.mark.parametrize("name,o,R,q", list(small_systems()), ids=lambda x: x if isinstance(x, str) else "")
def test_virial_owner_shares_add_up_to_the_molecular_virial(name, o, R, q):
    """The per-molecule owner shares 1/2 (sum_j sum_ab -r_ab.f_ab - 2 sum_a s_ia.F_ia)
    add up to the pair-form W_pair, itself pinned by the volume derivative above."""
    _, _, T = o.forces(R, q)
    mol = o.molecule_terms(R, q)
    assert mol[:, 3].sum() == pytest.approx(T["W_pair"], rel=1e-11, abs=1e-11 * abs(T["U_total"]))
    for k, key in enumerate(("U_lj", "U_qq", "U_dd")):
        assert mol[:, k].sum() == pytest.approx(T[key], rel=1e-11, abs=1e-11 * abs(T["U_total"]))


def test_virial_owner_share_of_point_molecules_is_the_pair_share():
    """Without site offsets the owner share is 1/2 sum_j (R_i - R_j).F_ij: checked
    against a brute-force LJ sum over minimum images."""
    wl = W.lj_fluid(N=108, rho=0.5, T=1.0, rc=2.5, seed=3)
    wl.R = wl.R + np.random.default_rng(5).normal(0, 0.05, wl.R.shape)
    o = Oracle.from_workload(wl)
    mol = o.molecule_terms(wl.R, wl.q)
    L = wl.L
    want = np.zeros(wl.N)
    for i in range(wl.N):
        d = wl.R - wl.R[i]
        d -= L * np.rint(d / L)
        r2 = (d * d).sum(1)
        m = (r2 < wl.rc ** 2) & (np.arange(wl.N) != i)
        sr6 = (1.0 / r2[m]) ** 3
        # force on i from j: 24 (2 sr^12 - sr^6) / r^2 * (R_i - R_j); virial (R_i - R_j).F
        want[i] = 0.5 * (24.0 * (2.0 * sr6 * sr6 - sr6)).sum()
    assert np.abs(mol[:, 3] - want).max() <= 1e-12 * np.abs(want).max()


# ------------------------------------------------------------ reaction field
def test_rf_shift_invariance_for_neutral_molecules():
    wl = W.water_box(N=64, rc=6.0, seed=41)
    o = Oracle.from_workload(wl)
    U0 = o.forces(wl.R, wl.q)[2]
    o.s.crf_shift = 0.37
    U1 = o.forces(wl.R, wl.q)[2]
    assert U1["U_qq"] == pytest.approx(U0["U_qq"], rel=1e-12)
    assert U1["W_total"] == pytest.approx(U0["W_total"], rel=1e-12)


def test_point_dipole_is_limit_of_charge_pairs():
    """Dipole-dipole energy (with its reaction-field term) equals the d -> 0 limit
    of two molecules carrying charges +-mu/d at +-d/2 on the dipole axis."""
    rng = np.random.default_rng(51)
    mu = 0.41639

    def model(d):
        m = W.stockmayer()
        m.sites = m.sites[:2]
        if d is None:
            m.sites.append(W.Site((0, 0, 0), 0.0, dipole=(0.0, 0.0, mu)))
        else:
            m.sites.append(W.Site((0, 0, d / 2), 0.0, charge=mu / d))
            m.sites.append(W.Site((0, 0, -d / 2), 0.0, charge=-mu / d))
        for s in m.sites:
            s.epsilon = 0.0
        return m

    R = np.array([[10.0, 10.0, 10.0], [13.1, 11.2, 9.4]])
    q = W.random_quaternions(2, rng)
    ref = Oracle([model(None)], [0, 0], 40.0, 12.0, elec=1, lrc=0).forces(R, q)
    vals = []
    for d in (2e-3, 1e-3):
        vals.append(Oracle([model(d)], [0, 0], 40.0, 12.0, elec=1, lrc=0).forces(R, q))
    # error of the charge pair is O(d^2): Richardson-extrapolate the two
    Ux = (4 * vals[1][2]["U_qq"] - vals[0][2]["U_qq"]) / 3
    assert Ux == pytest.approx(ref[2]["U_dd"], rel=1e-7)
    Fx = (4 * vals[1][0] - vals[0][0]) / 3
    Tx = (4 * vals[1][1] - vals[0][1]) / 3
    assert np.allclose(Fx, ref[0], rtol=1e-6, atol=1e-7 * np.abs(ref[0]).max())
    assert np.allclose(Tx, ref[1], rtol=1e-6, atol=1e-7 * np.abs(ref[1]).max())


# ------------------------------------------------------------------- Ewald
def nacl(n_cells=2):
    m = 2 * n_cells
    g = np.stack(np.meshgrid(*[np.arange(m)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(float)
    sp = (g.sum(1) % 2).astype(np.int32)
    models = [W.ion(+1.0, 0.0, 0.0, 1.0, "p"), W.ion(-1.0, 0.0, 0.0, 1.0, "m")]
    for mm in models:
        mm.sites[0].lj = False
    return models, sp, g, float(m)


@pytest.mark.parametrize("alpha,kmax", [(3.0, 20), (3.5, 24), (4.0, 30)])
def test_madelung_constant_rock_salt(alpha, kmax):
    """NaCl, nearest-neighbour distance 1, unit charges: U = -(N/2) * 1.747564594633."""
    models, sp, R, L = nacl()
    o = Oracle(models, sp, L, 0.499 * L, elec=2, alpha=alpha, kmax=(kmax,) * 3, reduced=True, lrc=0)
    F, _, T = o.forces(R, np.tile(IDQ, (len(sp), 1)))
    assert T["U_total"] / (-len(sp) / 2) == pytest.approx(1.747564594633, rel=1e-11)
    assert np.abs(F).max() < 1e-12


def test_ewald_equals_spherical_direct_sum_plus_surface_term():
    """de Leeuw-Perram-Smith: the direct Coulomb sum over images in growing
    spheres tends to U_Ewald(tin-foil) + 2 pi C |M|^2 / (3 V)."""
    rng = np.random.default_rng(61)
    L = 5.0
    pos = rng.uniform(0, L, (4, 3))
    qs = np.array([1.0, -1.0, 0.5, -0.5])
    mods = [W.ion(c, 0, 0, 1.0, "x") for c in qs]
    for mm in mods:
        mm.sites[0].lj = False
    o = Oracle(mods, np.arange(4, dtype=np.int32), L, 2.45, elec=2, alpha=2.0, kmax=(14,) * 3, reduced=True, lrc=0)
    Ue = o.forces(pos, np.tile(IDQ, (4, 1)))[2]["U_total"]
    M = (qs[:, None] * pos).sum(0)
    target = Ue + 2 * np.pi * (M @ M) / (3 * L ** 3)
    nmax = 30
    n = np.stack(np.meshgrid(*[np.arange(-nmax, nmax + 1)] * 3, indexing="ij"), -1).reshape(-1, 3)
    n = n[(n * n).sum(1) <= nmax * nmax]
    U = 0.0
    for a in range(4):
        for b in range(4):
            r = np.sqrt(((pos[b] - pos[a] + n * L) ** 2).sum(1))
            U += 0.5 * qs[a] * qs[b] * (1 / r[r > 0]).sum()
    assert U == pytest.approx(target, rel=2e-6)


def test_ewald_total_independent_of_alpha():
    wl = W.ionic_solution(n_water=100, n_ion_pairs=2, rc=7.0, seed=71)
    L = (len(wl.species) / W.WATER_NUMBER_DENSITY) ** (1 / 3)
    assert abs(L - wl.L) < 1e-12 and wl.L > 14.0
    res = []
    for alpha, kmax in [(1.2, 36), (1.5, 44)]:
        o = Oracle.from_workload(wl, alpha=alpha, kmax=(kmax,) * 3, lrc=0)
        res.append(o.forces(wl.R, wl.q))
    U0, U1 = res[0][2]["U_total"], res[1][2]["U_total"]
    assert U1 == pytest.approx(U0, rel=1e-9)
    F0, F1 = res[0][0], res[1][0]
    assert np.sqrt(((F1 - F0) ** 2).sum() / (F0 ** 2).sum()) < 1e-8
    T0, T1 = res[0][1], res[1][1]
    assert np.sqrt(((T1 - T0) ** 2).sum() / (T0 ** 2).sum()) < 1e-8


def test_ewald_reciprocal_site_forces_sum_to_zero():
    wl = W.ionic_solution(n_water=60, n_ion_pairs=2, rc=6.0, kmax=(6, 6, 6), alpha=0.5, seed=81)
    o = Oracle.from_workload(wl)
    fs, U, Wat = o.ewald_reciprocal(wl.R, wl.q)
    assert np.abs(fs.reshape(-1, 3).sum(0)).max() < 1e-11 * np.abs(fs).max() * fs.shape[0]
    assert U > 0


def test_ewald_constants_closed_forms():
    """Self term -C alpha/sqrt(pi) sum q^2; intramolecular erf term for water
    computed from the three site distances; background vanishes when neutral."""
    wl = W.ionic_solution(n_water=10, n_ion_pairs=1, rc=5.0, seed=91)
    o = Oracle.from_workload(wl)
    us, ui, ub = o.ewald_constants()
    m = W.water()
    qs = [s.charge for s in m.sites]
    C, a = o.coulomb, wl.alpha
    assert us == pytest.approx(-C * a / math.sqrt(math.pi) * (10 * sum(x * x for x in qs) + 2.0), rel=1e-14)
    P = [np.array(s.pos) for s in m.sites]
    rOH, rHH = np.linalg.norm(P[1] - P[0]), np.linalg.norm(P[2] - P[1])
    assert rOH == pytest.approx(1.0, rel=1e-14)
    assert rHH == pytest.approx(2 * math.sin(math.radians(109.47) / 2), rel=1e-14)
    intra = 2 * qs[0] * qs[1] * math.erf(a * rOH) / rOH + qs[1] * qs[2] * math.erf(a * rHH) / rHH
    assert ui == pytest.approx(-C * 10 * intra, rel=1e-13)
    assert ub == 0.0


# --------------------------------------------------------------------- LRC
def test_lj_lrc_matches_quadrature():
    wl = W.ionic_solution(n_water=30, n_ion_pairs=2, rc=5.0, seed=101)
    o = Oracle.from_workload(wl)
    U, P = o.lrc()
    kinds = []
    for k, m in enumerate(wl.models):
        n = int((wl.species == k).sum())
        kinds += [(n, s.sigma, s.epsilon) for s in m.sites if s.lj]
    V, rc = wl.L ** 3, wl.rc
    u_ref = p_ref = 0.0
    for na, sa, ea in kinds:
        for nb, sb, eb in kinds:
            sg, ep = 0.5 * (sa + sb), math.sqrt(ea * eb)
            u = lambda r: 4 * ep * ((sg / r) ** 12 - (sg / r) ** 6)
            du = lambda r: 4 * ep * (-12 * sg ** 12 / r ** 13 + 6 * sg ** 6 / r ** 7)
            u_ref += na * nb * integrate.quad(lambda r: r * r * u(r), rc, np.inf, epsabs=0, epsrel=1e-13)[0]
            p_ref += na * nb * integrate.quad(lambda r: r ** 3 * du(r), rc, np.inf, epsabs=0, epsrel=1e-13)[0]
    assert U == pytest.approx(2 * math.pi / V * u_ref, rel=1e-10)
    assert P == pytest.approx(-2 * math.pi / (3 * V * V) * p_ref, rel=1e-10)


# --------------------------------------------------------------- integrators
def lj_cluster(n=13, seed=111):
    """Cluster inside a box far larger than its extent, every pair within rc:
    the potential is smooth along the trajectory."""
    rng = np.random.default_rng(seed)
    R = 20.0 + W.fcc_lattice(2, 2 * 2 ** (1 / 6) * math.sqrt(2))[:n] + rng.normal(0, 0.05, (n, 3))
    v = rng.normal(0, 0.3, (n, 3))
    v -= v.mean(0)
    return Oracle([W.lj_atom()], np.zeros(n, np.int32), 60.0, 25.0, reduced=True, lrc=0), R, v


def test_velocity_verlet_energy_error_scales_as_dt2():
    o, R, v = lj_cluster()
    amp = []
    for dt in (0.004, 0.002):
        n = int(round(2.0 / dt))
        _, _, th = o.run_vv(R, v, dt, n)
        E = th[:, 0] + th[:, 2]
        amp.append(E.max() - E.min())
    assert 3.5 < amp[0] / amp[1] < 4.5


def test_velocity_verlet_no_secular_drift():
    o, R, v = lj_cluster()
    _, _, th = o.run_vv(R, v, 0.003, 10000)
    E = th[:, 0] + th[:, 2]
    amp = E.max() - E.min()
    assert amp / abs(E[0]) < 1e-3
    k = len(E) // 3
    assert abs(E[-k:].mean() - E[k:2 * k].mean()) < 0.05 * amp


def test_velocity_verlet_time_reversible():
    o, R, v = lj_cluster()
    R1, v1, _ = o.run_vv(R, v, 0.003, 400, thermo=False)
    R2, v2, _ = o.run_vv(R1, -v1, 0.003, 400, thermo=False)
    assert np.abs(R2 - R).max() < 1e-10
    assert np.abs(v2 + v).max() < 1e-10


def test_leapfrog_rigid_time_reversible():
    """Leapfrog state (R, q, v(t-dt/2), L(t-dt/2)): after n steps, one more
    kick gives v(t+dt/2); negating it and stepping n times returns R, q."""
    rng = np.random.default_rng(121)
    n = 5
    R = 30.0 + rng.uniform(-3.5, 3.5, (n, 3))
    q = W.random_quaternions(n, rng)
    o = Oracle([W.water()], np.zeros(n, np.int32), 60.0, 25.0, elec=1, lrc=0)
    v, Ls = W.thermal_velocities(o.models, o.species, q, 300.0, o.kconv, rng)
    dt, steps = 0.5, 200
    R1, q1, v1, L1, _, _ = o.run_leapfrog(R, q, v, Ls, dt, steps, n_iter=40, thermo=False)
    F, tau, _ = o.forces(R1, q1)
    M = W.water().mass
    vh = v1 + dt * o.kconv * F / M
    Lh = L1 + dt * o.kconv * tau
    R2, q2, _, _, _, _ = o.run_leapfrog(R1, q1, -vh, -Lh, dt, steps, n_iter=40, thermo=False)
    assert np.abs(R2 - R).max() < 1e-8
    sgn = np.sign((q2 * q).sum(1))[:, None]
    assert np.abs(q2 * sgn - q).max() < 1e-8


def test_leapfrog_rigid_water_nve_energy_error_scales_as_dt2():
    """Rigid leapfrog with the quaternion midpoint rule, NVE, on an isolated
    cluster of 8 waters taken from the liquid snapshot (no pair crosses the
    cut-off, so the energy is smooth).  The total energy at integer times -- U
    of (R_k, q_k) plus the kinetic energy of the half-step means of v and L at
    q_k -- fluctuates boundedly, its fluctuation falls ~4x when dt is halved over
    the same span, and it does not drift.  A wrong coupling of the torque into
    the rotation (an axis, a sign, a factor) breaks this at O(1)."""
    z = np.load(os.path.join(GOLDEN, "water_N216.npz"))
    L216 = W.water_box(N=216, rc=9.0, seed=9).L
    d = z["R"] - z["R"][0]
    d -= L216 * np.rint(d / L216)
    near = np.argsort((d * d).sum(1))[:8]
    R0, q0 = 30.0 + d[near], z["q"][near]
    rng = np.random.default_rng(43)
    models, sp = [W.water()], np.zeros(8, np.int32)
    o = Oracle(models, sp, 60.0, 25.0, elec=1, lrc=0)
    v0, L0 = W.thermal_velocities(models, sp, q0, 150.0, o.s.kconv, rng)

    def energies(dt, span):
        st = [(R0, q0, v0, L0)]
        R, q, v, Lg = R0, q0, v0, L0
        for _ in range(int(round(span / dt)) + 1):
            R, q, v, Lg, _, _ = o.run_leapfrog(R, q, v, Lg, dt, 1, T0=0.0, thermo=False)
            st.append((R, q, v, Lg))
        E = []
        for k in range(1, len(st) - 1):   # state k: R_k, q_k, v_{k-1/2}, L_{k-1/2}
            Rk, qk = st[k][0], st[k][1]
            vk, Lk = 0.5 * (st[k][2] + st[k + 1][2]), 0.5 * (st[k][3] + st[k + 1][3])
            E.append(o.energy(Rk, qk) + o.kinetic(qk, vk, Lk).sum())
        return np.array(E)

    e1, e2 = energies(1.0, 200.0), energies(0.5, 200.0)
    f1, f2 = np.ptp(e1), np.ptp(e2)
    assert f2 < 2e-3 * abs(e2.mean())                 # bounded
    assert 3.3 < f1 / f2 < 4.8, (f1, f2)              # ~dt^2
    q = len(e2) // 4                                  # no secular drift
    assert abs(e2[-q:].mean() - e2[:q].mean()) < 0.25 * f2


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_free_rotor_about_principal_axis(axis):
    """No torque, L along principal axis k, omega = |L| / I_k.  The implicit
    midpoint map (solved to convergence) turns the body about that axis by
    exactly 4 atan(omega dt / 4) per step (Cayley transform); the default three
    sweeps stay within 1e-7 of it, and both approach the exact rotation by
    omega t as dt^2.  L stays constant and |q| = 1."""
    m = W.water()
    I = W.principal_moments(m)
    rng = np.random.default_rng(131 + axis)
    q0 = W.random_quaternions(1, rng)[0]
    A = Rotation.from_quat([q0[1], q0[2], q0[3], q0[0]]).as_matrix()
    om = 0.02
    Ls = (A[:, axis] * om * I[axis])[None]
    o = Oracle([m], np.array([0], np.int32), 60.0, 25.0, elec=1, lrc=0)
    R = np.full((1, 3), 30.0)

    def run(dt, steps, n_iter):
        _, q1, _, L1, th, _ = o.run_leapfrog(R, q0[None], np.zeros((1, 3)), Ls, dt, steps, n_iter=n_iter)
        assert np.array_equal(L1, Ls)
        assert abs(np.linalg.norm(q1[0]) - 1) < 1e-14
        ke = th[:, 3]
        assert np.abs(ke - 0.5 * (om * I[axis]) ** 2 / I[axis] / o.kconv).max() < 1e-9 * ke[0]
        return q1[0]

    def dist(a, b):
        return min(np.abs(a - b).max(), np.abs(a + b).max())

    dt, steps = 1.0, 300
    q_conv = run(dt, steps, 40)
    assert dist(q_conv, qrot_space(q0, A[:, axis], steps * 4 * math.atan(om * dt / 4))) < 1e-12
    assert dist(run(dt, steps, 3), q_conv) < 1e-7
    e1 = dist(run(dt, steps, 40), qrot_space(q0, A[:, axis], om * dt * steps))
    e2 = dist(run(dt / 2, 2 * steps, 40), qrot_space(q0, A[:, axis], om * dt * steps))
    assert 3.9 < e1 / e2 < 4.1


def test_linear_rotor_precesses_uniformly():
    """Linear molecule with L perpendicular to its axis: the axis turns about L,
    by 4 atan(omega dt / 4) per step of the converged midpoint map."""
    m = W.stockmayer()
    I = W.principal_moments(m)
    assert I[2] < 1e-12 and abs(I[0] - I[1]) < 1e-12
    q0 = np.array([1.0, 0, 0, 0])
    om, dt, steps = 0.01, 2.0, 100
    Ls = np.array([[I[0] * om, 0.0, 0.0]])
    o = Oracle([m], np.array([0], np.int32), 60.0, 25.0, elec=1, lrc=0)
    _, q1, _, _, _, _ = o.run_leapfrog(np.full((1, 3), 30.0), q0[None], np.zeros((1, 3)), Ls, dt, steps, n_iter=40)
    axis = Rotation.from_quat([q1[0, 1], q1[0, 2], q1[0, 3], q1[0, 0]]).apply([0, 0, 1.0])
    ang = steps * 4 * math.atan(om * dt / 4)
    assert np.allclose(axis, [0, -math.sin(ang), math.cos(ang)], atol=1e-12)


def test_thermostat_sets_temperature_exactly():
    wl = W.water_box(N=64, rc=6.0, seed=141)
    o = Oracle.from_workload(wl)
    *_, ts = o.run_leapfrog(wl.R, wl.q, wl.v, wl.Lang, 1.0, 5, T0=298.0)
    assert np.allclose(ts, 298.0, rtol=1e-13)


def test_initial_velocities_have_requested_temperature():
    wl = W.water_box(N=64, rc=6.0, seed=151)
    o = Oracle.from_workload(wl)
    ke = o.kinetic(wl.q, wl.v, wl.Lang)
    assert 2 * ke.sum() / o.ndof() == pytest.approx(298.0, rel=1e-12)
    assert o.ndof() == 6 * 64 - 3


# --------------------------------------------------------------------- RDF
def test_rdf_counts_equal_bruteforce_and_ideal_gas():
    rng = np.random.default_rng(161)
    N, L = 400, 12.0
    m = W.lj_atom()
    m.sites[0].epsilon = 0.0     # dummy LJ sites: ideal gas
    R = rng.uniform(0, L, (N, 3))
    o = Oracle([m], np.zeros(N, np.int32), L, 5.9, reduced=True)
    r_max, nb = 5.9, 59
    c = o.rdf_counts(R, np.tile(IDQ, (N, 1)), r_max, nb)[0]
    i, j = np.triu_indices(N, 1)
    d = R[j] - R[i]
    d -= L * np.rint(d / L)
    r = np.sqrt((d ** 2).sum(1))
    r = r[r < r_max]
    ref = np.bincount(np.floor(r / (r_max / nb)).astype(int), minlength=nb)[:nb]
    assert np.array_equal(c, ref)
    edges = np.arange(nb + 1) * r_max / nb
    expect = N * (N - 1) / 2 * 4 * np.pi / 3 * (edges[1:] ** 3 - edges[:-1] ** 3) / L ** 3
    g = c / expect
    tail = slice(20, nb)
    assert abs(g[tail].mean() - 1) < 3 / math.sqrt(c[tail].sum())


def test_rdf_kind_pairs_for_mixture():
    wl = W.ionic_solution(n_water=30, n_ion_pairs=2, rc=5.0, seed=171)
    o = Oracle.from_workload(wl)
    T, k = o.rdf_kinds()
    assert T == 3                                # O, cation, anion
    c = o.rdf_counts(wl.R, wl.q, 5.0, 50)
    assert c.shape == (6, 50)
    # total unordered LJ-site pairs within r_max, counted by brute force
    pos = o.site_positions(wl.R, wl.q)[:, 0]
    i, j = np.triu_indices(len(pos), 1)
    d = pos[j] - pos[i]
    d -= wl.L * np.rint(d / wl.L)
    r = np.sqrt((d ** 2).sum(1))
    assert c.sum() == int((r < 5.0).sum())


# ------------------------------------------------- Massieu derivatives (Eq. 1)
def _volume_cases():
    wl = W.water_box(N=64, rc=6.0, seed=21)
    yield "water_rf", Oracle.from_workload(wl), wl.R, wl.q
    lj = W.lj_fluid(N=108, rho=0.7, rc=2.5)
    R = lj.R + np.random.default_rng(9).normal(0, 0.05, lj.R.shape)
    yield "lj", Oracle.from_workload(lj), R, lj.q


@pytest.mark.parametrize("name,o,R,q", list(_volume_cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_volume_derivatives_are_finite_differences_of_U(name, o, R, q):
    """dU/dV and d2U/dV2 at fixed scaled centres and orientations against central
    differences of U(s) with centres and box edge scaled by s (V = s^3 V0); the
    long-range parts are -P_LRC and 2 P_LRC / V."""
    s = o.s
    L0, h = s.L, 5e-6
    V = L0 ** 3
    # no centre pair so close to the cutoff that the scaling moves it across
    d = R[:, None, :] - R[None, :, :]
    d -= L0 * np.rint(d / L0)
    r = np.sqrt((d * d).sum(-1))
    assert np.min(np.abs(r - s.rc)) > 10 * h * s.rc

    def U(scale):
        s.L = L0 * scale
        try:
            t = o.forces(R * scale, q)[2]
        finally:
            s.L = L0
        return t["U_total"] - t["U_lrc"]

    up, u0, um = U(1 + h), U(1.0), U(1 - h)
    d1, d2 = (up - um) / (2 * h), (up - 2 * u0 + um) / h ** 2
    UV, UVV = o.volume_derivatives(R, q)
    Pl = o.forces(R, q)[2]["P_lrc"]
    assert UV + Pl == pytest.approx(d1 / (3 * V), rel=1e-7)
    assert UVV - 2 * Pl / V == pytest.approx((d2 - 2 * d1) / (9 * V * V), rel=1e-5)


def test_massieu_estimators_are_derivatives_of_the_exact_partition_function():
    """Two particles in a periodic box with the smooth pair potential
    u = eps exp(-(r/a)^2) (negligible at rc < L/2): Z_c / V^2 = 1 + B(beta) / V with
    B = int_0^rc 4 pi r^2 (exp(-beta u) - 1) dr, so A^r = -(1/2) ln(1 + rho B / 2)
    differentiates exactly; the canonical moments that feed the estimators are
    quadratures over the same weights."""
    sympy = pytest.importorskip("sympy")
    eps, a, rc, L, beta = 1.3, 0.5, 3.5, 8.0, 0.7
    V, N = L ** 3, 2
    x, w = np.polynomial.legendre.leggauss(400)
    r = 0.5 * rc * (x + 1)
    w = 0.5 * rc * w * 4 * np.pi * r ** 2
    u = eps * np.exp(-(r / a) ** 2)
    u1 = -2 * r / a ** 2 * u                      # u'
    u2 = (4 * r ** 2 / a ** 4 - 2 / a ** 2) * u   # u''
    e = np.exp(-beta * u)
    # centres scale with V: U_V = u' r / (3V), U_VV = (u'' r^2 - 2 u' r) / (9 V^2)
    UV = u1 * r / (3 * V)
    UVV = (u2 * r * r - 2 * u1 * r) / (9 * V * V)
    wout = V - 4 / 3 * np.pi * rc ** 3           # the rest of the cell: u = 0
    U0, V0 = 0.1, -0.002                          # arbitrary shifts
    X, Y = u - U0, UV - V0
    ww = w * e
    acc = [ww.sum() + wout]
    for f in (X, X ** 2, X ** 3, Y, Y ** 2, X * Y, X * X * Y, X * Y * Y, UVV, X * UVV):
        acc.append((ww * f).sum())
    xo, yo = -U0, -V0                             # the outer region's shifted values
    for k, f in enumerate((xo, xo ** 2, xo ** 3, yo, yo ** 2, xo * yo, xo * xo * yo, xo * yo * yo, 0.0, 0.0)):
        acc[k + 1] += wout * f
    got = Oracle.massieu(np.array(acc), U0, V0, beta, V, N)
    # exact: f(beta, rho) = -(1/2) ln(1 + rho B(beta) / 2)
    b, rho = sympy.symbols("b rho")
    Bf = sympy.Function("B")
    f = -sympy.Rational(1, 2) * sympy.log(1 + rho * Bf(b) / 2)
    vals = {rho: N / V}
    Bk = [(w * (e - 1)).sum()] + [(w * (-u) ** k * e).sum() for k in (1, 2, 3)]   # B and its beta-derivatives
    want = []
    for m, nn in ((1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (3, 0), (2, 1), (1, 2)):
        expr = sympy.diff(f, b, m, rho, nn) if nn else sympy.diff(f, b, m)
        expr = expr * b ** m * rho ** nn
        for k in (3, 2, 1):
            expr = expr.subs(sympy.Derivative(Bf(b), (b, k)), Bk[k])
        expr = expr.subs(Bf(b), Bk[0]).subs(vals).subs(b, beta)
        want.append(float(expr))
    np.testing.assert_allclose(got, want, rtol=1e-8, atol=1e-14)


# ------------------------------------------ Green-Kubo conductivity (Eqs. 3-4)
def test_current_counts_net_charges_only():
    wl = W.ionic_solution(n_water=30, n_ion_pairs=3, rc=5.0, seed=6)
    o = Oracle.from_workload(wl)
    v = np.zeros_like(wl.v)
    assert np.allclose(o.current(v + np.array([0.3, -0.1, 0.2])), 0.0, atol=1e-15)  # neutral overall: no current
    k = int(np.nonzero(wl.species == 1)[0][0])                                      # one cation alone
    v[k] = [1.0, 2.0, -3.0]
    np.testing.assert_allclose(o.current(v), [1.0, 2.0, -3.0], rtol=1e-15)
    v[:] = 0.0
    v[wl.species == 0] = 5.0                                                         # water carries no current
    assert np.allclose(o.current(v), 0.0, atol=1e-12)


def test_flux_acf_of_a_rotating_current_is_a_cosine():
    """j(t) = A (cos w t, sin w t, 0): j(t).j(t - m) = A^2 cos(w m dt) for every origin."""
    A, w, dt, n, M = 1.7, 0.31, 0.5, 300, 40
    t = np.arange(n) * dt
    j = A * np.stack([np.cos(w * t), np.sin(w * t), np.zeros(n)], 1)
    acf = Oracle.flux_acf(j, M)
    np.testing.assert_allclose(acf, A * A * np.cos(w * np.arange(M) * dt), rtol=1e-12, atol=1e-13)
    assert Oracle.flux_acf(j[:10], 20)[10:].max() == 0.0     # lags beyond the series stay empty


def test_conductivity_units_and_rule():
    """A constant ACF c over M lags integrates to c (M-1) dt; 1 (e A/fs)^2 fs over
    3 V kB T with V = 1000 A^3, T = 300 K is e^2 1e-5 / (3e-27 kB 300) S/m."""
    acf = np.full(11, 2.0)
    got = Oracle.conductivity(acf, 0.5, 1000.0, 300.0)
    e, kB = 1.602176634e-19, 1.380649e-23
    assert got == pytest.approx(2.0 * 10 * 0.5 * e * e * 1e-5 / (3 * 1000e-30 * kB * 300.0), rel=1e-14)
    cos_acf = np.cos(0.2 * np.arange(50))
    assert Oracle.conductivity(cos_acf, 1.0, 1.0, 1.0, reduced=True) == pytest.approx(
        np.trapezoid(cos_acf) / 3.0, rel=1e-14)


# -------------------------------------------- residence time (Eq. 7, Impey)
def _two_species_line():
    """One centre (species 0) at the origin and four shell molecules (species 1)
    on a line, far from the box edges; a scripted trajectory moves them."""
    models = [W.ion(1.0, 2.35, 65.0, 22.99, "c"), W.ion(-1.0, 4.40, 50.0, 35.45, "a")]
    sp = np.array([0, 1, 1, 1, 1], np.int32)
    o = Oracle(models, sp, 40.0, 10.0, elec=0, lrc=0)
    return o


def test_residence_of_a_static_shell_is_one():
    o = _two_species_line()
    R = np.array([[20.0, 20, 20], [22.0, 20, 20], [20, 22.5, 20], [20, 20, 17.0], [29.0, 20, 20]])
    corr, nsol = o.residence(np.repeat(R[None], 12, 0), 0, 1, 4.0, 0, 6)
    np.testing.assert_allclose(corr, 1.0)
    assert nsol == 3.0


def test_residence_departures_and_impey_tolerance():
    """Molecule 1 leaves at sample 3 for good; molecule 2 steps out for exactly two
    samples (4, 5) and returns; molecule 3 stays; molecule 4 is never in the shell."""
    o = _two_species_line()
    T = 8
    R = np.zeros((T, 5, 3)) + 20.0
    for t in range(T):
        R[t, 1] = [22.0 if t < 3 else 30.0, 20, 20]
        R[t, 2] = [20, 30.0 if t in (4, 5) else 22.0, 20]
        R[t, 3] = [20, 20, 17.0]
        R[t, 4] = [35.0, 20, 20]
    corr2, nsol = o.residence(R, 0, 1, 4.0, 2, T)
    corr1, _ = o.residence(R, 0, 1, 4.0, 1, T)
    # lag 7 has only origin 0 (members 1, 2, 3): molecule 1 is gone; molecule 2's
    # two-sample excursion is tolerated with t* = 2 but not with t* = 1
    assert corr2[7] == pytest.approx(2.0 / 3.0)
    assert corr1[7] == pytest.approx(1.0 / 3.0)
    assert corr2[0] == 1.0
    # lag 1, by hand: members(t0) that are inside again at t0 + 1, over origins 0..6
    inside = {t: [k for k in (1, 2, 3) if (k != 1 or t < 3) and (k != 2 or t not in (4, 5))] for t in range(T)}
    frac = [len([k for k in inside[t] if k in inside[t + 1]]) / len(inside[t]) for t in range(T - 1)]
    assert corr2[1] == pytest.approx(np.mean(frac))
    assert nsol == pytest.approx(np.mean([len(inside[t]) for t in range(T)]))


# --------------------------------------- thermal conductivity (Eqs. 5-6)
def test_heat_flux_is_the_time_derivative_of_the_energy_moment():
    """Without the enthalpy term, J_q = d/dt sum_k R_k E_k for Newtonian dynamics of
    an isolated cluster (E_k = kinetic energies + half the pair energies of k).
    Leapfrog NVE from the oracle; integer-time velocities as half-step means;
    central differences of the moment against J_q at the middle step.  The
    mismatch is the O(dt^2) of the differences: it falls ~4x per halving of dt
    (a dropped or mis-signed term would leave an O(1) part)."""
    rng = np.random.default_rng(41)
    n, L = 8, 60.0
    models = [W.water()]
    sp = np.zeros(n, np.int32)
    R0 = 30.0 + 3.1 * np.array([[x, y, z] for x in (0, 1) for y in (0, 1) for z in (0, 1)], float)
    R0 += rng.normal(0, 0.1, R0.shape)
    q0 = W.random_quaternions(n, rng)
    o = Oracle(models, sp, L, 25.0, elec=1, lrc=0)
    v0, L0 = W.thermal_velocities(models, sp, q0, 30.0, o.s.kconv, rng)
    M = sum(s.mass for s in models[0].sites)
    Iinv = 1.0 / W.principal_moments(models[0])

    def mismatch(dt):
        states = [(R0, q0, v0, L0)]
        R, q, v, Lg = R0, q0, v0, L0
        for _ in range(3):
            R, q, v, Lg, _, _ = o.run_leapfrog(R, q, v, Lg, dt, 1, T0=0.0)
            states.append((R, q, v, Lg))

        # state k holds R_k, q_k and the velocities v_{k-1/2}, L_{k-1/2}
        def moment(k):
            Rk, qk = states[k][0], states[k][1]
            vk = 0.5 * (states[k][2] + states[k + 1][2])
            Lk = 0.5 * (states[k][3] + states[k + 1][3])
            A = W.quat_to_matrix(qk)
            Lb = np.einsum("nij,ni->nj", A, Lk)
            ke = (0.5 * M * (vk * vk).sum(1) + 0.5 * (Iinv * Lb * Lb).sum(1)) / o.s.kconv
            u = o.molecule_terms(Rk, qk)[:, :3].sum(1)      # half of each pair energy per molecule
            return ((ke + u)[:, None] * Rk).sum(0), (Rk, qk, vk, Lk)

        D0, _ = moment(0)
        D2, _ = moment(2)
        J = o.heat_flux(*moment(1)[1], h=[0.0])
        return np.abs((D2 - D0) / (2 * dt) - J).max() / np.abs(J).max()

    e1, e2 = mismatch(0.125), mismatch(0.0625)
    assert e2 < 1e-4
    assert 3.0 < e1 / e2 < 5.0, (e1, e2)


def test_heat_flux_enthalpy_term_and_units():
    """The partial-enthalpy term subtracts h sum_k v_k; lambda units on a constant ACF."""
    wl = W.water_box(N=64, rc=6.0, seed=21)
    o = Oracle.from_workload(wl)
    J0 = o.heat_flux(wl.R, wl.q, wl.v, wl.Lang, h=[0.0])
    J1 = o.heat_flux(wl.R, wl.q, wl.v, wl.Lang, h=[1234.5])
    np.testing.assert_allclose(J0 - J1, 1234.5 * wl.v.sum(0), rtol=1e-9, atol=1e-9 * np.abs(J0).max())
    kB = 1.380649e-23
    lam = Oracle.thermal_conductivity(np.full(5, 3.0), 2.0, 500.0, 300.0)
    assert lam == pytest.approx(3.0 * 4 * 2.0 * kB * 1e-5 / (3 * 500e-30 * 300.0 ** 2), rel=1e-14)
