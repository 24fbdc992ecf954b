"""Seeded synthetic inputs: potential models, lattices, orientations, velocities.

This module produces inputs only.  It holds none of the method's arithmetic
(no energies, forces, cut-offs or integration); both the GPU library's tests and
the FP64 oracle consume what it returns.

Units (the library's fixed unit system): length Angstrom, time fs, mass g/mol,
charge e, dipole e*Angstrom, energy and temperature K (k_B = 1).  The LJ fluid
uses reduced units (sigma = epsilon = m = k_B = 1).

Workloads are shaped like the paper's: pure water at liquid density with
N ~ 10^3 molecules and a molecule-centre cut-off near half the box edge (Sec.
"Hybrid MPI & OpenMP Parallelization", Table 1), a single-site LJ fluid, an
ionic solution treated with Ewald summation, and a Stockmayer-like dipolar fluid.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# site kind bits (same meaning as MS2_SITE_* in include/ms2.h)
SITE_LJ, SITE_CHARGE, SITE_DIPOLE = 1, 2, 4

AVOGADRO = 6.02214076e23
DEBYE_EA = 0.2081943  # 1 Debye in e*Angstrom


@dataclass
class Site:
    pos: tuple            # body frame (centre of mass at origin, principal axes)
    mass: float
    sigma: float = 0.0
    epsilon: float = 0.0
    charge: float = 0.0
    dipole: tuple = (0.0, 0.0, 0.0)
    lj: bool = False

    @property
    def kind(self) -> int:
        k = SITE_LJ if self.lj else 0
        if self.charge != 0.0:
            k |= SITE_CHARGE
        if any(c != 0.0 for c in self.dipole):
            k |= SITE_DIPOLE
        return k


@dataclass
class Model:
    name: str
    sites: list = field(default_factory=list)

    @property
    def mass(self) -> float:
        return sum(s.mass for s in self.sites)


def _centre(sites):
    """Shift site positions so that the centre of mass is the origin."""
    M = sum(s.mass for s in sites)
    com = [sum(s.mass * s.pos[k] for s in sites) / M for k in range(3)]
    for s in sites:
        s.pos = tuple(s.pos[k] - com[k] for k in range(3))
    return sites


def lj_atom() -> Model:
    """Single LJ site, reduced units."""
    return Model("lj", [Site((0.0, 0.0, 0.0), 1.0, 1.0, 1.0, lj=True)])


def water(sigma=3.166, eps=78.2, qO=-0.8476, bond=1.0, angle_deg=109.47,
          mO=15.9994, mH=1.00794) -> Model:
    """Rigid 3-site water: LJ + charge on O, charges on the two H.

    The molecule lies in the xz plane with its symmetry axis along z, so that
    the coordinate axes are principal axes after the centre-of-mass shift."""
    h = 0.5 * math.radians(angle_deg)
    x, z = bond * math.sin(h), bond * math.cos(h)
    sites = [Site((0.0, 0.0, 0.0), mO, sigma, eps, qO, lj=True),
             Site((x, 0.0, z), mH, charge=-qO / 2),
             Site((-x, 0.0, z), mH, charge=-qO / 2)]
    return Model("water", _centre(sites))


def ion(charge, sigma, eps, mass, name) -> Model:
    return Model(name, [Site((0.0, 0.0, 0.0), mass, sigma, eps, charge, lj=True)])


def cation() -> Model:
    return ion(+1.0, 2.35, 65.0, 22.99, "cation")


def anion() -> Model:
    return ion(-1.0, 4.40, 50.0, 35.45, "anion")


def stockmayer(sigma=3.5, eps=120.0, elongation=1.0, dipole_debye=2.0, msite=20.0) -> Model:
    """Two LJ sites on the z axis and a point dipole at the centre (linear rotor)."""
    mu = dipole_debye * DEBYE_EA
    sites = [Site((0.0, 0.0, -0.5 * elongation), msite, sigma, eps, lj=True),
             Site((0.0, 0.0, +0.5 * elongation), msite, sigma, eps, lj=True),
             Site((0.0, 0.0, 0.0), 0.0, dipole=(0.0, 0.0, mu))]
    return Model("stockmayer", _centre(sites))


# ------------------------------------------------------------------ lattices
def fcc_lattice(ncell: int, L: float) -> np.ndarray:
    a = L / ncell
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.stack(np.meshgrid(*[np.arange(ncell)] * 3, indexing="ij"), -1).reshape(-1, 3)
    return ((g[:, None, :] + basis[None]) * a).reshape(-1, 3).astype(np.float64)


def sc_lattice(n: int, L: float) -> np.ndarray:
    """Simple-cubic lattice with the smallest m^3 >= n points; first n returned."""
    m = int(math.ceil(n ** (1.0 / 3.0) - 1e-9))
    a = L / m
    g = np.stack(np.meshgrid(*[np.arange(m)] * 3, indexing="ij"), -1).reshape(-1, 3)
    return ((g + 0.5) * a)[:n].astype(np.float64)


def random_quaternions(n: int, rng: np.random.Generator) -> np.ndarray:
    """Uniformly distributed unit quaternions (w, x, y, z) (Shoemake 1992)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1 - u1), np.sqrt(u1)
    q = np.stack([a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                  b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)], -1)
    return q.astype(np.float64)


def quat_to_matrix(q: np.ndarray) -> np.ndarray:
    """Body->space rotation matrices of unit quaternions (input preparation only)."""
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def principal_moments(m: Model) -> np.ndarray:
    I = np.zeros(3)
    for s in m.sites:
        p = np.array(s.pos)
        I += s.mass * (np.dot(p, p) - p * p)
    return I


def thermal_velocities(models, species, q, T, kconv, rng, exact=True):
    """Maxwell-Boltzmann centre velocities and space-frame angular momenta at
    temperature T: total momentum removed; if exact, scaled together so that the
    kinetic temperature with (3N - 3 + rotational) degrees of freedom is T."""
    N = len(species)
    M = np.array([models[s].mass for s in species])
    v = rng.normal(size=(N, 3)) * np.sqrt(T * kconv / M)[:, None]
    v -= (M[:, None] * v).sum(0) / M.sum()
    Lb = np.zeros((N, 3))
    ndof = 3 * N - 3
    for i, s in enumerate(species):
        I = principal_moments(models[s])
        free = I > 1e-12 * I.max() if I.max() > 0 else np.zeros(3, bool)
        ndof += int(free.sum())
        Lb[i, free] = rng.normal(size=int(free.sum())) * np.sqrt(T * kconv * I[free])
    A = quat_to_matrix(q)
    Ls = np.einsum("nij,nj->ni", A, Lb)
    if exact:
        ke = 0.5 * (M[:, None] * v * v).sum() / kconv
        for i, s in enumerate(species):
            I = principal_moments(models[s])
            nz = I > 1e-12 * I.max() if I.max() > 0 else np.zeros(3, bool)
            ke += 0.5 * (Lb[i, nz] ** 2 / I[nz]).sum() / kconv
        lam = math.sqrt(T / (2 * ke / ndof))
        v *= lam
        Ls *= lam
    return v, Ls


# ------------------------------------------------------------------ configs
@dataclass
class Workload:
    name: str
    models: list
    species: np.ndarray
    L: float
    rc: float
    elec: int                # 0 none, 1 reaction field, 2 Ewald
    T: float
    dt: float
    reduced: bool
    R: np.ndarray
    q: np.ndarray
    v: np.ndarray
    Lang: np.ndarray
    alpha: float = 0.0
    kmax: tuple = (0, 0, 0)
    eps_rf: float = 0.0      # <= 0: conducting
    integrator: int = 1      # 0 velocity Verlet, 1 leapfrog + quaternion
    lrc: int = 1
    seed: int = 0

    @property
    def N(self) -> int:
        return len(self.species)


WATER_NUMBER_DENSITY = 997.0 * 1e3 / 18.01528 * AVOGADRO * 1e-30  # per A^3 at 997 kg/m^3


def lj_fluid(N=256, rho=0.7, T=1.0, rc=3.5, seed=1, dt=0.002) -> Workload:
    """Single-site LJ fluid on an FCC lattice, reduced units, velocity Verlet."""
    ncell = round((N / 4) ** (1 / 3))
    assert 4 * ncell ** 3 == N
    L = (N / rho) ** (1 / 3)
    rng = np.random.default_rng(seed)
    models = [lj_atom()]
    sp = np.zeros(N, np.int32)
    q = np.tile([1.0, 0, 0, 0], (N, 1))
    v, Ls = thermal_velocities(models, sp, q, T, 1.0, rng)
    return Workload("lj_fluid_N%d" % N, models, sp, L, rc, 0, T, dt, True,
                    fcc_lattice(ncell, L), q, v, Ls, integrator=0, seed=seed)


def water_box(N=1000, rc=14.0, T=298.0, seed=2, dt=2.0, elec=1, density=None, jitter=0.05) -> Workload:
    """Rigid water on a simple-cubic lattice with random orientations."""
    rho = WATER_NUMBER_DENSITY if density is None else density
    L = (N / rho) ** (1 / 3)
    rng = np.random.default_rng(seed)
    models = [water()]
    sp = np.zeros(N, np.int32)
    R = sc_lattice(N, L) + rng.uniform(-jitter, jitter, size=(N, 3))
    q = random_quaternions(N, rng)
    v, Ls = thermal_velocities(models, sp, q, T, KCONV, rng)
    wl = Workload("water_N%d" % N, models, sp, L, rc, elec, T, dt, False, R, q, v, Ls, seed=seed)
    if elec == 2:
        wl.alpha, wl.kmax = 0.25, (8, 8, 8)
    return wl


def ionic_solution(n_water=1000, n_ion_pairs=20, rc=14.0, T=298.0, seed=3, dt=2.0,
                   alpha=0.25, kmax=(8, 8, 8)) -> Workload:
    """Water plus single-site cations and anions at water number density, Ewald.

    Molecules sit on the points of a simple-cubic lattice (seeded choice of
    which points hold ions), waters randomly oriented."""
    N = n_water + 2 * n_ion_pairs
    L = (N / WATER_NUMBER_DENSITY) ** (1 / 3)
    rng = np.random.default_rng(seed)
    models = [water(), cation(), anion()]
    m = int(math.ceil(N ** (1 / 3)))
    pts = sc_lattice(m ** 3, L)
    pick = rng.permutation(m ** 3)[:N]
    R = pts[pick] + rng.uniform(-0.05, 0.05, size=(N, 3))
    sp = np.zeros(N, np.int32)
    ions = rng.permutation(N)[:2 * n_ion_pairs]
    sp[ions[:n_ion_pairs]] = 1
    sp[ions[n_ion_pairs:]] = 2
    order = np.argsort(sp, kind="stable")      # molecules numbered model by model
    sp, R = sp[order], R[order]
    q = random_quaternions(N, rng)
    q[sp != 0] = [1.0, 0, 0, 0]
    v, Ls = thermal_velocities(models, sp, q, T, KCONV, rng)
    return Workload("ionic_N%d" % N, models, sp, L, rc, 2, T, dt, False, R, q, v, Ls,
                    alpha=alpha, kmax=tuple(kmax), seed=seed)


def water_argon(n_water=800, n_argon=200, rc=14.0, T=298.0, seed=6, dt=2.0) -> Workload:
    """Binary mixture of rigid water and argon-like LJ atoms (reaction field) at
    water number density: molecules on simple-cubic lattice points (a seeded
    choice of which hold argon), numbered species by species, waters randomly
    oriented (the multi-component heat flux of Sec. 4)."""
    N = n_water + n_argon
    L = (N / WATER_NUMBER_DENSITY) ** (1 / 3)
    rng = np.random.default_rng(seed)
    models = [water(), argon()]
    R = sc_lattice(N, L) + rng.uniform(-0.05, 0.05, size=(N, 3))
    sp = np.zeros(N, np.int32)
    sp[rng.permutation(N)[:n_argon]] = 1
    order = np.argsort(sp, kind="stable")
    sp, R = sp[order], R[order]
    q = random_quaternions(N, rng)
    q[sp != 0] = [1.0, 0, 0, 0]
    v, Ls = thermal_velocities(models, sp, q, T, KCONV, rng)
    return Workload("water_argon_N%d" % N, models, sp, L, rc, 1, T, dt, False, R, q, v, Ls, seed=seed)


def stockmayer_fluid(N=500, rho=0.012, T=300.0, rc=17.5, seed=4, dt=2.0) -> Workload:
    L = (N / rho) ** (1 / 3)
    rng = np.random.default_rng(seed)
    models = [stockmayer()]
    sp = np.zeros(N, np.int32)
    R = sc_lattice(N, L)
    q = random_quaternions(N, rng)
    v, Ls = thermal_velocities(models, sp, q, T, KCONV, rng)
    return Workload("stockmayer_N%d" % N, models, sp, L, min(rc, 0.49 * L), 1, T, dt, False, R, q, v, Ls,
                    seed=seed)


# unit conversion of the fixed unit system, needed to make thermal velocities:
# 1 K (energy) in g/mol * A^2 / fs^2
KCONV = 1.380649e-23 * 6.02214076e23 * 1e3 * 1e20 / 1e30


# ------------------------------------------------- many systems and jobs
def argon() -> Model:
    """LJ atom in the fixed unit system (argon-like: sigma 3.405 A, eps 119.8 K)."""
    return Model("argon", [Site((0.0, 0.0, 0.0), 39.948, 3.405, 119.8, lj=True)])


# nominal states of the three members of the many-system mix:
# (model factory, T0 in K, number density rho0 in 1/A^3, model cutoff in A, electrostatics)
MIX_STATES = {
    "lj": (argon, 119.8, 0.7 / 3.405 ** 3, 3.5 * 3.405, 0),           # T* = 1, rho* = 0.7, rc = 3.5 sigma
    "stockmayer": (stockmayer, 300.0, 0.012, 17.5, 1),
    "water": (water, 298.0, WATER_NUMBER_DENSITY, 14.0, 1),
}


def system_mix(n_systems=512, seed=4, n_range=(256, 2048)):
    """Independent systems: model uniform over {LJ, Stockmayer, water}, N uniform
    over n_range, T uniform in [0.7, 1.3] T0, rho uniform in [0.5, 1.0] rho0, and
    the model cutoff capped at 0.49 L.  Returns a list of dicts with keys name,
    models, counts, T, rho, cutoff, elec, seed."""
    rng = np.random.default_rng(seed)
    names = list(MIX_STATES)
    out = []
    for k in range(n_systems):
        name = names[int(rng.integers(len(names)))]
        make, T0, rho0, rc, elec = MIX_STATES[name]
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        T = T0 * rng.uniform(0.7, 1.3)
        rho = rho0 * rng.uniform(0.5, 1.0)
        L = (N / rho) ** (1 / 3)
        out.append(dict(name=name, models=[make()], counts=[N], T=T, rho=rho, cutoff=min(rc, 0.49 * L),
                        elec=elec, seed=seed * 100003 + k))
    return out


def job_stream(n_jobs=256, rate=50.0, seed=5, n_range=(500, 4000), steps=(10000, 100000), ionic_fraction=0.2):
    """Simulation jobs with Poisson arrivals (rate per second): N uniform over
    n_range, steps uniform over the multiples of 100 in the steps range; a
    fraction are ionic solutions (water + 2% ion pairs, Ewald), the rest drawn
    like system_mix.  Returns dicts as system_mix plus steps and arrival (s)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    names = list(MIX_STATES)
    out = []
    for k in range(n_jobs):
        t += rng.exponential(1.0 / rate)
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        nsteps = 100 * int(rng.integers(steps[0] // 100, steps[1] // 100 + 1))
        if rng.uniform() < ionic_fraction:
            pairs = max(1, int(round(0.02 * N)))
            job = dict(name="ionic", models=[water(), cation(), anion()], counts=[N - 2 * pairs, pairs, pairs],
                       T=298.0 * rng.uniform(0.9, 1.1), rho=WATER_NUMBER_DENSITY, elec=2)
            job["cutoff"] = min(14.0, 0.49 * (N / job["rho"]) ** (1 / 3))
        else:
            name = names[int(rng.integers(len(names)))]
            make, T0, rho0, rc, elec = MIX_STATES[name]
            T, rho = T0 * rng.uniform(0.7, 1.3), rho0 * rng.uniform(0.5, 1.0)
            job = dict(name=name, models=[make()], counts=[N], T=T, rho=rho,
                       cutoff=min(rc, 0.49 * (N / rho) ** (1 / 3)), elec=elec)
        job.update(steps=nsteps, arrival=t, seed=seed * 100003 + k)
        out.append(job)
    return out
