"""ctypes binding of the FP64 C oracle (test infrastructure only).

The C source is compiled with gcc (-O2 -ffp-contract=off -fopenmp) into
oracle/_build/ on first use or by build().  Arrays cross as contiguous float64
numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ms2_oracle.c")
LIB = os.path.join(HERE, "_build", "libms2oracle.so")
MAXSP, MAXS, NTERMS = 4, 8, 16
TERM_NAMES = ["U_lj", "U_qq", "U_dd", "U_rec", "U_self", "U_intra", "U_bg", "U_lrc", "U_total",
              "W_pair", "W_rec", "W_bg", "W_total", "P_lrc", "n_pairs", "spare"]


def units(reduced: bool):
    """(coulomb, kconv): Coulomb constant e^2/(4 pi eps0 k_B) in K*Angstrom and the
    kinetic conversion of 1 K to g/mol*A^2/fs^2, from CODATA 2018; 1, 1 in reduced units."""
    if reduced:
        return 1.0, 1.0
    e, eps0, kB, NA = 1.602176634e-19, 8.8541878128e-12, 1.380649e-23, 6.02214076e23
    coulomb = e * e / (4 * math.pi * eps0 * kB) * 1e10          # K * Angstrom
    kconv = kB * NA * 1e3 * 1e20 / 1e30                          # g/mol A^2 fs^-2 per K
    return coulomb, kconv


def build(force=False):
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Sys(C.Structure):
    _fields_ = [("n_species", C.c_int), ("n_sites", C.c_int * MAXSP),
                ("pos", C.c_double * 3 * MAXS * MAXSP), ("mass", C.c_double * MAXS * MAXSP),
                ("lj", C.c_int * MAXS * MAXSP), ("sigma", C.c_double * MAXS * MAXSP),
                ("epsilon", C.c_double * MAXS * MAXSP), ("charge", C.c_double * MAXS * MAXSP),
                ("dipole", C.c_double * 3 * MAXS * MAXSP),
                ("N", C.c_int), ("species", C.POINTER(C.c_int)), ("L", C.c_double), ("rc", C.c_double),
                ("elec", C.c_int), ("eps_rf", C.c_double), ("alpha", C.c_double), ("kmax", C.c_int * 3),
                ("coulomb", C.c_double), ("kconv", C.c_double), ("lrc", C.c_int),
                ("crf_shift", C.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER
        d, i32 = P(C.c_double), P(C.c_int)
        sig = {
            "or_rotation": [d, d], "or_site_positions": [P(_Sys), d, d, d],
            "or_partner_counts": [P(_Sys), d, i32], "or_forces": [P(_Sys), d, d, d, d, d],
            "or_forces_mol": [P(_Sys), d, d, d, d, d, d],
            "or_ewald_reciprocal": [P(_Sys), d, d, d, d, d], "or_ewald_constants": [P(_Sys), d, d, d],
            "or_lrc": [P(_Sys), d, d], "or_kinetic": [P(_Sys), d, d, d, d],
            "or_run_vv": [P(_Sys), d, d, C.c_double, C.c_int, d],
            "or_run_leapfrog": [P(_Sys), d, d, d, d, C.c_double, C.c_int, C.c_double, C.c_int, d, d],
            "or_rdf_counts": [P(_Sys), d, d, C.c_double, C.c_int, P(C.c_longlong)],
            "or_rdf_edge_pairs": [P(_Sys), d, d, C.c_double, C.c_int, C.c_double, P(C.c_longlong)],
            "or_rdf_kinds": [P(_Sys), i32], "or_ndof": [P(_Sys)],
            "or_rc2_lattice": [C.c_double, C.c_double], "or_lattice": [C.c_double, C.c_double],
            "or_volume_derivatives": [P(_Sys), d, d, d],
            "or_massieu": [d, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, d],
            "or_current": [P(_Sys), d, d], "or_flux_acf": [d, C.c_int, C.c_int, d],
            "or_residence": [P(_Sys), d, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, d, d],
            "or_heat_flux": [P(_Sys), d, d, d, d, d, d],
            "or_thermal_conductivity": [d, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int],
            "or_conductivity": [d, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int],
            "or_set_threads": [C.c_int],
        }
        for name, args in sig.items():
            getattr(_lib, name).argtypes = args
        _lib.or_conductivity.restype = C.c_double
        _lib.or_thermal_conductivity.restype = C.c_double
        _lib.or_pressure.argtypes = [P(_Sys), C.c_double, d]
        _lib.or_pressure.restype = C.c_double
        _lib.or_ndof.restype = C.c_int
        _lib.or_rdf_kinds.restype = C.c_int
        _lib.or_rc2_lattice.restype = C.c_uint64
        _lib.or_lattice.restype = C.c_uint32
    return _lib


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == shape, (a.shape, shape)
    return a


class Oracle:
    """FP64 reference for one system (cubic box, molecule-centre cut-off)."""

    def __init__(self, models, species, L, rc, elec=0, eps_rf=0.0, alpha=0.0, kmax=(0, 0, 0),
                 reduced=False, lrc=1, coulomb=None):
        self.lib = _load()
        s = _Sys()
        s.n_species = len(models)
        assert 1 <= len(models) <= MAXSP
        for k, m in enumerate(models):
            assert len(m.sites) <= MAXS
            s.n_sites[k] = len(m.sites)
            for a, st in enumerate(m.sites):
                for c in range(3):
                    s.pos[k][a][c] = st.pos[c]
                    s.dipole[k][a][c] = st.dipole[c]
                s.mass[k][a] = st.mass
                s.lj[k][a] = int(st.lj)
                s.sigma[k][a], s.epsilon[k][a], s.charge[k][a] = st.sigma, st.epsilon, st.charge
        self.species = np.ascontiguousarray(species, dtype=np.int32)
        s.N = len(self.species)
        s.species = self.species.ctypes.data_as(C.POINTER(C.c_int))
        s.L, s.rc, s.elec, s.eps_rf, s.alpha = L, rc, elec, eps_rf, alpha
        for c in range(3):
            s.kmax[c] = kmax[c]
        cl, kc = units(reduced)
        s.coulomb = cl if coulomb is None else coulomb
        s.kconv = kc
        s.lrc = lrc
        self.s, self.N, self.models, self.L = s, s.N, models, L
        self.kconv, self.coulomb = kc, s.coulomb

    @classmethod
    def from_workload(cls, wl, **kw):
        args = dict(elec=wl.elec, eps_rf=wl.eps_rf, alpha=wl.alpha, kmax=wl.kmax, reduced=wl.reduced, lrc=wl.lrc)
        args.update(kw)
        return cls(wl.models, wl.species, wl.L, wl.rc, **args)

    @property
    def ref(self):
        return C.byref(self.s)

    def forces(self, R, q):
        N = self.N
        R, q = _f64(R, (N, 3)), _f64(q, (N, 4))
        F, tau, terms = np.zeros((N, 3)), np.zeros((N, 3)), np.zeros(NTERMS)
        self.lib.or_forces(self.ref, _p(R), _p(q), _p(F), _p(tau), _p(terms))
        return F, tau, dict(zip(TERM_NAMES, terms))

    def molecule_terms(self, R, q):
        """Per-molecule shares (N x 4): 1/2 sum_j of u_lj, u_qq, u_dd and the pair virial."""
        N = self.N
        R, q = _f64(R, (N, 3)), _f64(q, (N, 4))
        F, tau, terms, mol = np.zeros((N, 3)), np.zeros((N, 3)), np.zeros(NTERMS), np.zeros((N, 4))
        self.lib.or_forces_mol(self.ref, _p(R), _p(q), _p(F), _p(tau), _p(terms), _p(mol))
        return mol

    def energy(self, R, q):
        return self.forces(R, q)[2]["U_total"]

    def partner_counts(self, R):
        R = _f64(R, (self.N, 3))
        c = np.zeros(self.N, np.int32)
        self.lib.or_partner_counts(self.ref, _p(R), c.ctypes.data_as(C.POINTER(C.c_int)))
        return c

    def site_positions(self, R, q):
        R, q = _f64(R, (self.N, 3)), _f64(q, (self.N, 4))
        out = np.zeros((self.N, MAXS, 3))
        self.lib.or_site_positions(self.ref, _p(R), _p(q), _p(out))
        return out

    def ewald_reciprocal(self, R, q):
        R, q = _f64(R, (self.N, 3)), _f64(q, (self.N, 4))
        fs, U, W = np.zeros((self.N, MAXS, 3)), C.c_double(), C.c_double()
        self.lib.or_ewald_reciprocal(self.ref, _p(R), _p(q), _p(fs), C.byref(U), C.byref(W))
        return fs, U.value, W.value

    def ewald_constants(self):
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        self.lib.or_ewald_constants(self.ref, C.byref(a), C.byref(b), C.byref(c))
        return a.value, b.value, c.value

    def volume_derivatives(self, R, q):
        """(dU/dV, d2U/dV2) at fixed scaled centres and orientations (Sec. 2, Eq. 1)."""
        out = np.zeros(2)
        self.lib.or_volume_derivatives(self.ref, _p(np.ascontiguousarray(R, np.float64)),
                                       _p(np.ascontiguousarray(q, np.float64)), _p(out))
        return out[0], out[1]

    def current(self, v):
        """Electric current flux sum_k q_k v_k over net-charged molecules (Eq. 4)."""
        j = np.zeros(3)
        self.lib.or_current(self.ref, _p(np.ascontiguousarray(v, np.float64)), _p(j))
        return j

    def heat_flux(self, R, q, v, Lang, h):
        """Microscopic heat flow J_q (Eqs. 5-6; K A/fs) with per-species partial enthalpies h (K)."""
        J = np.zeros(3)
        hh = np.zeros(8)
        hh[:len(h)] = h
        f = lambda a: _p(np.ascontiguousarray(a, np.float64))
        self.lib.or_heat_flux(self.ref, f(R), f(q), f(v), f(Lang), _p(hh), _p(J))
        return J

    @staticmethod
    def set_threads(n):
        """Host threads of the oracle's OpenMP loops (timing; results do not depend on it)."""
        _load().or_set_threads(C.c_int(int(n)))

    @staticmethod
    def thermal_conductivity(acf, dt_ext, V, T, reduced=False):
        """lambda (W/(m K), or reduced) from the ACF <J_q(t).J_q(0)> (Eq. 5)."""
        a = np.ascontiguousarray(acf, np.float64)
        return _load().or_thermal_conductivity(_p(a), C.c_int(len(a)), C.c_double(dt_ext), C.c_double(V),
                                               C.c_double(T), C.c_int(int(reduced)))

    def residence(self, R_series, si, sj, r_shell, t_star, n_lags):
        """Residence correlation (Eq. 7, Impey tolerance t_star in samples) of species sj
        around si over configurations R_series (T x N x 3); returns (corr, solvation number)."""
        Rs = np.ascontiguousarray(R_series, np.float64)
        corr = np.zeros(n_lags)
        nsol = C.c_double()
        self.lib.or_residence(self.ref, _p(Rs), C.c_int(len(Rs)), C.c_int(si), C.c_int(sj), C.c_double(r_shell),
                              C.c_int(t_star), C.c_int(n_lags), _p(corr), C.byref(nsol))
        return corr, nsol.value

    @staticmethod
    def flux_acf(j, n_lags):
        """Autocorrelation <j(t).j(0)> of a flux series j (n x 3) over all time origins."""
        a = np.ascontiguousarray(j, np.float64)
        out = np.zeros(n_lags)
        _load().or_flux_acf(_p(a), C.c_int(len(a)), C.c_int(n_lags), _p(out))
        return out

    @staticmethod
    def conductivity(acf, dt_ext, V, T, reduced=False):
        """Green-Kubo electric conductivity (Eq. 3) from the current ACF: S/m, or reduced."""
        a = np.ascontiguousarray(acf, np.float64)
        return _load().or_conductivity(_p(a), C.c_int(len(a)), C.c_double(dt_ext), C.c_double(V), C.c_double(T),
                                       C.c_int(int(reduced)))

    @staticmethod
    def massieu(acc, U0, V0, beta, V, N):
        """A^r_mn for mn = 10, 01, 20, 11, 02, 30, 21, 12 from the moment sums acc (11 values)."""
        lib = _load()
        a = np.ascontiguousarray(acc, np.float64)
        out = np.zeros(8)
        lib.or_massieu(_p(a), C.c_double(U0), C.c_double(V0), C.c_double(beta), C.c_double(V), C.c_int(N), _p(out))
        return out

    def lrc(self):
        U, P = C.c_double(), C.c_double()
        self.lib.or_lrc(self.ref, C.byref(U), C.byref(P))
        return U.value, P.value

    def kinetic(self, q, v, Lang):
        q, v, Lang = _f64(q, (self.N, 4)), _f64(v, (self.N, 3)), _f64(Lang, (self.N, 3))
        ke = np.zeros(2)
        self.lib.or_kinetic(self.ref, _p(q), _p(v), _p(Lang), _p(ke))
        return ke

    def ndof(self):
        return self.lib.or_ndof(self.ref)

    def pressure(self, ke_tr, terms):
        t = np.array([terms[n] for n in TERM_NAMES])
        return self.lib.or_pressure(self.ref, ke_tr, _p(t))

    def run_vv(self, R, v, dt, nsteps, thermo=True):
        R, v = _f64(R, (self.N, 3)).copy(), _f64(v, (self.N, 3)).copy()
        th = np.zeros((max(nsteps, 1), 5))
        self.lib.or_run_vv(self.ref, _p(R), _p(v), dt, nsteps, _p(th) if thermo else None)
        return R, v, th[:nsteps]

    def run_leapfrog(self, R, q, v, Lang, dt, nsteps, T0=0.0, n_iter=3, thermo=True):
        N = self.N
        R, q = _f64(R, (N, 3)).copy(), _f64(q, (N, 4)).copy()
        v, Lang = _f64(v, (N, 3)).copy(), _f64(Lang, (N, 3)).copy()
        th, ts = np.zeros((max(nsteps, 1), 5)), np.zeros(max(nsteps, 1))
        self.lib.or_run_leapfrog(self.ref, _p(R), _p(q), _p(v), _p(Lang), dt, nsteps, T0, n_iter,
                                 _p(th) if thermo else None, _p(ts))
        return R, q, v, Lang, th[:nsteps], ts[:nsteps]

    def rdf_kinds(self):
        k = np.zeros(MAXSP * MAXS, np.int32)
        T = self.lib.or_rdf_kinds(self.ref, k.ctypes.data_as(C.POINTER(C.c_int)))
        return T, k.reshape(MAXSP, MAXS)

    def rdf_counts(self, R, q, r_max, nbins):
        T, _ = self.rdf_kinds()
        c = np.zeros((T * (T + 1) // 2, nbins), np.int64)
        R, q = _f64(R, (self.N, 3)), _f64(q, (self.N, 4))
        self.lib.or_rdf_counts(self.ref, _p(R), _p(q), r_max, nbins, c.ctypes.data_as(C.POINTER(C.c_longlong)))
        return c

    def rdf_edge_pairs(self, R, q, r_max, nbins, delta):
        c = np.zeros(nbins + 1, np.int64)
        R, q = _f64(R, (self.N, 3)), _f64(q, (self.N, 4))
        self.lib.or_rdf_edge_pairs(self.ref, _p(R), _p(q), r_max, nbins, delta,
                                   c.ctypes.data_as(C.POINTER(C.c_longlong)))
        return c

    def rotation(self, q):
        A = np.zeros(9)
        qq = np.ascontiguousarray(q, np.float64)
        self.lib.or_rotation(_p(qq), _p(A))
        return A.reshape(3, 3)

    def rc2_lattice(self):
        return int(self.lib.or_rc2_lattice(self.s.rc, self.s.L))
