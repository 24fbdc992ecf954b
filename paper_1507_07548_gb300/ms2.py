"""ctypes binding of libms2 (include/ms2.h): argument marshalling only.

Every function of the C ABI is exposed under its own name (ms2_create_system,
ms2_step, ms2_energy_virial, ...).  `System` is a thin convenience wrapper that
converts numpy arrays and raises on error statuses; all computation happens in
the library's CUDA kernels.  There is no fallback: if libms2.so is missing or
cannot be loaded, importing the functions raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libms2.so")

STATUS = {0: "MS2_OK", 1: "MS2_EINVAL", 2: "MS2_ENOMEM", 3: "MS2_EBUDGET", 4: "MS2_ECUDA",
          5: "MS2_EUNSTABLE", 6: "MS2_ETIMEOUT", 7: "MS2_ESTATE"}
ELEC_NONE, ELEC_RF, ELEC_EWALD = 0, 1, 2
INT_VERLET, INT_LEAPFROG_Q = 0, 1


class Ms2Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class ms2_site(C.Structure):
    _fields_ = [("kind", C.c_int), ("pos", C.c_double * 3), ("mass", C.c_double), ("sigma", C.c_double),
                ("epsilon", C.c_double), ("charge", C.c_double), ("dipole", C.c_double * 3)]


class ms2_model(C.Structure):
    _fields_ = [("n_sites", C.c_int), ("sites", C.POINTER(ms2_site))]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class ms2_options(C.Structure):
    _fields_ = [("eps_rf", C.c_double), ("lrc", C.c_int), ("dt", C.c_double), ("thermostat", C.c_int),
                ("seed", C.c_ulonglong), ("integrator", C.c_int), ("reduced", C.c_int), ("quat_iters", C.c_int),
                ("graph_chunk", C.c_int), ("fp64", C.c_int), ("massieu", C.c_int), ("fused_step", C.c_int), ("stream", C.c_void_p), ("dev_alloc", ALLOC_FN),
                ("dev_free", FREE_FN), ("alloc_ctx", C.c_void_p)]


class ms2_job(C.Structure):
    _fields_ = [("models", C.POINTER(ms2_model)), ("N_per_model", C.POINTER(C.c_int)), ("n_models", C.c_int),
                ("T", C.c_double), ("rho", C.c_double), ("cutoff", C.c_double), ("elec", C.c_int),
                ("steps", C.c_longlong), ("arrival_time", C.c_double), ("seed", C.c_ulonglong),
                ("rdf_bins", C.c_int), ("rdf_every", C.c_int), ("R0", C.POINTER(C.c_double)),
                ("q0", C.POINTER(C.c_double))]


class ms2_job_result(C.Structure):
    _fields_ = [("job_id", C.c_longlong), ("status", C.c_int), ("U_avg", C.c_double), ("U_err", C.c_double),
                ("P_avg", C.c_double), ("P_err", C.c_double), ("T_avg", C.c_double), ("t_arrive", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("n_rows", C.c_int), ("n_bins", C.c_int),
                ("g", C.c_double * 4096)]


_P = C.POINTER
_d = _P(C.c_double)
_vp = C.c_void_p
SIGNATURES = {
    "ms2_default_options": (C.c_int, [_P(ms2_options)]),
    "ms2_create_system": (C.c_int, [_P(ms2_model), _P(C.c_int), C.c_int, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_int, _P(ms2_options), _P(_vp)]),
    "ms2_destroy_system": (C.c_int, [_vp]),
    "ms2_system_info": (C.c_int, [_vp, _P(C.c_int), _d, _d, _P(C.c_int)]),
    "ms2_step": (C.c_int, [_vp, C.c_longlong]),
    "ms2_energy_virial": (C.c_int, [_vp, _d, _d, _d, _d]),
    "ms2_energy_terms": (C.c_int, [_vp, _d]),
    "ms2_forces_torques": (C.c_int, [_vp, _d, _d]),
    "ms2_forces_torques_dev": (C.c_int, [_vp, _vp, _vp]),
    "ms2_ewald_params": (C.c_int, [_vp, C.c_double, C.c_int, C.c_int, C.c_int]),
    "ms2_get_state": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _P(C.c_longlong)]),
    "ms2_set_state": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "ms2_partner_counts": (C.c_int, [_vp, _P(C.c_int)]),
    "ms2_site_offsets": (C.c_int, [_vp, _d, _P(C.c_int)]),
    "ms2_molecule_energies": (C.c_int, [_vp, _d]),
    "ms2_rdf_setup": (C.c_int, [_vp, C.c_double, C.c_int, C.c_int]),
    "ms2_rdf_sample": (C.c_int, [_vp]),
    "ms2_rdf": (C.c_int, [_vp, _P(C.c_longlong), _d, _P(C.c_int), _P(C.c_int)]),
    "ms2_averages": (C.c_int, [_vp, _d, _P(C.c_longlong)]),
    "ms2_reset_averages": (C.c_int, [_vp]),
    "ms2_batch_create": (C.c_int, [_P(_vp), C.c_int, _P(_vp)]),
    "ms2_batch_step": (C.c_int, [_vp, C.c_longlong]),
    "ms2_batch_destroy": (C.c_int, [_vp]),
    "ms2_serve_open": (C.c_int, [C.c_size_t, C.c_int, _P(ms2_options), _P(_vp)]),
    "ms2_serve_submit": (C.c_int, [_vp, _P(ms2_job), _P(C.c_longlong)]),
    "ms2_serve_poll": (C.c_int, [_vp, _P(ms2_job_result), C.c_int, _P(C.c_int)]),
    "ms2_serve_drain": (C.c_int, [_vp, C.c_double]),
    "ms2_serve_close": (C.c_int, [_vp]),
    "ms2_enable_timing": (C.c_int, [_vp, C.c_int]),
    "ms2_volume_derivatives": (C.c_int, [_vp, _d, _d]),
    "ms2_massieu": (C.c_int, [_vp, _d, _P(C.c_longlong)]),
    "ms2_conductivity_setup": (C.c_int, [_vp, C.c_int, C.c_int]),
    "ms2_current": (C.c_int, [_vp, _d]),
    "ms2_conductivity": (C.c_int, [_vp, _d, _d, _P(C.c_longlong)]),
    "ms2_heat_setup": (C.c_int, [_vp, C.c_int, C.c_int, _d]),
    "ms2_heat_flux": (C.c_int, [_vp, _d]),
    "ms2_thermal_conductivity": (C.c_int, [_vp, _d, _d, _P(C.c_longlong)]),
    "ms2_residence_setup": (C.c_int, [_vp, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int]),
    "ms2_residence": (C.c_int, [_vp, _d, _d, _d, _P(C.c_longlong)]),
    "ms2_step_kernel": (C.c_int, [_vp, _P(C.c_int)]),
    "ms2_last_step_phases": (C.c_int, [_vp, _d]),
    "ms2_last_step_times": (C.c_int, [_vp, _d]),
    "ms2_fault_inject": (C.c_int, [_vp, C.c_int, C.c_double]),
    "ms2_forces_noalloc": (C.c_int, [_P(ms2_model), _P(C.c_int), C.c_int, C.c_double, C.c_double, C.c_int,
                                     _P(ms2_options), _vp, _vp, _vp, _vp, _vp, _vp]),
    "ms2_noalloc_scratch_bytes": (C.c_size_t, []),
    "ms2_last_error": (C.c_char_p, []),
    "ms2_kernel_launches": (C.c_longlong, []),
    "ms2_version": (C.c_char_p, []),
}

_lib = None


def lib():
    """Loads libms2.so (raises if it is not built: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise ImportError("libms2.so is not built (run __graft_entry__.build()); no CPU fallback exists")
        L = C.CDLL(LIBPATH)
        missing = []
        for name, (res, args) in SIGNATURES.items():
            try:
                f = getattr(L, name)
            except AttributeError:
                missing.append(name)
                continue
            f.restype = res
            f.argtypes = args
        if missing:
            raise ImportError("libms2.so lacks %s" % ", ".join(missing))
        _lib = L
    return _lib


def check(status):
    if status != 0:
        raise Ms2Error(status, lib().ms2_last_error().decode())
    return status


def __getattr__(name):  # module-level access to the C functions under their own names
    if name in SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)


# ----------------------------------------------------------------- helpers
def make_models(models):
    """workloads.Model list -> (ms2_model array, keep-alive list)."""
    keep = []
    arr = (ms2_model * len(models))()
    for k, m in enumerate(models):
        sites = (ms2_site * len(m.sites))()
        for a, s in enumerate(m.sites):
            sites[a].kind = s.kind
            for c in range(3):
                sites[a].pos[c] = s.pos[c]
                sites[a].dipole[c] = s.dipole[c]
            sites[a].mass, sites[a].sigma, sites[a].epsilon, sites[a].charge = s.mass, s.sigma, s.epsilon, s.charge
        keep.append(sites)
        arr[k].n_sites = len(m.sites)
        arr[k].sites = C.cast(sites, C.POINTER(ms2_site))
    return arr, keep


def default_options(**kw):
    o = ms2_options()
    check(lib().ms2_default_options(C.byref(o)))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _dp(a):
    return a.ctypes.data_as(_d)


def _f64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == shape, (a.shape, shape)
    return a


class System:
    """One ms2 system on the GPU (wraps an ms2_system handle)."""

    def __init__(self, models, counts, T, cutoff, elec, box=0.0, rho=0.0, **opts):
        self.models_py = models
        self._models, self._keep = make_models(models)
        cnt = (C.c_int * len(counts))(*[int(c) for c in counts])
        self._opts = default_options(**opts)
        h = _vp()
        check(lib().ms2_create_system(self._models, cnt, len(models), box, T, rho, cutoff, elec,
                                      C.byref(self._opts), C.byref(h)))
        self.h = h
        N, L, rc, nd = C.c_int(), C.c_double(), C.c_double(), C.c_int()
        check(lib().ms2_system_info(h, C.byref(N), C.byref(L), C.byref(rc), C.byref(nd)))
        self.N, self.L, self.rc, self.ndof = N.value, L.value, rc.value, nd.value

    @classmethod
    def from_workload(cls, wl, set_state=True, **kw):
        counts = [int((wl.species == k).sum()) for k in range(len(wl.models))]
        assert np.all(np.diff(wl.species) >= 0), "species must be sorted model by model"
        opts = dict(dt=wl.dt, reduced=int(wl.reduced), integrator=wl.integrator, lrc=wl.lrc,
                    eps_rf=wl.eps_rf, seed=wl.seed)
        opts.update(kw)
        s = cls(wl.models, counts, wl.T, wl.rc, wl.elec, box=wl.L, **opts)
        if wl.elec == ELEC_EWALD:
            s.ewald_params(wl.alpha, *wl.kmax)
        if set_state:
            s.set_state(wl.R, wl.q, wl.v, wl.Lang)
        return s

    def close(self):
        if getattr(self, "h", None):
            lib().ms2_destroy_system(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n):
        check(lib().ms2_step(self.h, n))

    def energy_virial(self):
        U, Wv, T, P = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        check(lib().ms2_energy_virial(self.h, C.byref(U), C.byref(Wv), C.byref(T), C.byref(P)))
        return U.value, Wv.value, T.value, P.value

    TERM_NAMES = ["U_lj", "U_qq", "U_dd", "U_rec", "U_self", "U_intra", "U_bg", "U_lrc", "U_total",
                  "W_pair", "W_rec", "W_bg", "W_total", "P_lrc", "n_pairs", "KE_total"]

    def energy_terms(self):
        t = np.zeros(16)
        check(lib().ms2_energy_terms(self.h, _dp(t)))
        return dict(zip(self.TERM_NAMES, t))

    def forces_torques(self):
        F, tau = np.zeros((self.N, 3)), np.zeros((self.N, 3))
        check(lib().ms2_forces_torques(self.h, _dp(F), _dp(tau)))
        return F, tau

    def ewald_params(self, alpha, kx, ky, kz):
        check(lib().ms2_ewald_params(self.h, alpha, kx, ky, kz))

    def get_state(self):
        R, q, v, Lg = np.zeros((self.N, 3)), np.zeros((self.N, 4)), np.zeros((self.N, 3)), np.zeros((self.N, 3))
        st = C.c_longlong()
        check(lib().ms2_get_state(self.h, R.ctypes.data, q.ctypes.data, v.ctypes.data, Lg.ctypes.data, C.byref(st)))
        return R, q, v, Lg, st.value

    def set_state(self, R=None, q=None, v=None, Lang=None):
        N = self.N
        keep = [None if a is None else _f64(a, (N, n)) for a, n in ((R, 3), (q, 4), (v, 3), (Lang, 3))]
        check(lib().ms2_set_state(self.h, *[None if a is None else a.ctypes.data for a in keep]))

    def partner_counts(self):
        c = np.zeros(self.N, np.int32)
        check(lib().ms2_partner_counts(self.h, c.ctypes.data_as(_P(C.c_int))))
        return c

    def molecule_energies(self):
        out = np.zeros((self.N, 4))
        check(lib().ms2_molecule_energies(self.h, _dp(out)))
        return out

    def site_offsets(self):
        ns = C.c_int()
        check(lib().ms2_site_offsets(self.h, None, C.byref(ns)))
        out = np.zeros((self.N, ns.value, 3))
        check(lib().ms2_site_offsets(self.h, _dp(out), C.byref(ns)))
        return out

    def rdf_setup(self, r_max, n_bins, every=0):
        check(lib().ms2_rdf_setup(self.h, r_max, n_bins, every))
        self._rdf_bins = n_bins

    def rdf_sample(self):
        check(lib().ms2_rdf_sample(self.h))

    def rdf(self):
        ns, nr = C.c_int(), C.c_int()
        check(lib().ms2_rdf(self.h, None, None, C.byref(ns), C.byref(nr)))
        c = np.zeros((nr.value, self._rdf_bins), np.int64)
        g = np.zeros((nr.value, self._rdf_bins))
        check(lib().ms2_rdf(self.h, c.ctypes.data_as(_P(C.c_longlong)), _dp(g), C.byref(ns), C.byref(nr)))
        return c, g, ns.value

    def enable_timing(self, on=True):
        check(lib().ms2_enable_timing(self.h, int(on)))

    def fault_inject_barrier(self, wait_s):
        """The next fused launch's first grid barrier waits for one arrival more than
        the grid has, each wait limited to wait_s (a fault-path test)."""
        check(lib().ms2_fault_inject(self.h, 1, float(wait_s)))

    def volume_derivatives(self):
        """(dU/dV, d2U/dV2) of the current configuration (needs massieu=1 at creation)."""
        a, b = C.c_double(), C.c_double()
        check(lib().ms2_volume_derivatives(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def residence_setup(self, species_i, species_j, r_shell, every, n_lags, t_star=0):
        """Residence correlation of species_j molecules within r_shell of species_i ones."""
        check(lib().ms2_residence_setup(self.h, species_i, species_j, r_shell, every, n_lags, t_star))
        self._res_lags = n_lags

    def residence(self):
        """(correlation per lag, residence time tau, solvation number, samples)."""
        corr = np.zeros(getattr(self, "_res_lags", 1))
        tau, nsol, n = C.c_double(), C.c_double(), C.c_longlong()
        check(lib().ms2_residence(self.h, _dp(corr), C.byref(tau), C.byref(nsol), C.byref(n)))
        return corr, tau.value, nsol.value, n.value

    def conductivity_setup(self, every, n_lags):
        """Sample the electric current flux every `every` steps into an ACF of n_lags lags."""
        check(lib().ms2_conductivity_setup(self.h, every, n_lags))
        self._gk_lags = n_lags

    def current(self):
        """Electric current flux of the last sample (e A/fs)."""
        j = np.zeros(3)
        check(lib().ms2_current(self.h, _dp(j)))
        return j

    def conductivity(self):
        """(sigma in S/m, the flux ACF, number of samples)."""
        sig = C.c_double()
        acf = np.zeros(getattr(self, "_gk_lags", 1))
        n = C.c_longlong()
        check(lib().ms2_conductivity(self.h, C.byref(sig), _dp(acf), C.byref(n)))
        return sig.value, acf, n.value

    def heat_setup(self, every, n_lags, h=None):
        """Sample the heat flux J_q every `every` steps into an ACF of n_lags lags;
        h: partial molar enthalpy per species (energy units per molecule), default 0."""
        hh = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
        check(lib().ms2_heat_setup(self.h, every, n_lags, None if hh is None else _dp(hh)))
        self._hf_lags = n_lags

    def heat_flux(self):
        """Heat flux J_q of the last sample (K A/fs, energies in K)."""
        j = np.zeros(3)
        check(lib().ms2_heat_flux(self.h, _dp(j)))
        return j

    def thermal_conductivity(self):
        """(lambda in W/(m K), the heat-flux ACF, number of samples)."""
        lam = C.c_double()
        acf = np.zeros(getattr(self, "_hf_lags", 1))
        n = C.c_longlong()
        check(lib().ms2_thermal_conductivity(self.h, C.byref(lam), _dp(acf), C.byref(n)))
        return lam.value, acf, n.value

    MASSIEU_NAMES = ("A10", "A01", "A20", "A11", "A02", "A30", "A21", "A12")

    def massieu(self):
        """Residual Massieu derivatives A^r_mn from the samples since reset_averages, and their count."""
        out = np.zeros(8)
        n = C.c_longlong()
        check(lib().ms2_massieu(self.h, _dp(out), C.byref(n)))
        return dict(zip(self.MASSIEU_NAMES, out)), n.value

    def fused_step(self):
        """1 if the next chunk of steps runs as the fused cooperative kernel."""
        f = C.c_int()
        check(lib().ms2_step_kernel(self.h, C.byref(f)))
        return f.value

    def last_step_phases(self):
        """Fused step, timing on, device ms of the last step: drift, barrier, pair, reduction,
        barrier, totals, kernel entry to the last step, the whole last step, its end to exit;
        Ewald: structure-factor, sum and force task phases (else 0)."""
        out = np.zeros(12)
        check(lib().ms2_last_step_phases(self.h, _dp(out)))
        return out

    def last_step_times(self):
        """(pair kernel ms, Ewald kernels ms, whole last step ms, rest ms) of the last enqueued step;
        a fused chunk gives its pair phase and Ewald task phases (device timer) and its mean step."""
        out = np.zeros(4)
        check(lib().ms2_last_step_times(self.h, _dp(out)))
        return out

    def averages(self):
        out = np.zeros(5)
        n = C.c_longlong()
        check(lib().ms2_averages(self.h, _dp(out), C.byref(n)))
        return dict(U=out[0], P=out[1], T=out[2], U_err=out[3], P_err=out[4], n=n.value)

    def reset_averages(self):
        check(lib().ms2_reset_averages(self.h))


class Batch:
    """Many systems advanced together by the multi-system step kernels (ms2_batch_*)."""

    def __init__(self, systems):
        self.systems = list(systems)
        arr = (_vp * len(self.systems))(*[x.h for x in self.systems])
        h = _vp()
        check(lib().ms2_batch_create(arr, len(self.systems), C.byref(h)))
        self.h = h

    def step(self, n):
        check(lib().ms2_batch_step(self.h, n))

    def close(self):
        if getattr(self, "h", None):
            lib().ms2_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving front end: jobs are queued, admitted by memory budget, advanced
    together in chunks, and retired with averages and RDF (ms2_serve_*)."""

    def __init__(self, budget_bytes, max_slots=256, **opts):
        self._opts = default_options(**opts)
        h = _vp()
        check(lib().ms2_serve_open(budget_bytes, max_slots, C.byref(self._opts), C.byref(h)))
        self.h = h
        self._keep = []

    def submit(self, models, counts, T, rho, cutoff, elec, steps, arrival=0.0, seed=1, rdf_bins=0, rdf_every=10,
               R0=None, q0=None):
        m, keep = make_models(models)
        cnt = (C.c_int * len(counts))(*[int(c) for c in counts])
        n = int(sum(counts))
        R0 = None if R0 is None else np.ascontiguousarray(R0, np.float64).reshape(n, 3)
        q0 = None if q0 is None else np.ascontiguousarray(q0, np.float64).reshape(n, 4)
        self._keep.append((m, keep, cnt, R0, q0))
        j = ms2_job(models=C.cast(m, C.POINTER(ms2_model)), N_per_model=C.cast(cnt, C.POINTER(C.c_int)),
                    n_models=len(models), T=T, rho=rho, cutoff=cutoff, elec=elec, steps=steps,
                    arrival_time=arrival, seed=seed, rdf_bins=rdf_bins, rdf_every=rdf_every,
                    R0=None if R0 is None else _dp(R0), q0=None if q0 is None else _dp(q0))
        jid = C.c_longlong()
        check(lib().ms2_serve_submit(self.h, C.byref(j), C.byref(jid)))
        return jid.value

    def poll(self, max_results=64):
        arr = (ms2_job_result * max_results)()
        n = C.c_int()
        check(lib().ms2_serve_poll(self.h, arr, max_results, C.byref(n)))
        out = []
        for k in range(n.value):
            r = arr[k]
            g = np.array(r.g[:r.n_rows * r.n_bins]).reshape(r.n_rows, r.n_bins) if r.n_bins else None
            out.append(dict(job_id=r.job_id, status=r.status, U=r.U_avg, U_err=r.U_err, P=r.P_avg, P_err=r.P_err,
                            T=r.T_avg, t_arrive=r.t_arrive, t_admit=r.t_admit, t_done=r.t_done, g=g))
        return out

    def drain(self, timeout=600.0):
        check(lib().ms2_serve_drain(self.h, timeout))

    def close(self):
        if getattr(self, "h", None):
            lib().ms2_serve_close(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_launches():
    return lib().ms2_kernel_launches()
