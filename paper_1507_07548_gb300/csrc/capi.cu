// C-ABI of libms2: system lifetime, state, time stepping and outputs.
// See include/ms2.h for the contract of every entry point.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ms2.h"
#include "ms2_internal.cuh"
#include "ms2_host.h"

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};

void ms2_count_launches(long long n) { g_launches += n; }

ms2_status ms2_fail(ms2_status st, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

ms2_status ms2_fail_cuda(cudaError_t e, const char *what, const char *file, int line) {
    cudaGetLastError();
    return ms2_fail(e == cudaErrorMemoryAllocation ? MS2_ENOMEM : MS2_ECUDA, "%s failed: %s (%s:%d)", what,
                    cudaGetErrorString(e), file, line);
}

// Dynamic shared memory of a kernel: the limit is one setting per kernel and
// device, shared by every system and batch that launches the kernel, so it only
// ever rises (a small system created after a large one must not lower the limit
// the large one launches with).  A fixed table, no host allocation; if it is
// ever full, the kernel gets the largest amount the device allows.
namespace {
struct SmemMark {
    int dev;
    const void *fn;
    size_t bytes;
};
constexpr int kSmemMarks = 1024;
SmemMark g_smem_mark[kSmemMarks];
int g_smem_marks = 0;
std::mutex g_smem_mu;
}  // namespace

cudaError_t ms2_allow_smem(const void *fn, size_t bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const size_t want = std::max<size_t>(bytes, 48 * 1024);
    std::lock_guard<std::mutex> lk(g_smem_mu);
    SmemMark *m = nullptr;
    for (int k = 0; k < g_smem_marks && !m; ++k)
        if (g_smem_mark[k].fn == fn && g_smem_mark[k].dev == dev) m = &g_smem_mark[k];
    if (m && want <= m->bytes) return cudaSuccess;
    size_t set = want;
    if (!m && g_smem_marks == kSmemMarks) {  // untracked from here on: the device maximum
        int optin = 0;
        cudaFuncAttributes fa;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
        if (e != cudaSuccess) return e;
        set = std::max(want, (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0);
    }
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)set);
    if (e != cudaSuccess) return e;
    if (m) m->bytes = set;
    else if (g_smem_marks < kSmemMarks) g_smem_mark[g_smem_marks++] = SmemMark{dev, fn, set};
    return cudaSuccess;
}

extern "C" const char *ms2_last_error(void) { return g_err.c_str(); }
extern "C" long long ms2_kernel_launches(void) { return g_launches.load(); }
extern "C" const char *ms2_version(void) { return "ms2-gb300 1.0 (sm_103a)"; }

// kernels (defined in the other translation units)
__global__ void k_build(const SysParams *, DevSys);
__global__ void k_reduce(const SysParams *, DevSys, int);
__global__ void k_heat_reduce(const SysParams *, DevSys);
__global__ void k_drift(const SysParams *, DevSys, int);
__global__ void k_pair_lj64(const SysParams *, DevSys, int);
__global__ void k_ewald_skp(const SysParams *, DevSys);
__global__ void k_ewald_sksum(const SysParams *, DevSys, float2 *, int);
void *ms2_ewald_force_kernel(int kx, int kz);
size_t ms2_ewald_skp_smem(int kx, int ky, int kz, int skc);
int ms2_ewald_sk_sites(int M, int G);
int ms2_ewald_skp_blocks(int M, int skc);
int ms2_ewald_sksum_blocks(int K);
size_t ms2_ewald_force_smem(int kx, int kz, int ny_per_chunk);
__global__ void k_rdf(const SysParams *, DevSys);
__global__ void k_terms(const SysParams *, DevSys, double *);
size_t ms2_pair_smem_bytes(int NS, int tile, bool multi, int TJ, int wpb);
size_t ms2_pair64_smem_bytes(int TJ, int wpb);
void *ms2_pick_pair_kernel(int ns, unsigned ljm, unsigned qm, unsigned dm, int elec, bool multi, int *ns_used,
                           int *tile, bool *mult_used, bool mass);
void *ms2_pick_heat_kernel(int ns, unsigned ljm, unsigned qm, unsigned dm, int elec, bool multi, const void *pair_fn);


// ------------------------------------------------------------ allocation
cudaError_t DevAlloc::alloc(void **p, size_t n) {
    n = std::max<size_t>(n, 256);
    if (fa && ff) {
        *p = fa(n, ctx);
        if (!*p) return cudaErrorMemoryAllocation;
    } else {
        cudaError_t e = cudaMalloc(p, n);
        if (e != cudaSuccess) return e;
    }
    live.push_back(*p);
    bytes += n;
    return cudaSuccess;
}
void DevAlloc::release_all() {
    for (void *p : live) {
        if (fa && ff) ff(p, ctx);
        else cudaFree(p);
    }
    live.clear();
    bytes = 0;
}

// ------------------------------------------------------------- constants
void ms2_unit_constants(bool reduced, double *coulomb, double *kconv) {
    if (reduced) {
        *coulomb = 1.0;
        *kconv = 1.0;
        return;
    }
    const double e = 1.602176634e-19, eps0 = 8.8541878128e-12, kB = 1.380649e-23, NA = 6.02214076e23;
    *coulomb = e * e / (4.0 * M_PI * eps0 * kB) * 1e10;  // K * Angstrom per e^2
    *kconv = kB * NA * 1e3 * 1e20 / 1e30;                // 1 K in g/mol A^2 fs^-2
}

// ---------------------------------------------------------- seeded input
namespace {
struct SplitMix64 {  // Steele, Lea & Flood (2014) generator, as published by Vigna
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * 0x1.0p-53; }
    double normal() {  // Box-Muller
        double u1 = uniform(), u2 = uniform();
        if (u1 < 1e-300) u1 = 1e-300;
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
    }
};
}  // namespace

// ------------------------------------------------------------- validation
ms2_status ms2_validate_models(const ms2_model *models, int n_models, ms2_elec elec) {
    if (!models || n_models < 1 || n_models > MS2_MAXSP) return ms2_fail(MS2_EINVAL, "n_models must be 1..%d", MS2_MAXSP);
    bool any_q = false, any_d = false;
    int nljt = 0;
    for (int m = 0; m < n_models; ++m) {
        const ms2_model &md = models[m];
        if (md.n_sites < 1 || md.n_sites > MS2_MAXS || !md.sites)
            return ms2_fail(MS2_EINVAL, "model %d: n_sites must be 1..%d", m, MS2_MAXS);
        double M = 0, com[3] = {0, 0, 0}, ext = 0, qsum = 0, I[3][3] = {{0}};
        for (int a = 0; a < md.n_sites; ++a) {
            const ms2_site &s = md.sites[a];
            if (!(s.mass >= 0)) return ms2_fail(MS2_EINVAL, "model %d site %d: negative mass", m, a);
            M += s.mass;
            for (int k = 0; k < 3; ++k) {
                com[k] += s.mass * s.pos[k];
                ext = std::max(ext, std::fabs(s.pos[k]));
            }
            if (s.kind & MS2_SITE_LJ) {
                if (!(s.sigma >= 0 && s.epsilon >= 0)) return ms2_fail(MS2_EINVAL, "model %d site %d: bad LJ", m, a);
                ++nljt;
            }
            if ((s.kind & MS2_SITE_CHARGE) && s.charge != 0) any_q = true;
            if ((s.kind & MS2_SITE_DIPOLE) && (s.dipole[0] != 0 || s.dipole[1] != 0 || s.dipole[2] != 0)) any_d = true;
            if (s.kind & MS2_SITE_CHARGE) qsum += s.charge;
            const double r2 = s.pos[0] * s.pos[0] + s.pos[1] * s.pos[1] + s.pos[2] * s.pos[2];
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) I[r][c] += s.mass * ((r == c ? r2 : 0.0) - s.pos[r] * s.pos[c]);
        }
        if (!(M > 0)) return ms2_fail(MS2_EINVAL, "model %d: total mass must be > 0", m);
        for (int k = 0; k < 3; ++k)
            if (std::fabs(com[k]) > 1e-9 * M * std::max(ext, 1e-30))
                return ms2_fail(MS2_EINVAL, "model %d: sites not in the centre-of-mass frame", m);
        const double tr = I[0][0] + I[1][1] + I[2][2];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                if (r != c && std::fabs(I[r][c]) > 1e-9 * std::max(tr, 1e-300) && tr > 0)
                    return ms2_fail(MS2_EINVAL, "model %d: body axes are not principal axes", m);
        if (elec == MS2_ELEC_RF && std::fabs(qsum) > 1e-9)
            return ms2_fail(MS2_EINVAL, "model %d carries net charge %g: reaction field needs neutral molecules "
                                        "(use MS2_ELEC_EWALD)", m, qsum);
    }
    if (nljt > MS2_MAXT) return ms2_fail(MS2_EINVAL, "at most %d LJ sites over all models", MS2_MAXT);
    if (elec == MS2_ELEC_NONE && (any_q || any_d))
        return ms2_fail(MS2_EINVAL, "charges or dipoles present but electrostatics is MS2_ELEC_NONE");
    if (any_q && any_d) return ms2_fail(MS2_EINVAL, "charges and point dipoles in one system are not supported");
    if (any_d && elec != MS2_ELEC_RF) return ms2_fail(MS2_EINVAL, "point dipoles need MS2_ELEC_RF");
    if (elec < MS2_ELEC_NONE || elec > MS2_ELEC_EWALD) return ms2_fail(MS2_EINVAL, "unknown electrostatics %d", (int)elec);
    return MS2_OK;
}

// Fills the per-system constants from the models (host FP64).
void ms2_fill_params(SysParams &P, const ms2_model *models, int n_models, const std::vector<int> &species,
                     double L, double rc, ms2_elec elec, const ms2_options &o, double T0) {
    memset(&P, 0, sizeof P);
    const int N = (int)species.size();
    P.N = N;
    P.n_species = n_models;
    P.elec = (int)elec;
    P.integrator = o.integrator;
    P.thermostat = o.thermostat;
    P.quat_iters = o.quat_iters > 0 ? o.quat_iters : 3;
    P.L = L;
    P.V = L * L * L;
    P.dt = o.dt;
    double coulomb, kconv;
    ms2_unit_constants(o.reduced != 0, &coulomb, &kconv);
    P.kconv = kconv;
    P.T0 = T0;
    P.lat_scale = 4294967296.0 / L;
    {
        const double sc = rc * 4294967296.0 / L;
        P.rc2 = (unsigned long long)std::ceil(sc * sc);
    }
    P.lat_to_len = (float)(L / 4294967296.0);
    P.lat_to_len_lo = (float)(L / 4294967296.0 - (double)P.lat_to_len);
    P.len_to_lat = (float)(4294967296.0 / L);
    P.coulomb = (float)coulomb;
    P.coulomb_lo = (float)(coulomb - (double)P.coulomb);
    const double rc3 = rc * rc * rc;
    const bool conducting = o.eps_rf <= 0 || o.eps_rf >= 1e30;
    const double krf = conducting ? 1.0 / (2.0 * rc3) : (o.eps_rf - 1.0) / ((2.0 * o.eps_rf + 1.0) * rc3);
    P.krf = (float)krf;
    P.crf = (float)(1.0 / rc + krf * rc * rc);
    int ns = 0, t = 0, ndof = 3 * N - 3;
    double tsig[MS2_MAXT], teps[MS2_MAXT];
    int rotdof[MS2_MAXSP];
    for (int m = 0; m < n_models; ++m) {
        const ms2_model &md = models[m];
        ns = std::max(ns, md.n_sites);
        P.n_sites[m] = md.n_sites;
        double M = 0, I[3] = {0, 0, 0};
        for (int a = 0; a < MS2_MAXS; ++a) {
            P.ljt[m][a] = -1;
        }
        for (int a = 0; a < md.n_sites; ++a) {
            const ms2_site &s = md.sites[a];
            for (int k = 0; k < 3; ++k) {
                P.bpos[m][a][k] = s.pos[k];
                P.bdip[m][a][k] = (s.kind & MS2_SITE_DIPOLE) ? s.dipole[k] : 0.0;
            }
            const double qa = (s.kind & MS2_SITE_CHARGE) ? s.charge : 0.0;
            P.qd[m][a] = qa;
            P.q[m][a] = (float)qa;
            P.qlo[m][a] = (float)(qa - (double)P.q[m][a]);
            P.cq[m][a] = (float)(coulomb * qa);
            P.cqlo[m][a] = (float)(coulomb * qa - (double)P.cq[m][a]);
            if (s.kind & MS2_SITE_LJ) {
                P.ljt[m][a] = t;
                tsig[t] = s.sigma;
                teps[t] = s.epsilon;
                ++t;
            }
            M += s.mass;
            I[0] += s.mass * (s.pos[1] * s.pos[1] + s.pos[2] * s.pos[2]);
            I[1] += s.mass * (s.pos[0] * s.pos[0] + s.pos[2] * s.pos[2]);
            I[2] += s.mass * (s.pos[0] * s.pos[0] + s.pos[1] * s.pos[1]);
        }
        P.mass[m] = M;
        const double mx = std::max(I[0], std::max(I[1], I[2]));
        rotdof[m] = 0;
        for (int k = 0; k < 3; ++k) {
            P.Iinv[m][k] = (mx > 0 && I[k] > 1e-12 * mx) ? 1.0 / I[k] : 0.0;
            rotdof[m] += P.Iinv[m][k] != 0.0;
        }
    }
    for (int i = 0; i < N; ++i) ndof += rotdof[species[i]];
    P.ndof = ndof;
    P.inv_kconv = 1.0 / kconv;
    P.inv_ndof = 1.0 / ndof;
    P.inv_V = 1.0 / P.V;
    P.inv_T0 = T0 > 0 ? 1.0 / T0 : 0.0;
    for (int m = 0; m < n_models; ++m) P.inv_mass[m] = 1.0 / P.mass[m];
    P.dtk = P.dt * P.kconv;
    for (int m = 0; m < n_models; ++m) {
        P.kick[m] = P.dtk * P.inv_mass[m];
        P.half_mass[m] = 0.5 * P.mass[m];
        for (int k = 0; k < 3; ++k) P.half_Iinv[m][k] = 0.5 * P.Iinv[m][k];
    }
    P.lam_c = 2.0 * P.inv_kconv * P.inv_ndof * P.inv_T0;
    for (int m = 0; m < MS2_MAXSP; ++m) {
        P.qmol[m] = 0.0;
        if (m < n_models)
            for (int a = 0; a < models[m].n_sites; ++a) P.qmol[m] += models[m].sites[a].charge;
    }
    P.ns = ns;
    P.n_ljt = t;
    for (int a = 0; a < t; ++a)
        for (int b = 0; b < t; ++b) {
            const double sg = 0.5 * (tsig[a] + tsig[b]), ep = std::sqrt(teps[a] * teps[b]);
            const double s6 = std::pow(sg, 6.0);
            P.c6d[a][b] = 4.0 * ep * s6;
            P.c12d[a][b] = 4.0 * ep * s6 * s6;
            P.c6[a][b] = (float)P.c6d[a][b];
            P.c12[a][b] = (float)P.c12d[a][b];
            P.c6lo[a][b] = (float)(P.c6d[a][b] - (double)P.c6[a][b]);
            P.c12lo[a][b] = (float)(P.c12d[a][b] - (double)P.c12[a][b]);
        }
    P.multi = n_models > 1;
    bool any_d = false;
    for (int m = 0; m < n_models; ++m)
        for (int a = 0; a < models[m].n_sites; ++a)
            if (P.bdip[m][a][0] != 0 || P.bdip[m][a][1] != 0 || P.bdip[m][a][2] != 0) any_d = true;
    P.has_dipole = any_d;
    // Close-contact LJ pairs in double-float where point charges make the
    // molecular virial a small difference of large LJ and Coulomb sums (liquid
    // water at ambient pressure: |W| ~ 1/25 of its LJ part); without charges the
    // FP32 terms meet the same relative bound and the pass is off.
    {
        bool any_q = false;
        for (int m = 0; m < n_models; ++m)
            for (int a = 0; a < models[m].n_sites; ++a) any_q = any_q || P.qd[m][a] != 0.0;
        P.close_k6 = any_q ? (float)std::pow(1.1, -6.0) : INFINITY;
    }
    for (int m = 0; m < MS2_MAXSP; ++m) {
        P.rot[m] = m < n_models && (P.Iinv[m][0] != 0 || P.Iinv[m][1] != 0 || P.Iinv[m][2] != 0);
        bool pt = m < n_models;
        for (int a = 0; pt && a < models[m].n_sites; ++a)
            for (int k = 0; k < 3; ++k) pt = pt && P.bpos[m][a][k] == 0.0 && P.bdip[m][a][k] == 0.0;
        P.point[m] = pt;
    }
    P.massieu = o.massieu != 0;
}

// Ewald constants (self, intramolecular, background) and the LJ long-range
// correction (site-site homogeneous form), host FP64.
void ms2_energy_constants(const SysParams &P, const std::vector<int> &species, double alpha, double rc,
                          bool lrc, double coulomb, double *uconst, double *wbg, double *ulrc, double *plrc) {
    const int N = (int)species.size();
    int cnt[MS2_MAXSP] = {0};
    for (int i = 0; i < N; ++i) cnt[species[i]]++;
    double c = 0, w = 0;
    if (P.elec == ELEC_EWALD) {
        double sq2 = 0, Q = 0, intra = 0;
        for (int m = 0; m < P.n_species; ++m) {
            double ms = 0, mq = 0, mi = 0;
            for (int a = 0; a < P.n_sites[m]; ++a) {
                const double qa = P.q[m][a];
                ms += qa * qa;
                mq += qa;
                for (int b = a + 1; b < P.n_sites[m]; ++b) {
                    const double qb = P.q[m][b];
                    if (qa == 0 || qb == 0) continue;
                    double d2 = 0;
                    for (int k = 0; k < 3; ++k) d2 += (P.bpos[m][b][k] - P.bpos[m][a][k]) * (P.bpos[m][b][k] - P.bpos[m][a][k]);
                    const double r = std::sqrt(d2);
                    mi += qa * qb * std::erf(alpha * r) / r;
                }
            }
            sq2 += cnt[m] * ms;
            Q += cnt[m] * mq;
            intra += cnt[m] * mi;
        }
        const double ubg = -M_PI * coulomb * Q * Q / (2.0 * P.V * alpha * alpha);
        c = -coulomb * alpha / std::sqrt(M_PI) * sq2 - coulomb * intra + ubg;
        w = 3.0 * ubg;
    }
    *uconst = c;
    *wbg = w;
    double u = 0, p = 0;
    if (lrc) {
        for (int m1 = 0; m1 < P.n_species; ++m1)
            for (int a = 0; a < P.n_sites[m1]; ++a)
                for (int m2 = 0; m2 < P.n_species; ++m2)
                    for (int b = 0; b < P.n_sites[m2]; ++b) {
                        const int ta = P.ljt[m1][a], tb = P.ljt[m2][b];
                        if (ta < 0 || tb < 0) continue;
                        // c6 = 4 eps sig^6, c12 = 4 eps sig^12
                        const double c6 = P.c6d[ta][tb], c12 = P.c12d[ta][tb];
                        const double r3 = rc * rc * rc, r9 = r3 * r3 * r3;
                        const double Iu = c12 / (9.0 * r9) - c6 / (3.0 * r3);             // int r^2 u
                        const double Ip = -12.0 * c12 / (9.0 * r9) + 6.0 * c6 / (3.0 * r3);  // int r^3 u'
                        const double nn = (double)cnt[m1] * cnt[m2];
                        u += nn * Iu;
                        p += nn * Ip;
                    }
    }
    *ulrc = 2.0 * M_PI / P.V * u;
    *plrc = -2.0 * M_PI / (3.0 * P.V * P.V) * p;
}

// ------------------------------------------------------------------ system
static ms2_status sys_alloc(ms2_system s) {
    const int N = s->N, NS = s->ns;
    DevSys &d = s->d;
    memset(&d, 0, sizeof d);
    d.N = N;
    d.ns = NS;
    d.jsplit = s->jsplit;
    auto A = [&](void **p, size_t n) { return s->al.alloc(p, n); };
    MS2_CUDA_OK(A((void **)&s->dP, sizeof(SysParams)));
    // R, q, v, Lm back to back: a state upload is one copy
    MS2_CUDA_OK(A((void **)&d.R, sizeof(double) * 13 * N));
    d.q = d.R + 3 * (size_t)N;
    d.v = d.q + 4 * (size_t)N;
    d.Lm = d.v + 3 * (size_t)N;
    MS2_CUDA_OK(A((void **)&d.species, sizeof(int) * N));
    MS2_CUDA_OK(A((void **)&d.X, sizeof(uint32_t) * 3 * N));
    MS2_CUDA_OK(A((void **)&d.s, sizeof(float) * 3 * NS * N));
    if (s->hp.has_dipole) MS2_CUDA_OK(A((void **)&d.mu, sizeof(float) * 3 * NS * N));
    if (s->hp.elec == ELEC_RF) MS2_CUDA_OK(A((void **)&d.mum, sizeof(float) * 3 * N));
    if (s->fp64) MS2_CUDA_OK(A((void **)&d.part64, sizeof(double) * s->jsplit * MS2_NPV * N));
    else MS2_CUDA_OK(A((void **)&d.part, sizeof(float) * s->jsplit * MS2_NPV * N));
    MS2_CUDA_OK(A((void **)&d.F, sizeof(double) * 3 * N));
    MS2_CUDA_OK(A((void **)&d.tau, sizeof(double) * 3 * N));
    MS2_CUDA_OK(A((void **)&d.Ui, sizeof(double) * 4 * N));
    MS2_CUDA_OK(A((void **)&d.npart, sizeof(int) * N));
    d.nunits = s->nunits;  // reduction units: one warp each, a quad of lanes per molecule
    MS2_CUDA_OK(A((void **)&d.terms, sizeof(double) * 8));
    if (s->hp.elec == ELEC_EWALD) MS2_CUDA_OK(A((void **)&d.wcorr, sizeof(double) * N));
    MS2_CUDA_OK(A((void **)&d.blk, sizeof(double) * MS2_NRED * d.nunits));
    MS2_CUDA_OK(A((void **)&d.counter, 256));
    MS2_CUDA_OK(A((void **)&d.scal, sizeof(double) * SC_COUNT_));
    MS2_CUDA_OK(A((void **)&d.acc, sizeof(double) * AC_COUNT_));
    MS2_CUDA_OK(A((void **)&d.rdf_kind, sizeof(int) * MS2_MAXSP * MS2_MAXS));
    MS2_CUDA_OK(cudaMemsetAsync(d.counter, 0, 256, s->stream));
    MS2_CUDA_OK(cudaMemsetAsync(d.scal, 0, sizeof(double) * SC_COUNT_, s->stream));
    MS2_CUDA_OK(cudaMemsetAsync(d.acc, 0, sizeof(double) * AC_COUNT_, s->stream));
    return MS2_OK;
}

static void pick_launch_shape(ms2_system s) {
    const int N = s->N;
    // pair kernel: warps own molecules; ~2 resident blocks of 8 warps per SM:
    // split the j loop only as far as the grid still fits one wave (a partial
    // second wave costs a whole wave)
    s->wpb = 8;
    const int iblocks = (N + s->wpb - 1) / s->wpb;
    s->jsplit = std::max(1, std::min(8, (s->sms * 2) / std::max(iblocks, 1)));
    s->nunits = (N + 7) / 8;  // reduction units of 8 molecules
    if (s->fuse_fn) {         // the fused decomposition (see setup_fused)
        s->jsplit = std::max(1, std::min(8, 16 / s->mcap));
        s->nunits = s->step_grid;
    }
    if (s->tune_jsplit > 0) s->jsplit = s->tune_jsplit;
    if (s->tune_wpb > 0) s->wpb = s->tune_wpb;
}

static ms2_status upload_params(ms2_system s) {
    MS2_CUDA_OK(cudaMemcpyAsync(s->dP, &s->hp, sizeof(SysParams), cudaMemcpyHostToDevice, s->stream));
    double sc[SC_COUNT_];
    memset(sc, 0, sizeof sc);
    sc[SC_UCONST] = s->uconst;
    sc[SC_PLRC] = s->plrc;
    sc[SC_ULRC] = s->ulrc;
    sc[SC_WBG] = s->wbg;
    sc[SC_LAMBDA] = 1.0;
    // only the constant slots are written here; the others keep their values
    MS2_CUDA_OK(cudaMemcpyAsync(s->d.scal + SC_UCONST, sc + SC_UCONST, sizeof(double) * 4, cudaMemcpyHostToDevice,
                                s->stream));
    return MS2_OK;
}

static ms2_status setup_pair(ms2_system s) {
    const SysParams &P = s->hp;
    unsigned ljm = 0, qm = 0, dm = 0;
    for (int m = 0; m < P.n_species; ++m)
        for (int a = 0; a < P.n_sites[m]; ++a) {
            if (P.ljt[m][a] >= 0) ljm |= 1u << a;
            if (P.q[m][a] != 0.f) qm |= 1u << a;
            if (P.bdip[m][a][0] != 0 || P.bdip[m][a][1] != 0 || P.bdip[m][a][2] != 0) dm |= 1u << a;
        }
    s->ljm = ljm;
    s->qm = qm;
    s->dm = dm;
    if (s->fp64) {
        s->ns = 1;
        s->pair_fn = (void *)&k_pair_lj64;
        s->tile = 0;
        s->multi_used = false;
    } else {
        s->pair_fn = ms2_pick_pair_kernel(P.ns, ljm, qm, dm, P.elec, P.multi != 0, &s->ns, &s->tile, &s->multi_used,
                                          P.massieu != 0);
    }
    s->hp.ns = s->ns;
    return MS2_OK;
}

static ms2_status size_pair_tiles(ms2_system s) {
    const int N = s->N;
    const int range = (N + s->jsplit - 1) / s->jsplit;
    const size_t cap = 96 * 1024;
    int TJ = std::max(32, range);
    auto bytes = [&](int tj) {
        return s->fp64 ? ms2_pair64_smem_bytes(tj, s->wpb) : ms2_pair_smem_bytes(s->ns, s->tile, s->multi_used, tj, s->wpb);
    };
    while (bytes(TJ) > cap && TJ > 64) TJ = (TJ + 1) / 2;
    s->TJ = TJ;
    s->pair_smem = bytes(TJ);
    MS2_CUDA_OK(ms2_allow_smem((const void *)s->pair_fn, s->pair_smem));
    return MS2_OK;
}

// reciprocal-space scratch of a fused block for the system's current k range (0 without Ewald)
static size_t step_ews(ms2_system s) {
    return s->hp.elec == ELEC_EWALD ? ms2_step_ewald_scratch(s->d.kx, s->d.ky, s->d.kz, s->ny_per_chunk, s->d.sk_sites) : 0;
}

// fused step: a system is fusable where a variant exists, the device launches
// cooperative kernels, every block owns at most 32 molecules (above 16 a block's
// warps take two pair items each, j-split 1) and the whole system plus the own
// region fits one SM's shared memory.  A fusable system gets the fused
// decomposition (reduction units = the grid's block ranges, j-split 16 /
// molecules per block, at least 1) on both
// paths, so fused and per-phase chunks agree bit for bit; ms2_options.fused_step
// only chooses which path runs.
static void setup_fused(ms2_system s, const ms2_options &o) {
    s->fuse_fn = s->step_fn = nullptr;
    if (s->fp64 || s->hp.integrator == MS2_INT_VERLET) return;
    void *fn = ms2_pick_step_kernel(s->ns, s->ljm, s->qm, s->dm, s->hp.elec, s->multi_used, s->hp.massieu != 0, false);
    if (!fn) return;
    int coop = 0, sms = 0, optin = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->device) != cudaSuccess || !coop) return;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
    const int mcap = (s->N + sms - 1) / std::max(sms, 1);
    if (sms < 1 || mcap > 32) return;  // (the whole-system tile must fit one block as well)
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const int js = std::max(1, std::min(8, 16 / mcap));
    const int Np = (s->N + 3) & ~3;
    const size_t maxdyn = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    // Ewald: the reciprocal-space scratch of the default |n| <= 8 (ms2_ewald_params may change it later;
    // a launch that then does not fit takes the per-phase kernels)
    const size_t ews = s->hp.elec == ELEC_EWALD ? ms2_step_ewald_scratch(8, 8, 8, 1, ms2_ewald_sk_sites(s->N * s->ns, sms)) : 0;
    const size_t base = ms2_step_smem_bytes(s->ns, s->tile, s->multi_used, Np, mcap, js, 0, ews);
    int nb = 0;
    if (base > maxdyn || ms2_allow_smem(fn, maxdyn) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, ms2_step_threads(), base) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        return;
    }
    s->fuse_fn = fn;
    s->step_fn = o.fused_step ? fn : nullptr;
    s->step_grid = sms;
    s->Np = Np;
    s->mcap = mcap;
    s->step_smem_max = maxdyn;
}

// ------------------------------------------------------------ launchers
ms2_status launch_build(ms2_system s) {
    const int th = 128;  // 4 lanes per molecule
    k_build<<<(4 * s->N + th - 1) / th, th, 0, s->stream>>>(s->dP, s->d);
    s->launch_acc += 1;
    return MS2_OK;
}

ms2_status launch_pair(ms2_system s) {
    dim3 grid((s->N + s->wpb - 1) / s->wpb, s->jsplit);
    void (*fn)(const SysParams *, DevSys, int) = (void (*)(const SysParams *, DevSys, int))s->pair_fn;
    fn<<<grid, s->wpb * 32, s->pair_smem, s->stream>>>(s->dP, s->d, s->TJ);
    s->launch_acc += 1;
    return MS2_OK;
}

ms2_status launch_ewald(ms2_system s) {
    if (s->hp.elec != ELEC_EWALD) return MS2_OK;
    DevSys &d = s->d;
    const int K = (2 * d.ky + 1) * (2 * d.kz + 1) * (d.kx + 1), nb = ms2_ewald_skp_blocks(d.nsite_q, d.sk_sites);
    k_ewald_skp<<<nb, 320, ms2_ewald_skp_smem(d.kx, d.ky, d.kz, d.sk_sites), s->stream>>>(s->dP, d);
    k_ewald_sksum<<<ms2_ewald_sksum_blocks(K), 1024, 0, s->stream>>>(s->dP, d, s->AS, nb);
    {
        void (*fk)(const SysParams *, DevSys, const float2 *, int) =
            (void (*)(const SysParams *, DevSys, const float2 *, int))ms2_ewald_force_kernel(d.kx, d.kz);
        fk<<<dim3((d.nsite_q + 127) / 128, d.kchunks), 128, ms2_ewald_force_smem(d.kx, d.kz, s->ny_per_chunk),
             s->stream>>>(s->dP, d, s->AS, s->ny_per_chunk);
    }
    s->launch_acc += 3;
    return MS2_OK;
}

ms2_status launch_reduce(ms2_system s, int mode) {
    if (s->fp64) mode |= RED_FP64PART;
    if (s->hp.elec == ELEC_EWALD) mode |= RED_EWALD;
    if (s->hp.integrator != MS2_INT_VERLET) mode |= RED_LAMBDA;
    k_reduce<<<(s->d.nunits + 3) / 4, 128, 0, s->stream>>>(s->dP, s->d, mode);
    s->launch_acc += 1;
    return MS2_OK;
}

// heat-flux pass of a sampled step (after launch_reduce): the pair decomposition
ms2_status launch_heat(ms2_system s) {
    dim3 grid((s->N + s->wpb - 1) / s->wpb, s->jsplit);
    void (*fn)(const SysParams *, DevSys, int) = (void (*)(const SysParams *, DevSys, int))s->heat_fn;
    fn<<<grid, s->wpb * 32, s->pair_smem, s->stream>>>(s->dP, s->d, s->TJ);
    k_heat_reduce<<<(s->d.nunits + 3) / 4, 128, 0, s->stream>>>(s->dP, s->d);
    s->launch_acc += 2;
    return MS2_OK;
}

ms2_status launch_drift(ms2_system s) {
    const int th = 128;  // 4 lanes per molecule
    k_drift<<<(4 * s->N + th - 1) / th, th, 0, s->stream>>>(s->dP, s->d, s->hp.integrator == MS2_INT_VERLET ? 1 : 0);
    s->launch_acc += 1;
    return MS2_OK;
}

ms2_status launch_rdf(ms2_system s) {
    const int rows = s->d.rdf_rows, nb = s->d.rdf_bins;
    const int blocks = std::min(s->N, 2 * s->sms);
    k_rdf<<<blocks, 256, sizeof(unsigned) * rows * nb, s->stream>>>(s->dP, s->d);
    s->launch_acc += 1;
    return MS2_OK;
}

static void flush_launches(ms2_system s) {
    ms2_count_launches(s->launch_acc);
    s->launch_acc = 0;
}

// forces/energies of the current configuration (no integration)
ms2_status ms2_eval_forces(ms2_system s) {
    launch_build(s);
    launch_pair(s);
    launch_ewald(s);
    launch_reduce(s, RED_SUM);
    flush_launches(s);
    MS2_CUDA_OK(cudaGetLastError());
    return MS2_OK;
}

// enqueue n steps starting at step counter s0 (no host sync)
static void enqueue_steps(ms2_system s, long long n, long long s0) {
    const bool verlet = s->hp.integrator == MS2_INT_VERLET;
    const int every = s->rdf_every;
    for (long long k = 0; k < n; ++k) {
        const bool sample = every > 0 && ((s0 + k + 1) % every) == 0;
        const bool gk = s->d.gk && s->gk_every > 0 && ((s0 + k + 1) % s->gk_every) == 0;
        const bool res = s->res_every > 0 && ((s0 + k + 1) % s->res_every) == 0;
        const bool hf = s->hf_every > 0 && ((s0 + k + 1) % s->hf_every) == 0;
        const bool tm = s->timing && k == n - 1;
        if (tm) cudaEventRecordWithFlags(s->ev[0], s->stream, cudaEventRecordExternal);
        launch_drift(s);
        if (sample) launch_rdf(s);
        if (res) {
            ms2_launch_residence(s->stream, s->dP, s->d, s->res);
            s->launch_acc += 2;
        }
        if (tm) cudaEventRecordWithFlags(s->ev[1], s->stream, cudaEventRecordExternal);
        launch_pair(s);
        if (tm) cudaEventRecordWithFlags(s->ev[2], s->stream, cudaEventRecordExternal);
        launch_ewald(s);
        if (tm) cudaEventRecordWithFlags(s->ev[3], s->stream, cudaEventRecordExternal);
        launch_reduce(s, (verlet ? (RED_SUM | RED_RECORD | RED_HALFKICK) : (RED_SUM | RED_RECORD)) | (gk ? RED_GK : 0));
        if (hf) launch_heat(s);
        if (tm) cudaEventRecordWithFlags(s->ev[4], s->stream, cudaEventRecordExternal);
    }
}

static ms2_status run_graph(ms2_system s, long long n, long long s0) {
    const int phase = s->rdf_every > 0 ? (int)(s0 % s->rdf_every) : 0;
    const int gphase = (s->d.gk && s->gk_every > 0) ? (int)(s0 % s->gk_every) : -1;
    const int rphase = s->res_every > 0 ? (int)(s0 % s->res_every) : -1;
    const int hphase = s->hf_every > 0 ? (int)(s0 % s->hf_every) : -1;
    const auto key = std::make_tuple((int)n, phase, gphase, rphase, hphase);
    auto it = s->graphs.find(key);
    if (it == s->graphs.end()) {
        if (s->graphs.size() > 16) {
            for (auto &g : s->graphs) cudaGraphExecDestroy(g.second.exec);
            s->graphs.clear();
        }
        cudaGraph_t g;
        s->launch_acc = 0;
        MS2_CUDA_OK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
        enqueue_steps(s, n, s0);
        const long long nodes = s->launch_acc;
        s->launch_acc = 0;
        MS2_CUDA_OK(cudaStreamEndCapture(s->stream, &g));
        cudaGraphExec_t ex;
        cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        MS2_CUDA_OK(e);
        it = s->graphs.emplace(key, GraphEntry{ex, nodes}).first;
    }
    MS2_CUDA_OK(cudaGraphLaunch(it->second.exec, s->stream));
    ms2_count_launches(it->second.nodes);
    return MS2_OK;
}

// ------------------------------------------------------------- C ABI
extern "C" ms2_status ms2_default_options(ms2_options *o) {
    if (!o) return ms2_fail(MS2_EINVAL, "null options");
    memset(o, 0, sizeof *o);
    o->eps_rf = 0.0;
    o->lrc = 1;
    o->dt = 2.0;
    o->thermostat = 1;
    o->seed = 1;
    o->integrator = MS2_INT_LEAPFROG_Q;
    o->quat_iters = 3;
    o->graph_chunk = 50;
    o->fused_step = 1;
    return MS2_OK;
}

// seeded lattice start (see ms2.h)
static void initial_state(ms2_system s, const ms2_model *models, double T, unsigned long long seed) {
    const int N = s->N;
    const SysParams &P = s->hp;
    SplitMix64 rng{seed * 0x2545F4914F6CDD1DULL + 0x1234567ULL};
    std::vector<double> &R = s->hR, &q = s->hq, &v = s->hv, &L = s->hL;
    R.assign(3 * N, 0);
    q.assign(4 * N, 0);
    v.assign(3 * N, 0);
    L.assign(3 * N, 0);
    const double Lb = P.L;
    bool point = true;
    for (int m = 0; m < P.n_species; ++m)
        if (P.Iinv[m][0] != 0 || P.Iinv[m][1] != 0 || P.Iinv[m][2] != 0) point = false;
    int mc = (int)std::round(std::cbrt(N / 4.0));
    std::vector<double> pts;
    if (point && P.n_species == 1 && 4 * mc * mc * mc == N) {
        const double a = Lb / mc, bas[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};
        for (int x = 0; x < mc; ++x)
            for (int y = 0; y < mc; ++y)
                for (int z = 0; z < mc; ++z)
                    for (int b = 0; b < 4; ++b) {
                        pts.push_back((x + bas[b][0]) * a);
                        pts.push_back((y + bas[b][1]) * a);
                        pts.push_back((z + bas[b][2]) * a);
                    }
    } else {
        int m = (int)std::ceil(std::cbrt((double)N) - 1e-9);
        while (m * m * m < N) ++m;
        const double a = Lb / m;
        for (int x = 0; x < m; ++x)
            for (int y = 0; y < m; ++y)
                for (int z = 0; z < m; ++z) {
                    pts.push_back((x + 0.5) * a);
                    pts.push_back((y + 0.5) * a);
                    pts.push_back((z + 0.5) * a);
                }
    }
    const int npts = (int)pts.size() / 3;
    std::vector<int> perm(npts);
    for (int k = 0; k < npts; ++k) perm[k] = k;
    if (P.n_species > 1)  // mix species over the lattice (Fisher-Yates)
        for (int k = npts - 1; k > 0; --k) std::swap(perm[k], perm[(int)(rng.uniform() * (k + 1))]);
    double ke = 0, mom[3] = {0, 0, 0}, Mt = 0;
    for (int i = 0; i < N; ++i) {
        const int sp = s->species[i];
        for (int k = 0; k < 3; ++k) R[3 * i + k] = pts[3 * perm[i] + k];
        const bool rot = P.Iinv[sp][0] != 0 || P.Iinv[sp][1] != 0 || P.Iinv[sp][2] != 0;
        if (rot) {  // Shoemake uniform rotation
            const double u1 = rng.uniform(), u2 = rng.uniform(), u3 = rng.uniform();
            const double a = std::sqrt(1 - u1), b = std::sqrt(u1);
            q[4 * i] = a * std::sin(2 * M_PI * u2);
            q[4 * i + 1] = a * std::cos(2 * M_PI * u2);
            q[4 * i + 2] = b * std::sin(2 * M_PI * u3);
            q[4 * i + 3] = b * std::cos(2 * M_PI * u3);
        } else {
            q[4 * i] = 1.0;
        }
        const double M = P.mass[sp];
        for (int k = 0; k < 3; ++k) {
            v[3 * i + k] = rng.normal() * std::sqrt(T * P.kconv / M);
            mom[k] += M * v[3 * i + k];
        }
        Mt += M;
        double A[9];
        {
            const double w = q[4 * i], x = q[4 * i + 1], y = q[4 * i + 2], z = q[4 * i + 3];
            A[0] = 1 - 2 * (y * y + z * z); A[1] = 2 * (x * y - w * z); A[2] = 2 * (x * z + w * y);
            A[3] = 2 * (x * y + w * z); A[4] = 1 - 2 * (x * x + z * z); A[5] = 2 * (y * z - w * x);
            A[6] = 2 * (x * z - w * y); A[7] = 2 * (y * z + w * x); A[8] = 1 - 2 * (x * x + y * y);
        }
        double lb[3] = {0, 0, 0};
        for (int k = 0; k < 3; ++k)
            if (P.Iinv[sp][k] != 0) {
                lb[k] = rng.normal() * std::sqrt(T * P.kconv / P.Iinv[sp][k]);
                ke += 0.5 * lb[k] * lb[k] * P.Iinv[sp][k];
            }
        for (int r = 0; r < 3; ++r) L[3 * i + r] = A[3 * r] * lb[0] + A[3 * r + 1] * lb[1] + A[3 * r + 2] * lb[2];
    }
    for (int i = 0; i < N; ++i) {
        const double M = P.mass[s->species[i]];
        for (int k = 0; k < 3; ++k) {
            v[3 * i + k] -= mom[k] / Mt;
            ke += 0.5 * M * v[3 * i + k] * v[3 * i + k];
        }
    }
    const double Tk = 2.0 * ke / P.kconv / P.ndof, lam = (Tk > 0 && T > 0) ? std::sqrt(T / Tk) : 0.0;
    for (int k = 0; k < 3 * N; ++k) {
        v[k] *= lam;
        L[k] *= lam;
    }
}

static ms2_status ensure_pinned(ms2_system s) {
    if (!s->pinned) MS2_CUDA_OK(cudaMallocHost((void **)&s->pinned, sizeof(double) * 39 * s->N));
    for (int k = 0; k < 2; ++k)
        if (!s->up_ev[k]) MS2_CUDA_OK(cudaEventCreateWithFlags(&s->up_ev[k], cudaEventDisableTiming));
    return MS2_OK;
}

// host state -> device, through the upload buffer whose previous copy has ended;
// returns without waiting for this copy
static ms2_status upload_state(ms2_system s) {
    const int N = s->N;
    ms2_status st = ensure_pinned(s);
    if (st != MS2_OK) return st;
    const int k = s->up_k;
    MS2_CUDA_OK(cudaEventSynchronize(s->up_ev[k]));
    double *buf = s->pinned + (size_t)13 * N * k;
    size_t off = 0;
    auto put = [&](const std::vector<double> &src, int nc) {  // AoS -> the device SoA order
        double *b = buf + off;
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < nc; ++k) b[k * N + i] = src[nc * i + k];
        off += (size_t)nc * N;
    };
    put(s->hR, 3);
    put(s->hq, 4);
    put(s->hv, 3);
    put(s->hL, 3);
    // the device arrays R, q, v, Lm are contiguous in this order (sys_alloc)
    MS2_CUDA_OK(cudaMemcpyAsync(s->d.R, buf, sizeof(double) * 13 * N, cudaMemcpyHostToDevice, s->stream));
    MS2_CUDA_OK(cudaEventRecord(s->up_ev[k], s->stream));
    s->up_k = 1 - k;
    return MS2_OK;
}

// forces, energies and site build of the current state (after ms2_set_state)
ms2_status ms2_ensure_forces(ms2_system s) {
    if (!s->stale) return MS2_OK;
    ms2_status st = ms2_eval_forces(s);
    if (st == MS2_OK) s->stale = false;
    return st;
}

static ms2_status setup_ewald(ms2_system s, double alpha, int kx, int ky, int kz) {
    DevSys &d = s->d;
    // the splitting parameter is its FP32 value in every part (real space, k-space
    // tables, self and intramolecular terms): exact in the kernels' FP32 arithmetic
    alpha = (double)(float)alpha;
    s->alpha = alpha;
    s->hp.alpha = (float)alpha;
    {
        const double tasp = 2.0 * alpha / std::sqrt(M_PI);
        s->hp.two_alpha_sqrtpi = (float)tasp;
        s->hp.two_alpha_sqrtpi_lo = (float)(tasp - (double)s->hp.two_alpha_sqrtpi);
    }
    d.kx = kx;
    d.ky = ky;
    d.kz = kz;
    d.nsite_q = s->N * s->ns;
    const int M = d.nsite_q, kst = std::max(kx, std::max(ky, kz)) + 1;
    d.kchunks = 2 * ky + 1;
    s->ny_per_chunk = 1;
    const int cols = (2 * ky + 1) * (2 * kz + 1), K = cols * (kx + 1);
    auto A = [&](void **p, size_t n) { return s->al.alloc(p, n); };
    // (re)allocation: old buffers stay owned by the allocator list until destroy
    MS2_CUDA_OK(A((void **)&d.qs, sizeof(float) * M));
    MS2_CUDA_OK(A((void **)&d.eik, sizeof(float2) * 3 * kst * M));
    MS2_CUDA_OK(A((void **)&d.frec, sizeof(float) * d.kchunks * 3 * M));
    // sites per structure-factor task: one round over the fused grid (the same on both paths)
    d.sk_sites = ms2_ewald_sk_sites(M, s->step_grid > 0 ? s->step_grid : s->sms);
    {
        const double C64 = (double)s->hp.coulomb + (double)s->hp.coulomb_lo;  // C to ~48 bits
        const double fpre = 8.0 * 3.141592653589793 * C64 / s->hp.V * 2.0 * 3.141592653589793 / s->hp.L;
        d.ew_fpre = (float)fpre;
        d.ew_fpre_lo = (float)(fpre - (double)d.ew_fpre);
    }
    MS2_CUDA_OK(A((void **)&d.skpart, sizeof(float2) * (size_t)ms2_ewald_skp_blocks(M, d.sk_sites) * K));
    MS2_CUDA_OK(A((void **)&d.kblk, sizeof(double) * 2 * ms2_ewald_sksum_blocks(K)));
    MS2_CUDA_OK(A((void **)&s->AS, sizeof(float2) * K));
    {  // the k-space tables of this box and alpha (k = (col, nx) with col = (ny + ky)(2 kz + 1) + nz + kz)
        std::vector<double> Ak(K), Bk(K);
        const double tw = 2.0 * M_PI / s->hp.L, ia2 = 1.0 / (alpha * alpha);
        for (int k = 0; k < K; ++k) {
            const int col = k / (kx + 1), nx = k % (kx + 1);
            const int ny = col / (2 * kz + 1) - ky, nz = col % (2 * kz + 1) - kz;
            const bool on = nx > 0 || ny > 0 || (ny == 0 && nz > 0);  // the half space
            const double kk = tw * tw * ((double)nx * nx + (double)ny * ny + (double)nz * nz);
            Ak[k] = on ? std::exp(-0.25 * kk * ia2) / kk : 0.0;
            Bk[k] = Ak[k] * (1.0 - 0.5 * kk * ia2);
        }
        MS2_CUDA_OK(A((void **)&d.Ak, sizeof(double) * K));
        MS2_CUDA_OK(A((void **)&d.Bk, sizeof(double) * K));
        MS2_CUDA_OK(cudaMemcpyAsync(d.Ak, Ak.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s->stream));
        MS2_CUDA_OK(cudaMemcpyAsync(d.Bk, Bk.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s->stream));
        MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    }
    {
        const size_t sm = ms2_ewald_skp_smem(kx, ky, kz, d.sk_sites), fm = ms2_ewald_force_smem(kx, kz, s->ny_per_chunk);
        MS2_CUDA_OK(ms2_allow_smem((const void *)k_ewald_skp, sm));
        MS2_CUDA_OK(ms2_allow_smem(ms2_ewald_force_kernel(kx, kz), fm));
    }
    double coulomb, kconv;
    ms2_unit_constants(s->reduced, &coulomb, &kconv);
    ms2_energy_constants(s->hp, s->species, alpha, s->rc, s->lrc, coulomb, &s->uconst, &s->wbg, &s->ulrc, &s->plrc);
    return MS2_OK;
}

static void destroy_graphs(ms2_system s) {
    for (auto &g : s->graphs) cudaGraphExecDestroy(g.second.exec);
    s->graphs.clear();
}

extern "C" ms2_status ms2_create_system(const ms2_model *models, const int *N_per_model, int n_models, double box,
                                        double T, double rho, double cutoff, ms2_elec elec, const ms2_options *opt,
                                        ms2_system *out) {
    if (!out) return ms2_fail(MS2_EINVAL, "null output handle");
    *out = nullptr;
    ms2_status st = ms2_validate_models(models, n_models, elec);
    if (st != MS2_OK) return st;
    if (!N_per_model) return ms2_fail(MS2_EINVAL, "null N_per_model");
    long long Nt = 0;
    for (int m = 0; m < n_models; ++m) {
        if (N_per_model[m] < 0) return ms2_fail(MS2_EINVAL, "negative molecule count");
        Nt += N_per_model[m];
    }
    if (Nt < 2 || Nt > (1 << 24)) return ms2_fail(MS2_EINVAL, "total molecule count %lld outside 2..2^24", Nt);
    ms2_options o;
    ms2_default_options(&o);
    if (opt) o = *opt;
    if (!(T >= 0)) return ms2_fail(MS2_EINVAL, "temperature must be >= 0");
    double L = box;
    if (box > 0 && rho > 0) {
        const double L2 = std::cbrt((double)Nt / rho);
        if (std::fabs(L2 - box) > 1e-12 * box) return ms2_fail(MS2_EINVAL, "box and rho disagree (%.15g vs %.15g)", box, L2);
    } else if (!(box > 0)) {
        if (!(rho > 0)) return ms2_fail(MS2_EINVAL, "give box > 0 or rho > 0");
        L = std::cbrt((double)Nt / rho);
    }
    if (!(cutoff > 0) || !(cutoff < 0.5 * L))
        return ms2_fail(MS2_EINVAL, "cutoff %.6g must satisfy 0 < rc < box/2 = %.6g", cutoff, 0.5 * L);
    if (!(o.dt > 0)) return ms2_fail(MS2_EINVAL, "dt must be > 0");
    if (o.integrator != MS2_INT_VERLET && o.integrator != MS2_INT_LEAPFROG_Q)
        return ms2_fail(MS2_EINVAL, "unknown integrator");
    ms2_system s = new ms2_system_s();
    s->al.fa = o.dev_alloc;
    s->al.ff = o.dev_free;
    s->al.ctx = o.alloc_ctx;
    cudaGetDevice(&s->device);
    if (cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess || s->sms < 1)
        s->sms = 1;
    if (o.stream) {
        s->stream = (cudaStream_t)o.stream;
        s->own_stream = false;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete s;
            return ms2_fail_cuda(e, "cudaStreamCreate", __FILE__, __LINE__);
        }
        s->own_stream = true;
    }
    s->N = (int)Nt;
    for (int m = 0; m < n_models; ++m)
        for (int k = 0; k < N_per_model[m]; ++k) s->species.push_back(m);
    s->rc = cutoff;
    s->lrc = o.lrc != 0;
    s->reduced = o.reduced != 0;
    s->graph_chunk = o.graph_chunk > 0 ? o.graph_chunk : 50;
    ms2_fill_params(s->hp, models, n_models, s->species, L, cutoff, elec, o, T);
    // velocity Verlet integrates point molecules only
    bool point = true;
    for (int m = 0; m < n_models; ++m)
        if (s->hp.Iinv[m][0] != 0 || s->hp.Iinv[m][1] != 0 || s->hp.Iinv[m][2] != 0) point = false;
    if (o.integrator == MS2_INT_VERLET && !point) {
        delete s;
        return ms2_fail(MS2_EINVAL, "velocity Verlet is for molecules without rotational freedom; use MS2_INT_LEAPFROG_Q");
    }
    s->fp64 = o.fp64 != 0;
    if (s->fp64 && !(n_models == 1 && models[0].n_sites == 1 && elec == MS2_ELEC_NONE)) {
        delete s;
        return ms2_fail(MS2_EINVAL, "fp64 pair arithmetic is available for single-site LJ models only");
    }
    setup_pair(s);
    if (s->hp.massieu && (elec == MS2_ELEC_EWALD || s->hp.has_dipole || !s->pair_fn)) {
        delete s;
        return ms2_fail(MS2_EINVAL, "Massieu derivatives: LJ and point-charge models with the reaction field or no "
                                    "electrostatics (no Ewald, no point dipoles)");
    }
    setup_fused(s, o);
    pick_launch_shape(s);
    st = sys_alloc(s);
    if (st == MS2_OK) st = size_pair_tiles(s);
    if (st == MS2_OK && elec == MS2_ELEC_EWALD) st = setup_ewald(s, 3.2 / cutoff, 8, 8, 8);
    if (st == MS2_OK && elec != MS2_ELEC_EWALD) {
        double coulomb, kconv;
        ms2_unit_constants(s->reduced, &coulomb, &kconv);
        ms2_energy_constants(s->hp, s->species, 1.0, cutoff, s->lrc, coulomb, &s->uconst, &s->wbg, &s->ulrc, &s->plrc);
    }
    if (st == MS2_OK) {
        int kinds[MS2_MAXSP * MS2_MAXS];
        for (int m = 0; m < MS2_MAXSP; ++m)
            for (int a = 0; a < MS2_MAXS; ++a) kinds[m * MS2_MAXS + a] = m < n_models ? s->hp.ljt[m][a] : -1;
        cudaError_t e = cudaMemcpyAsync(s->d.rdf_kind, kinds, sizeof kinds, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s->d.species, s->species.data(), sizeof(int) * s->N,
                                                  cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) st = ms2_fail_cuda(e, "upload", __FILE__, __LINE__);
    }
    if (st == MS2_OK) st = upload_params(s);
    if (st == MS2_OK) {
        initial_state(s, models, T, o.seed);
        st = upload_state(s);
    }
    if (st == MS2_OK) st = ms2_eval_forces(s);
    if (st == MS2_OK) {
        cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) st = ms2_fail_cuda(e, "initial force evaluation", __FILE__, __LINE__);
    }
    if (st != MS2_OK) {
        std::string msg = g_err;
        ms2_destroy_system(s);
        g_err = msg;
        return st;
    }
    *out = s;
    return MS2_OK;
}

extern "C" ms2_status ms2_fault_inject(ms2_system s, int what, double wait_s) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    if (what != MS2_FAULT_BARRIER) return ms2_fail(MS2_EINVAL, "unknown fault %d", what);
    if (!(wait_s >= 1e-6 && wait_s <= 2.0)) return ms2_fail(MS2_EINVAL, "wait limit must be 1e-6..2 s");
    if (!s->step_fn) return ms2_fail(MS2_ESTATE, "the system has no fused step kernel");
    s->fault_barrier = 1;
    s->fault_wait_ns = (unsigned long long)(wait_s * 1e9);
    return MS2_OK;
}

extern "C" ms2_status ms2_enable_timing(ms2_system s, int on) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    if (on && !s->ev[0])
        for (int k = 0; k < 5; ++k) MS2_CUDA_OK(cudaEventCreate(&s->ev[k]));
    if ((on != 0) != s->timing) destroy_graphs(s);
    s->timing = on != 0;
    return MS2_OK;
}

extern "C" ms2_status ms2_step_kernel(ms2_system s, int *fused) {
    if (!s || !fused) return ms2_fail(MS2_EINVAL, "null argument");
    const int cells = s->d.rdf ? s->d.rdf_rows * s->d.rdf_bins : 0;
    *fused = s->step_fn && s->res_every == 0 && (s->hf_every == 0 || s->step_heat_fn) &&
                     ms2_step_smem_bytes(s->ns, s->tile, s->multi_used, s->Np, s->mcap, s->jsplit, cells, step_ews(s)) <=
                         s->step_smem_max
                 ? 1 : 0;
    return MS2_OK;
}

// the system scalars, through a page-locked buffer (a copy into pageable memory
// takes the driver's staged path)
static ms2_status read_scalars(ms2_system s, double *sc) {
    if (!s->hscal) MS2_CUDA_OK(cudaMallocHost((void **)&s->hscal, sizeof(double) * SC_COUNT_));
    MS2_CUDA_OK(cudaMemcpyAsync(s->hscal, s->d.scal, sizeof(double) * SC_COUNT_, cudaMemcpyDeviceToHost, s->stream));
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    std::memcpy(sc, s->hscal, sizeof(double) * SC_COUNT_);
    return MS2_OK;
}

// The server's status round: the system scalars queued to the page-locked host
// copy (ms2_scalars_enqueue, for many systems), one synchronisation by the
// caller, then each system's status from its copy (ms2_scalars_status): the
// checks of ms2_energy_virial without a synchronisation per system.
ms2_status ms2_scalars_enqueue(ms2_system s) {
    if (!s->hscal) MS2_CUDA_OK(cudaMallocHost((void **)&s->hscal, sizeof(double) * SC_COUNT_));
    MS2_CUDA_OK(cudaMemcpyAsync(s->hscal, s->d.scal, sizeof(double) * SC_COUNT_, cudaMemcpyDeviceToHost, s->stream));
    return MS2_OK;
}

ms2_status ms2_scalars_status(ms2_system s) {
    const double *sc = s->hscal;
    if (sc[SC_KERR] != 0.0) {
        const double zero = 0.0;
        cudaMemcpyAsync(s->d.scal + SC_KERR, &zero, sizeof zero, cudaMemcpyHostToDevice, s->stream);
        cudaMemsetAsync(s->d.counter + 48, 0, sizeof(unsigned), s->stream);
        cudaStreamSynchronize(s->stream);
        return ms2_fail(MS2_ETIMEOUT, "a grid-barrier wait of the step kernels timed out");
    }
    if (sc[SC_UNSTABLE] != 0.0 || !std::isfinite(sc[SC_UTOT]))
        return ms2_fail(MS2_EUNSTABLE, "non-finite or exploding forces in the current configuration");
    return MS2_OK;
}

extern "C" ms2_status ms2_last_step_phases(ms2_system s, double out[12]) {
    if (!s || !out) return ms2_fail(MS2_EINVAL, "null argument");
    if (!s->timing || !s->last_fused) return ms2_fail(MS2_ESTATE, "no timed fused chunk (timing off or per-phase kernels)");
    double sc[SC_COUNT_];
    ms2_status st = read_scalars(s, sc);
    if (st != MS2_OK) return st;
    for (int k = 0; k < 12; ++k) out[k] = sc[SC_TPH0 + k] * 1e-6;
    if (s->hp.elec != ELEC_EWALD) out[9] = out[10] = out[11] = 0.0;
    return MS2_OK;
}

extern "C" ms2_status ms2_last_step_times(ms2_system s, double out[4]) {
    if (!s || !out) return ms2_fail(MS2_EINVAL, "null argument");
    if (!s->timing) return ms2_fail(MS2_ESTATE, "timing is off (ms2_enable_timing)");
    MS2_CUDA_OK(cudaEventSynchronize(s->ev[4]));
    float a, b, c;
    if (s->last_fused) {  // one kernel per chunk: the step is the chunk's mean, the pair phase from %globaltimer
        double tp[SC_TPH11 - SC_TPAIR + 1];
        MS2_CUDA_OK(cudaMemcpy(tp, s->d.scal + SC_TPAIR, sizeof tp, cudaMemcpyDeviceToHost));
        MS2_CUDA_OK(cudaEventElapsedTime(&c, s->ev[0], s->ev[4]));
        out[2] = c / std::max(1, s->last_launch_steps);
        out[0] = tp[0] * 1e-6;
        // the reciprocal-space task phases (structure factor, sums, forces)
        out[1] = s->hp.elec == ELEC_EWALD
                     ? (tp[SC_TPH9 - SC_TPAIR] + tp[SC_TPH10 - SC_TPAIR] + tp[SC_TPH11 - SC_TPAIR]) * 1e-6
                     : 0.0;
        out[3] = out[2] - out[0];
        return MS2_OK;
    }
    MS2_CUDA_OK(cudaEventElapsedTime(&a, s->ev[1], s->ev[2]));
    MS2_CUDA_OK(cudaEventElapsedTime(&b, s->ev[2], s->ev[3]));
    MS2_CUDA_OK(cudaEventElapsedTime(&c, s->ev[0], s->ev[4]));
    out[0] = a;
    out[1] = b;
    out[2] = c;
    out[3] = c - a - b;
    return MS2_OK;
}

extern "C" ms2_status ms2_destroy_system(ms2_system s) {
    if (!s) return MS2_OK;
    cudaStreamSynchronize(s->stream);
    destroy_graphs(s);
    for (int k = 0; k < 5; ++k)
        if (s->ev[k]) cudaEventDestroy(s->ev[k]);
    if (s->pinned) cudaFreeHost(s->pinned);
    if (s->hscal) cudaFreeHost(s->hscal);
    for (int k = 0; k < 2; ++k)
        if (s->up_ev[k]) cudaEventDestroy(s->up_ev[k]);
    s->al.release_all();
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
    return MS2_OK;
}

extern "C" ms2_status ms2_system_info(ms2_system s, int *N, double *box, double *cutoff, int *ndof) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    if (N) *N = s->N;
    if (box) *box = s->hp.L;
    if (cutoff) *cutoff = s->rc;
    if (ndof) *ndof = s->hp.ndof;
    return MS2_OK;
}

// one fused launch of m steps from step counter s0; false: not possible now
// (no variant, RDF histogram too large for shared memory, launch refused)
static bool run_fused(ms2_system s, long long m, long long s0) {
    if (!s->step_fn || s->res_every > 0) return false;  // residence sampling runs on the per-phase path
    void *fn = s->hf_every > 0 ? s->step_heat_fn : s->step_fn;
    if (!fn) return false;
    const int cells = s->d.rdf ? s->d.rdf_rows * s->d.rdf_bins : 0;
    const size_t smem = ms2_step_smem_bytes(s->ns, s->tile, s->multi_used, s->Np, s->mcap, s->jsplit, cells, step_ews(s));
    if (smem > s->step_smem_max) return false;
    unsigned *cnt = s->d.counter;
    StepArgs A;
    A.nsteps = (int)m;
    A.s0 = s0;
    A.rdf_every = s->d.rdf ? s->rdf_every : 0;
    A.gk_every = s->d.gk ? s->gk_every : 0;
    A.hf_every = s->hf_every;
    A.TJ = s->TJ;
    A.Np = s->Np;
    A.mcap = s->mcap;
    A.bar = cnt + 16 + 16 * s->bar_parity;
    A.bar_next = cnt + 16 + 16 * (1 - s->bar_parity);
    A.err = cnt + 48;
    A.timing = s->timing ? 1 : 0;
    A.init = s->stale ? 1 : 0;
    A.AS = s->AS;
    A.ny_per_chunk = s->ny_per_chunk;
    A.ews = (int)step_ews(s);
    A.tmax = (unsigned long long *)(cnt + 56);  // 3 x 8 bytes at byte 224 of the counter block (zero at entry)
    A.wait_ns = s->fault_barrier ? s->fault_wait_ns : 2000000000ull;  // 2 s (grid_dev::WAIT_NS)
    A.bar_extra = s->fault_barrier ? 1u : 0u;
    s->fault_barrier = 0;  // one launch
    if (s->timing) cudaEventRecord(s->ev[0], s->stream);
    const cudaError_t e = ms2_launch_step(fn, s->step_grid, smem, s->stream, s->dP, s->d, A);
    if (e != cudaSuccess) {  // e.g. co-residency refused: the per-phase kernels from now on
        cudaGetLastError();
        s->step_fn = nullptr;
        return false;
    }
    if (s->timing) cudaEventRecord(s->ev[4], s->stream);
    s->bar_parity ^= 1;
    s->stale = false;
    s->last_launch_steps = (int)m;
    s->last_fused = true;
    ms2_count_launches(1);
    return true;
}

extern "C" ms2_status ms2_step(ms2_system s, long long n) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    if (n < 0) return ms2_fail(MS2_EINVAL, "negative step count");
    long long done = 0;
    const long long chunk = s->graph_chunk;
    while (done < n) {
        const long long m = std::min(chunk, n - done);
        if (!run_fused(s, m, s->step + done)) {
            ms2_status st = ms2_ensure_forces(s);
            if (st == MS2_OK) st = run_graph(s, m, s->step + done);
            if (st != MS2_OK) return st;
            s->last_fused = false;
        }
        done += m;
    }
    s->step += n;
    if (s->d.rdf && s->rdf_every > 0) {
        // samples taken inside the steps: configurations at steps multiple of every
        s->rdf_samples += (int)((s->step) / s->rdf_every - (s->step - n) / s->rdf_every);
    }
    MS2_CUDA_OK(cudaGetLastError());
    return MS2_OK;
}


extern "C" ms2_status ms2_energy_virial(ms2_system s, double *U, double *W, double *T_inst, double *P) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    if (ms2_status e = ms2_ensure_forces(s)) return e;
    double sc[SC_COUNT_];
    ms2_status st = read_scalars(s, sc);
    if (st != MS2_OK) return st;
    if (U) *U = sc[SC_UTOT];
    if (W) *W = sc[SC_WTOT];
    if (T_inst) *T_inst = sc[SC_T];
    if (P) *P = sc[SC_P];
    if (sc[SC_KERR] != 0.0) {  // a fused-step barrier wait ran out: the state is not to be trusted
        const double zero = 0.0;
        cudaMemcpyAsync(s->d.scal + SC_KERR, &zero, sizeof zero, cudaMemcpyHostToDevice, s->stream);
        cudaMemsetAsync(s->d.counter + 48, 0, sizeof(unsigned), s->stream);
        cudaStreamSynchronize(s->stream);
        return ms2_fail(MS2_ETIMEOUT, "a grid-barrier wait of the fused step kernel timed out");
    }
    if (sc[SC_UNSTABLE] != 0.0 || !std::isfinite(sc[SC_UTOT]))
        return ms2_fail(MS2_EUNSTABLE, "non-finite or exploding forces in the current configuration");
    return MS2_OK;
}

extern "C" ms2_status ms2_energy_terms(ms2_system s, double terms[16]) {
    if (!s || !terms) return ms2_fail(MS2_EINVAL, "null argument");
    if (ms2_status e = ms2_ensure_forces(s)) return e;
    double sc[SC_COUNT_];
    ms2_status st = read_scalars(s, sc);
    if (st != MS2_OK) return st;
    const bool ew = s->hp.elec == ELEC_EWALD;
    double coulomb, kconv;
    ms2_unit_constants(s->reduced, &coulomb, &kconv);
    double uself = 0, uintra = 0, ubg = 0;
    if (ew) {  // split of the constant part for reporting
        SysParams P = s->hp;
        double c_all, w, ul, pl;
        ms2_energy_constants(P, s->species, s->alpha, s->rc, false, coulomb, &c_all, &w, &ul, &pl);
        ubg = w / 3.0;
        double sq2 = 0;
        for (int i = 0; i < s->N; ++i)
            for (int a = 0; a < P.n_sites[s->species[i]]; ++a)
                sq2 += P.qd[s->species[i]][a] * P.qd[s->species[i]][a];
        uself = -coulomb * s->alpha / std::sqrt(M_PI) * sq2;
        uintra = c_all - uself - ubg;
    }
    // breakdown of the pair part, summed on demand from the per-molecule arrays
    double tb[8];
    k_terms<<<1, 256, 0, s->stream>>>(s->dP, s->d, s->d.terms);
    ms2_count_launches(1);
    MS2_CUDA_OK(cudaMemcpyAsync(tb, s->d.terms, sizeof tb, cudaMemcpyDeviceToHost, s->stream));
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    terms[0] = 0.5 * tb[0];
    terms[1] = 0.5 * tb[1];
    terms[2] = 0.5 * tb[2];
    terms[3] = ew ? sc[SC_UREC] : 0.0;
    terms[4] = uself;
    terms[5] = uintra;
    terms[6] = ubg;
    terms[7] = sc[SC_ULRC];
    terms[8] = sc[SC_UTOT];
    terms[9] = 0.5 * tb[3];
    terms[10] = ew ? sc[SC_WREC_AT] - tb[5] : 0.0;
    terms[11] = sc[SC_WBG];
    terms[12] = sc[SC_WTOT];
    terms[13] = sc[SC_PLRC];
    terms[14] = 0.5 * tb[4];
    terms[15] = sc[SC_KETR_NOW] + sc[SC_KEROT_NOW];
    return MS2_OK;
}

static ms2_status ensure_pinned(ms2_system s);
static ms2_status get_soa(ms2_system s, const double *src, int nc, double *dst) {
    const int N = s->N;
    ms2_status st = ensure_pinned(s);
    if (st != MS2_OK) return st;
    double *buf = s->pinned + (size_t)26 * N;  // the download buffer
    MS2_CUDA_OK(cudaMemcpyAsync(buf, src, sizeof(double) * nc * N, cudaMemcpyDeviceToHost, s->stream));
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < nc; ++k) dst[nc * i + k] = buf[(size_t)k * N + i];
    return MS2_OK;
}

extern "C" ms2_status ms2_forces_torques(ms2_system s, double *F, double *tau) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    ms2_status st = ms2_ensure_forces(s);
    if (F) st = get_soa(s, s->d.F, 3, F);
    if (st == MS2_OK && tau) st = get_soa(s, s->d.tau, 3, tau);
    return st;
}

__global__ void k_aos3(const double *src, double *dst, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N)
        for (int k = 0; k < 3; ++k) dst[3 * i + k] = src[(size_t)k * N + i];
}

extern "C" ms2_status ms2_forces_torques_dev(ms2_system s, double *F_dev, double *tau_dev) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    if (ms2_status e = ms2_ensure_forces(s)) return e;
    if (F_dev) k_aos3<<<(s->N + 127) / 128, 128, 0, s->stream>>>(s->d.F, F_dev, s->N);
    if (tau_dev) k_aos3<<<(s->N + 127) / 128, 128, 0, s->stream>>>(s->d.tau, tau_dev, s->N);
    ms2_count_launches((F_dev ? 1 : 0) + (tau_dev ? 1 : 0));
    MS2_CUDA_OK(cudaGetLastError());
    return MS2_OK;
}

extern "C" ms2_status ms2_ewald_params(ms2_system s, double alpha, int kx, int ky, int kz) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    if (s->hp.elec != ELEC_EWALD) return ms2_fail(MS2_EINVAL, "system does not use Ewald summation");
    if (!(alpha > 0) || kx < 1 || ky < 1 || kz < 1 || kx > 64 || ky > 64 || kz > 64)
        return ms2_fail(MS2_EINVAL, "need alpha > 0 and kmax in 1..64");
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    destroy_graphs(s);
    ms2_status st = setup_ewald(s, alpha, kx, ky, kz);
    if (st == MS2_OK) st = upload_params(s);
    if (st == MS2_OK) st = ms2_eval_forces(s);
    if (st == MS2_OK) s->stale = false;
    return st;
}

extern "C" ms2_status ms2_get_state(ms2_system s, double *R, double *q, double *v, double *Lang, long long *step) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    if (step) *step = s->step;
    if (!R && !q && !v && !Lang) return MS2_OK;
    ms2_status st = ensure_pinned(s);
    if (st != MS2_OK) return st;
    // one copy of the contiguous R, q, v, Lm (sys_alloc) into the download buffer
    const int N = s->N;
    double *buf = s->pinned + (size_t)26 * N;
    MS2_CUDA_OK(cudaMemcpyAsync(buf, s->d.R, sizeof(double) * 13 * N, cudaMemcpyDeviceToHost, s->stream));
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    auto out = [&](double *dst, size_t off, int nc) {
        if (dst)
            for (int i = 0; i < N; ++i)
                for (int k = 0; k < nc; ++k) dst[nc * i + k] = buf[off + (size_t)k * N + i];
    };
    out(R, 0, 3);
    out(q, (size_t)3 * N, 4);
    out(v, (size_t)7 * N, 3);
    out(Lang, (size_t)10 * N, 3);
    return MS2_OK;
}

extern "C" ms2_status ms2_set_state(ms2_system s, const double *R, const double *q, const double *v,
                                    const double *Lang) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    const int N = s->N;
    if (R && q && v && Lang) {  // the whole state: validated and staged in one pass, straight into pinned memory
        ms2_status st = ensure_pinned(s);
        if (st != MS2_OK) return st;
        const int k = s->up_k;
        MS2_CUDA_OK(cudaEventSynchronize(s->up_ev[k]));
        double *b = s->pinned + (size_t)13 * N * k;  // R, q, v, Lm in the device order (sys_alloc)
        for (int i = 0; i < N; ++i) {
            for (int c = 0; c < 3; ++c) {
                const double x = R[3 * i + c], y = v[3 * i + c], z = Lang[3 * i + c];
                if (!std::isfinite(x) || !std::isfinite(y) || !std::isfinite(z))
                    return ms2_fail(MS2_EINVAL, "non-finite state value for molecule %d", i);
                b[(size_t)c * N + i] = x;
                b[(size_t)(7 + c) * N + i] = y;
                b[(size_t)(10 + c) * N + i] = z;
            }
            double n2 = 0;
            for (int c = 0; c < 4; ++c) n2 += q[4 * i + c] * q[4 * i + c];
            if (!(n2 > 0) || !std::isfinite(n2)) return ms2_fail(MS2_EINVAL, "quaternion %d has zero norm", i);
            const double inv = std::fabs(n2 - 1.0) > 1e-13 ? 1.0 / std::sqrt(n2) : 1.0;  // unit ones bit for bit
            for (int c = 0; c < 4; ++c) b[(size_t)(3 + c) * N + i] = inv == 1.0 ? q[4 * i + c] : q[4 * i + c] * inv;
        }
        MS2_CUDA_OK(cudaMemcpyAsync(s->d.R, b, sizeof(double) * 13 * N, cudaMemcpyHostToDevice, s->stream));
        MS2_CUDA_OK(cudaEventRecord(s->up_ev[k], s->stream));
        s->up_k = 1 - k;
        s->stale = true;
        return MS2_OK;
    }
    if (R || q || v || Lang) {
        std::vector<double> cur;
        // fetch what is not replaced
        if (!R) { s->hR.resize(3 * N); ms2_status st = get_soa(s, s->d.R, 3, s->hR.data()); if (st) return st; }
        else s->hR.assign(R, R + 3 * N);
        if (!q) { s->hq.resize(4 * N); ms2_status st = get_soa(s, s->d.q, 4, s->hq.data()); if (st) return st; }
        else s->hq.assign(q, q + 4 * N);
        if (!v) { s->hv.resize(3 * N); ms2_status st = get_soa(s, s->d.v, 3, s->hv.data()); if (st) return st; }
        else s->hv.assign(v, v + 3 * N);
        if (!Lang) { s->hL.resize(3 * N); ms2_status st = get_soa(s, s->d.Lm, 3, s->hL.data()); if (st) return st; }
        else s->hL.assign(Lang, Lang + 3 * N);
        for (int i = 0; i < N; ++i) {
            for (int k = 0; k < 3; ++k)
                if (!std::isfinite(s->hR[3 * i + k]) || !std::isfinite(s->hv[3 * i + k]) || !std::isfinite(s->hL[3 * i + k]))
                    return ms2_fail(MS2_EINVAL, "non-finite state value for molecule %d", i);
            double n2 = 0;
            for (int k = 0; k < 4; ++k) n2 += s->hq[4 * i + k] * s->hq[4 * i + k];
            if (!(n2 > 0) || !std::isfinite(n2)) return ms2_fail(MS2_EINVAL, "quaternion %d has zero norm", i);
            if (std::fabs(n2 - 1.0) > 1e-13) {  // unit quaternions are taken bit for bit
                const double inv = 1.0 / std::sqrt(n2);
                for (int k = 0; k < 4; ++k) s->hq[4 * i + k] *= inv;
            }
        }
        ms2_status st = upload_state(s);
        if (st != MS2_OK) return st;
    }
    s->stale = true;
    return MS2_OK;
}

extern "C" ms2_status ms2_partner_counts(ms2_system s, int *counts) {
    if (!s || !counts) return ms2_fail(MS2_EINVAL, "null argument");
    if (ms2_status e = ms2_ensure_forces(s)) return e;
    MS2_CUDA_OK(cudaMemcpyAsync(counts, s->d.npart, sizeof(int) * s->N, cudaMemcpyDeviceToHost, s->stream));
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    return MS2_OK;
}

extern "C" ms2_status ms2_molecule_energies(ms2_system s, double *out) {
    if (!s || !out) return ms2_fail(MS2_EINVAL, "null argument");
    if (ms2_status e = ms2_ensure_forces(s)) return e;
    ms2_status st = get_soa(s, s->d.Ui, 4, out);
    if (st != MS2_OK) return st;
    for (int k = 0; k < 4 * s->N; ++k) out[k] *= 0.5;
    return MS2_OK;
}

extern "C" ms2_status ms2_site_offsets(ms2_system s, double *offsets, int *n_site_slots) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    if (ms2_status e = ms2_ensure_forces(s)) return e;
    const int N = s->N, NS = s->ns;
    if (n_site_slots) *n_site_slots = NS;
    if (!offsets) return MS2_OK;
    std::vector<float> buf((size_t)3 * NS * N);
    MS2_CUDA_OK(cudaMemcpyAsync(buf.data(), s->d.s, sizeof(float) * buf.size(), cudaMemcpyDeviceToHost, s->stream));
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < NS; ++a)
            for (int k = 0; k < 3; ++k) offsets[((size_t)i * NS + a) * 3 + k] = buf[((size_t)k * NS + a) * N + i];
    return MS2_OK;
}

extern "C" ms2_status ms2_rdf_setup(ms2_system s, double r_max, int n_bins, int every) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    const int T = s->hp.n_ljt;
    if (T < 1) return ms2_fail(MS2_EINVAL, "no LJ sites: the RDF is sampled between LJ sites");
    const int rows = T * (T + 1) / 2;
    if (n_bins < 1 || rows * n_bins > 12288) return ms2_fail(MS2_EINVAL, "need 1 <= n_bins and rows*bins <= 12288");
    if (!(r_max > 0) || r_max > std::min(s->rc, 0.5 * s->hp.L) * (1 + 1e-12))
        return ms2_fail(MS2_EINVAL, "r_max must be in (0, min(cutoff, box/2)]");
    if (every < 0) return ms2_fail(MS2_EINVAL, "negative sampling interval");
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    destroy_graphs(s);
    if (!s->d.rdf || rows * n_bins > s->rdf_cap) {
        MS2_CUDA_OK(s->al.alloc((void **)&s->d.rdf, sizeof(unsigned long long) * rows * n_bins));
        s->rdf_cap = rows * n_bins;
    }
    MS2_CUDA_OK(cudaMemsetAsync(s->d.rdf, 0, sizeof(unsigned long long) * rows * n_bins, s->stream));
    s->d.rdf_bins = n_bins;
    s->d.rdf_rows = rows;
    s->d.rdf_inv_dr = (float)(n_bins / r_max);
    s->d.rdf_rmax2 = (float)(r_max * r_max);
    s->rdf_rmax = r_max;
    s->rdf_every = every;
    s->rdf_samples = 0;
    return MS2_OK;
}

extern "C" ms2_status ms2_rdf_sample(ms2_system s) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    if (!s->d.rdf) return ms2_fail(MS2_ESTATE, "call ms2_rdf_setup first");
    if (ms2_status e = ms2_ensure_forces(s)) return e;
    launch_rdf(s);
    flush_launches(s);
    MS2_CUDA_OK(cudaGetLastError());
    s->rdf_samples += 1;
    return MS2_OK;
}

extern "C" ms2_status ms2_rdf(ms2_system s, long long *counts, double *g, int *n_samples, int *n_rows) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    if (!s->d.rdf) return ms2_fail(MS2_ESTATE, "call ms2_rdf_setup first");
    const int rows = s->d.rdf_rows, nb = s->d.rdf_bins;
    std::vector<unsigned long long> c((size_t)rows * nb);
    MS2_CUDA_OK(cudaMemcpyAsync(c.data(), s->d.rdf, sizeof(unsigned long long) * c.size(), cudaMemcpyDeviceToHost,
                                s->stream));
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    if (n_samples) *n_samples = s->rdf_samples;
    if (n_rows) *n_rows = rows;
    if (counts)
        for (size_t k = 0; k < c.size(); ++k) counts[k] = (long long)c[k];
    if (g) {
        const SysParams &P = s->hp;
        int cnt[MS2_MAXSP] = {0}, kind_sp[MS2_MAXT];
        for (int i = 0; i < s->N; ++i) cnt[s->species[i]]++;
        for (int m = 0; m < P.n_species; ++m)
            for (int a = 0; a < P.n_sites[m]; ++a)
                if (P.ljt[m][a] >= 0) kind_sp[P.ljt[m][a]] = m;
        const int T = P.n_ljt;
        const double dr = s->rdf_rmax / nb;
        int row = 0;
        for (int t1 = 0; t1 < T; ++t1)
            for (int t2 = t1; t2 < T; ++t2, ++row) {
                const int a = kind_sp[t1], b = kind_sp[t2];
                double pairs = (t1 == t2) ? 0.5 * cnt[a] * (cnt[a] - 1.0)
                                          : (a == b ? cnt[a] * (cnt[a] - 1.0) : (double)cnt[a] * cnt[b]);
                for (int k = 0; k < nb; ++k) {
                    const double shell = 4.0 * M_PI / 3.0 * (std::pow((k + 1) * dr, 3) - std::pow(k * dr, 3));
                    const double ideal = pairs * shell / P.V * std::max(s->rdf_samples, 1);
                    g[(size_t)row * nb + k] = ideal > 0 ? c[(size_t)row * nb + k] / ideal : 0.0;
                }
            }
    }
    return MS2_OK;
}

extern "C" ms2_status ms2_averages(ms2_system s, double out[5], long long *n_steps) {
    if (!s || !out) return ms2_fail(MS2_EINVAL, "null argument");
    double ac[AC_COUNT_];
    MS2_CUDA_OK(cudaMemcpyAsync(ac, s->d.acc, sizeof ac, cudaMemcpyDeviceToHost, s->stream));
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    const double n = std::max(ac[AC_N], 1.0), nb = ac[AC_NB];
    out[0] = ac[AC_U] / n;
    out[1] = ac[AC_P] / n;
    out[2] = ac[AC_T] / n;
    auto err = [&](double s1, double s2) {
        if (nb < 2) return 0.0;
        const double m = s1 / nb, var = std::max(0.0, s2 / nb - m * m);
        return std::sqrt(var / (nb - 1));
    };
    out[3] = err(ac[AC_SBU], ac[AC_SBU2]);
    out[4] = err(ac[AC_SBP], ac[AC_SBP2]);
    if (n_steps) *n_steps = (long long)ac[AC_N];
    return MS2_OK;
}

extern "C" ms2_status ms2_volume_derivatives(ms2_system s, double *dUdV, double *d2UdV2) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    if (ms2_status e = ms2_ensure_forces(s)) return e;
    if (!s->hp.massieu) return ms2_fail(MS2_ESTATE, "created without ms2_options.massieu");
    double sc[SC_COUNT_];
    ms2_status st = read_scalars(s, sc);
    if (st != MS2_OK) return st;
    if (dUdV) *dUdV = sc[SC_UV];
    if (d2UdV2) *d2UdV2 = sc[SC_UVV];
    return MS2_OK;
}

// Residual Massieu derivatives from the running moments (formulas in ms2.h):
// canonical moments of U, U_V = dU/dV and U_VV = d2U/dV2, with beta = 1/T0.
extern "C" ms2_status ms2_massieu(ms2_system s, double A[8], long long *n_samples) {
    if (!s || !A) return ms2_fail(MS2_EINVAL, "null argument");
    if (!s->hp.massieu) return ms2_fail(MS2_ESTATE, "created without ms2_options.massieu");
    double ac[AC_COUNT_];
    MS2_CUDA_OK(cudaMemcpyAsync(ac, s->d.acc, sizeof ac, cudaMemcpyDeviceToHost, s->stream));
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    if (n_samples) *n_samples = (long long)ac[AC_MN];
    if (ac[AC_MN] < 1.0) return ms2_fail(MS2_ESTATE, "no samples since the last ms2_reset_averages");
    const double n = ac[AC_MN], b = s->hp.inv_T0, V = s->hp.V, Nm = (double)s->N;
    // first moments of the shifted samples, then central second and third moments
    const double ex = ac[AC_MX] / n, ey = ac[AC_MY] / n, ew = ac[AC_MW] / n;
    const double exx = ac[AC_MX2] / n, eyy = ac[AC_MY2] / n, exy = ac[AC_MXY] / n;
    const double varU = exx - ex * ex, varV = eyy - ey * ey, covUV = exy - ex * ey;
    const double covUW = ac[AC_MXW] / n - ex * ew;
    const double cU3 = ac[AC_MX3] / n - 3.0 * ex * exx + 2.0 * ex * ex * ex;
    const double cU2V = ac[AC_MX2Y] / n - 2.0 * ex * exy - ey * exx + 2.0 * ex * ex * ey;
    const double cUV2 = ac[AC_MXY2] / n - 2.0 * ey * exy - ex * eyy + 2.0 * ex * ey * ey;
    const double mU = ac[AC_MU0] + ex, mUV = ac[AC_MV0] + ey;
    A[0] = b * mU / Nm;                                                    // A10
    A[1] = -b * V * mUV / Nm;                                              // A01
    A[2] = -b * b * varU / Nm;                                             // A20
    A[3] = -b * V / Nm * (mUV - b * covUV);                                // A11
    A[4] = b / Nm * (2.0 * V * mUV + V * V * (ew - b * varV));             // A02
    A[5] = b * b * b * cU3 / Nm;                                           // A30
    A[6] = b * b * V / Nm * (2.0 * covUV - b * cU2V);                      // A21
    A[7] = b / Nm * (2.0 * V * (mUV - b * covUV) +
                     V * V * (ew - 2.0 * b * varV - b * covUW + b * b * cUV2));  // A12
    return MS2_OK;
}

// ------------------------------------------------ residence time (Eq. 7)
extern "C" ms2_status ms2_residence_setup(ms2_system s, int species_i, int species_j, double r_shell, int every,
                                          int n_lags, int t_star) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    const int ns = s->hp.n_species;
    if (species_i < 0 || species_i >= ns || species_j < 0 || species_j >= ns)
        return ms2_fail(MS2_EINVAL, "species indices must be in 0..%d", ns - 1);
    if (!(r_shell > 0) || !(r_shell < 0.5 * s->hp.L)) return ms2_fail(MS2_EINVAL, "need 0 < r_shell < L/2");
    if (every < 1 || n_lags < 2 || n_lags > 4096 || t_star < 0 || t_star > 254)
        return ms2_fail(MS2_EINVAL, "need every >= 1, 2 <= n_lags <= 4096, 0 <= t_star <= 254");
    int first[MS2_MAXSP + 1] = {0}, count[MS2_MAXSP] = {0};
    for (int sp : s->species) count[sp]++;
    for (int m = 0; m < ns; ++m) first[m + 1] = first[m] + count[m];
    ResArgs a{};
    a.A0 = first[species_i];
    a.NA = count[species_i];
    a.B0 = first[species_j];
    a.NB = count[species_j];
    a.WB = (a.NB + 31) / 32;
    a.M = n_lags;
    a.t_star = t_star;
    if (a.NA < 1 || a.NB < 1) return ms2_fail(MS2_EINVAL, "both species need molecules");
    const double sc = r_shell * 4294967296.0 / s->hp.L;
    a.r2 = (unsigned long long)std::ceil(sc * sc);
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    const size_t M = (size_t)a.M, NA = (size_t)a.NA;
    MS2_CUDA_OK(s->al.alloc((void **)&a.alive, sizeof(unsigned) * M * NA * a.WB));
    MS2_CUDA_OK(s->al.alloc((void **)&a.out, M * NA * (size_t)a.NB));
    MS2_CUDA_OK(s->al.alloc((void **)&a.n0, sizeof(int) * M * NA));
    MS2_CUDA_OK(s->al.alloc((void **)&a.counts, sizeof(int) * M * NA));
    MS2_CUDA_OK(s->al.alloc((void **)&a.state, sizeof(double) * ms2_residence_state_doubles(a.M)));
    MS2_CUDA_OK(cudaMemsetAsync(a.alive, 0, sizeof(unsigned) * M * NA * a.WB, s->stream));
    MS2_CUDA_OK(cudaMemsetAsync(a.out, 0, M * NA * (size_t)a.NB, s->stream));
    MS2_CUDA_OK(cudaMemsetAsync(a.n0, 0, sizeof(int) * M * NA, s->stream));
    MS2_CUDA_OK(cudaMemsetAsync(a.counts, 0, sizeof(int) * M * NA, s->stream));
    MS2_CUDA_OK(cudaMemsetAsync(a.state, 0, sizeof(double) * ms2_residence_state_doubles(a.M), s->stream));
    s->res = a;  // buffers of an earlier setup stay with the system until it is destroyed
    s->res_every = every;
    destroy_graphs(s);
    return MS2_OK;
}

extern "C" ms2_status ms2_residence(ms2_system s, double *corr, double *tau, double *solvation,
                                    long long *n_samples) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    if (s->res_every <= 0) return ms2_fail(MS2_ESTATE, "residence sampling is off (ms2_residence_setup)");
    const int M = s->res.M;
    std::vector<double> st(ms2_residence_state_doubles(M));
    MS2_CUDA_OK(cudaMemcpyAsync(st.data(), s->res.state, sizeof(double) * st.size(), cudaMemcpyDeviceToHost,
                                s->stream));
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    if (n_samples) *n_samples = (long long)st[0];
    if (solvation) *solvation = st[2] > 0 ? st[1] / st[2] : 0.0;
    const double *num = st.data() + 3, *cnt = num + M;
    double integral = 0.0;
    for (int m = 0; m < M; ++m) {
        const double c = cnt[m] > 0 ? num[m] / cnt[m] : 0.0;
        if (corr) corr[m] = c;
        integral += ((m == 0 || m == M - 1) ? 0.5 : 1.0) * c;
    }
    if (tau) *tau = integral * s->res_every * s->hp.dt;
    return MS2_OK;
}

// ------------------------------------------------ Green-Kubo conductivity
extern "C" ms2_status ms2_conductivity_setup(ms2_system s, int every, int n_lags) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    if (every < 1 || n_lags < 2 || n_lags > (1 << 20))
        return ms2_fail(MS2_EINVAL, "need every >= 1 and 2 <= n_lags <= 2^20");
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    if (!s->d.gk || s->d.gk_lags != n_lags) {
        double *g = nullptr;
        MS2_CUDA_OK(s->al.alloc((void **)&g, sizeof(double) * (4 + 4 * (size_t)n_lags)));
        s->d.gk = g;  // a previous, smaller buffer stays with the system until it is destroyed
        s->d.gk_lags = n_lags;
    }
    MS2_CUDA_OK(cudaMemsetAsync(s->d.gk, 0, sizeof(double) * (4 + 4 * (size_t)n_lags), s->stream));
    s->gk_every = every;
    destroy_graphs(s);
    return MS2_OK;
}

extern "C" ms2_status ms2_current(ms2_system s, double j[3]) {
    if (!s || !j) return ms2_fail(MS2_EINVAL, "null argument");
    if (!s->d.gk) return ms2_fail(MS2_ESTATE, "conductivity sampling is off (ms2_conductivity_setup)");
    double sc[SC_COUNT_];
    ms2_status st = read_scalars(s, sc);
    if (st != MS2_OK) return st;
    for (int k = 0; k < 3; ++k) j[k] = sc[SC_JX + k];
    return MS2_OK;
}

extern "C" ms2_status ms2_conductivity(ms2_system s, double *sigma, double *acf, long long *n_samples) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    if (!s->d.gk) return ms2_fail(MS2_ESTATE, "conductivity sampling is off (ms2_conductivity_setup)");
    const int M = s->d.gk_lags;
    std::vector<double> g(4 + 4 * (size_t)M);
    MS2_CUDA_OK(cudaMemcpyAsync(g.data(), s->d.gk, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, s->stream));
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    const long long n = (long long)g[0];
    if (n_samples) *n_samples = n;
    const double *sums = g.data() + 4 + 3 * (size_t)M;
    // autocorrelation over all time origins, then the trapezoidal integral
    double integral = 0.0;
    for (int m = 0; m < M; ++m) {
        const double c = m < n ? sums[m] / (double)(n - m) : 0.0;
        if (acf) acf[m] = c;
        integral += ((m == 0 || m == M - 1) ? 0.5 : 1.0) * c;
    }
    integral *= s->gk_every * s->hp.dt;
    if (sigma) {
        if (s->reduced) {
            *sigma = integral / (3.0 * s->hp.V * s->hp.T0);
        } else {  // e^2 (A/fs)^2 fs / (A^3 kB K) -> S/m
            const double e = 1.602176634e-19, kB = 1.380649e-23;
            *sigma = integral * e * e * 1e-5 / (3.0 * s->hp.V * 1e-30 * kB * s->hp.T0);
        }
    }
    return MS2_OK;
}

// ------------------------------------------ Green-Kubo thermal conductivity
extern "C" ms2_status ms2_heat_setup(ms2_system s, int every, int n_lags, const double *h) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    if (every < 1 || n_lags < 2 || n_lags > (1 << 20))
        return ms2_fail(MS2_EINVAL, "need every >= 1 and 2 <= n_lags <= 2^20");
    if (s->hp.elec == ELEC_EWALD) return ms2_fail(MS2_EINVAL, "heat flux: pairwise interactions only (no Ewald)");
    void *hfn = s->fp64 ? nullptr : ms2_pick_heat_kernel(s->ns, s->ljm, s->qm, s->dm, s->hp.elec, s->multi_used, s->pair_fn);
    if (!hfn) return ms2_fail(MS2_EINVAL, "heat flux: no heat-flux kernel for this system (FP64 or 8-slot models)");
    for (int m = 0; h && m < s->hp.n_species; ++m)
        if (!std::isfinite(h[m])) return ms2_fail(MS2_EINVAL, "partial molar enthalpy %d is not finite", m);
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    MS2_CUDA_OK(ms2_allow_smem((const void *)hfn, s->pair_smem));
    if (!s->d.hpart) MS2_CUDA_OK(s->al.alloc((void **)&s->d.hpart, sizeof(float) * 3 * (size_t)s->jsplit * s->N));
    if (!s->d.hf || s->d.hf_lags != n_lags) {
        double *g = nullptr;
        MS2_CUDA_OK(s->al.alloc((void **)&g, sizeof(double) * (4 + 4 * (size_t)n_lags)));
        s->d.hf = g;  // a previous buffer stays with the system until it is destroyed
        s->d.hf_lags = n_lags;
    }
    MS2_CUDA_OK(cudaMemsetAsync(s->d.hf, 0, sizeof(double) * (4 + 4 * (size_t)n_lags), s->stream));
    for (int m = 0; m < MS2_MAXSP; ++m) s->hp.henth[m] = (h && m < s->hp.n_species) ? h[m] : 0.0;
    MS2_CUDA_OK(cudaMemcpyAsync(s->dP, &s->hp, sizeof(SysParams), cudaMemcpyHostToDevice, s->stream));
    // the fused variant with the heat pass, on the same decomposition
    s->step_heat_fn = nullptr;
    if (s->fuse_fn && s->step_fn) {
        void *fn = ms2_pick_step_kernel(s->ns, s->ljm, s->qm, s->dm, s->hp.elec, false, s->hp.massieu != 0, true);
        int nb = 0;
        const size_t base = ms2_step_smem_bytes(s->ns, s->tile, s->multi_used, s->Np, s->mcap, s->jsplit, 0, 0);
        if (fn && ms2_allow_smem(fn, s->step_smem_max) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, ms2_step_threads(), base) == cudaSuccess && nb >= 1)
            s->step_heat_fn = fn;
        cudaGetLastError();
    }
    s->heat_fn = hfn;
    s->hf_every = every;
    destroy_graphs(s);
    return MS2_OK;
}

extern "C" ms2_status ms2_heat_flux(ms2_system s, double J[3]) {
    if (!s || !J) return ms2_fail(MS2_EINVAL, "null argument");
    if (s->hf_every <= 0) return ms2_fail(MS2_ESTATE, "heat-flux sampling is off (ms2_heat_setup)");
    double sc[SC_COUNT_];
    ms2_status st = read_scalars(s, sc);
    if (st != MS2_OK) return st;
    for (int k = 0; k < 3; ++k) J[k] = sc[SC_HX + k];
    return MS2_OK;
}

extern "C" ms2_status ms2_thermal_conductivity(ms2_system s, double *lambda, double *acf, long long *n_samples) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    if (s->hf_every <= 0) return ms2_fail(MS2_ESTATE, "heat-flux sampling is off (ms2_heat_setup)");
    const int M = s->d.hf_lags;
    std::vector<double> g(4 + 4 * (size_t)M);
    MS2_CUDA_OK(cudaMemcpyAsync(g.data(), s->d.hf, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, s->stream));
    MS2_CUDA_OK(cudaStreamSynchronize(s->stream));
    const long long n = (long long)g[0];
    if (n_samples) *n_samples = n;
    const double *sums = g.data() + 4 + 3 * (size_t)M;
    double integral = 0.0;
    for (int m = 0; m < M; ++m) {
        const double c = m < n ? sums[m] / (double)(n - m) : 0.0;
        if (acf) acf[m] = c;
        integral += ((m == 0 || m == M - 1) ? 0.5 : 1.0) * c;
    }
    integral *= s->hf_every * s->hp.dt;
    if (lambda) {
        const double T = s->hp.T0;
        if (s->reduced) {
            *lambda = integral / (3.0 * s->hp.V * T * T);
        } else {  // (K A/fs)^2 fs / (A^3 K^2) with energies in K: kB 1e-5 / 1e-30 -> W/(m K)
            const double kB = 1.380649e-23;
            *lambda = integral * kB * 1e-5 / (3.0 * s->hp.V * 1e-30 * T * T);
        }
    }
    return MS2_OK;
}

extern "C" ms2_status ms2_reset_averages(ms2_system s) {
    if (!s) return ms2_fail(MS2_EINVAL, "null system");
    MS2_CUDA_OK(cudaMemsetAsync(s->d.acc, 0, sizeof(double) * AC_COUNT_, s->stream));
    return MS2_OK;
}
