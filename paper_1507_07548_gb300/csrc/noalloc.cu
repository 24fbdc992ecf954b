// Allocation-free force evaluation.
//
// Some callers cannot allocate device memory: code that runs inside a
// pre-reserved memory pool or under a strict memory cap, plugins handed a
// stream and a few buffers by a host application that owns all allocations,
// and sections that must not call cudaMalloc because it can implicitly
// synchronise the device.  ms2_forces_noalloc serves them: it evaluates one
// configuration with the same kernels as an ms2_system, but keeps all of its
// working memory in one statically sized __device__ array.  The caller passes
// inputs and outputs only.
//
// The array (NOALLOC_BYTES below, ~2.9 MB) exists on every GPU that loads this
// library, for the life of the process.  Every call uses the same array, so
// calls that overlap on the GPU (different streams, or threads) race; the
// array keeps the last call's contents, and each call clears what must start
// at zero.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "ms2_host.h"

namespace {

constexpr int NA_NMAX = 4096;  // molecules
constexpr int NA_NS = 4;       // site slots
constexpr int NA_JS = 8;       // j-range split of the pair kernel

constexpr size_t al256(size_t n) { return (n + 255) & ~(size_t)255; }
constexpr size_t O_PARAMS = 0;
constexpr size_t O_X = O_PARAMS + al256(sizeof(SysParams));
constexpr size_t O_S = O_X + al256(3 * sizeof(uint32_t) * NA_NMAX);
constexpr size_t O_MU = O_S + al256(3 * NA_NS * sizeof(float) * NA_NMAX);
constexpr size_t O_MUM = O_MU + al256(3 * NA_NS * sizeof(float) * NA_NMAX);
constexpr size_t O_PART = O_MUM + al256(3 * sizeof(float) * NA_NMAX);
constexpr size_t O_F = O_PART + al256((size_t)NA_JS * MS2_NPV * sizeof(float) * NA_NMAX);
constexpr size_t O_TAU = O_F + al256(3 * sizeof(double) * NA_NMAX);
constexpr size_t O_UI = O_TAU + al256(3 * sizeof(double) * NA_NMAX);
constexpr size_t O_NP = O_UI + al256(4 * sizeof(double) * NA_NMAX);
constexpr size_t O_BLK = O_NP + al256(sizeof(int) * NA_NMAX);
constexpr size_t O_CNT = O_BLK + al256((size_t)MS2_NRED * sizeof(double) * ((NA_NMAX + 7) / 8));
constexpr size_t O_SCAL = O_CNT + 256;
constexpr size_t O_SPEC = O_SCAL + al256(SC_COUNT_ * sizeof(double));
constexpr size_t O_R = O_SPEC + al256(sizeof(int) * NA_NMAX);
constexpr size_t O_Q = O_R + al256(3 * sizeof(double) * NA_NMAX);
constexpr size_t O_V = O_Q + al256(4 * sizeof(double) * NA_NMAX);
constexpr size_t O_L = O_V + al256(3 * sizeof(double) * NA_NMAX);
constexpr size_t NOALLOC_BYTES = O_L + al256(3 * sizeof(double) * NA_NMAX);

}  // namespace

// The scratch: a host-side name for device memory.  Host code must not use
// &g_noalloc_scratch as a device address; it asks the runtime for the address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

__global__ void k_build(const SysParams *, DevSys);
__global__ void k_reduce(const SysParams *, DevSys, int);
__global__ void k_aos3(const double *src, double *dst, int N);
size_t ms2_pair_smem_bytes(int NS, int tile, bool multi, int TJ, int wpb);
void *ms2_pick_pair_kernel(int ns, unsigned ljm, unsigned qm, unsigned dm, int elec, bool multi, int *ns_used,
                           int *tile, bool *mult_used, bool mass);
ms2_status ms2_validate_models(const ms2_model *models, int n_models, ms2_elec elec);
void ms2_fill_params(SysParams &P, const ms2_model *models, int n_models, const std::vector<int> &species, double L,
                     double rc, ms2_elec elec, const ms2_options &o, double T0);
void ms2_energy_constants(const SysParams &P, const std::vector<int> &species, double alpha, double rc, bool lrc,
                          double coulomb, double *uconst, double *wbg, double *ulrc, double *plrc);

// Everything a call sets up in the scratch, passed by value (no host buffer, so
// no pageable copy): the system constants, the energy constants, the counts per
// model.
struct NaSetup {
    double uconst, ulrc, plrc, wbg;
    int counts[MS2_MAXSP];
    int n_models;
};

// One thread per molecule: SoA copies of the row-major inputs, the species from
// the model counts, zero velocities and angular momenta (the reduction reads
// them: kinetic energy 0).  Block 0 also writes the constants, the scalars and
// the zeroed last-block counter.
__global__ void k_noalloc_setup(SysParams P, NaSetup c, DevSys d, SysParams *dP, const double *R, const double *q) {
    const int N = d.N, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0) {
        const int4 *src = (const int4 *)&P;
        int4 *dst = (int4 *)dP;
        for (int k = threadIdx.x; k < (int)(sizeof(SysParams) / sizeof(int4)); k += blockDim.x) dst[k] = src[k];
        for (int k = threadIdx.x; k < SC_COUNT_; k += blockDim.x) d.scal[k] = 0.0;
        for (int k = threadIdx.x; k < 64; k += blockDim.x) d.counter[k] = 0u;
        __syncthreads();
        if (threadIdx.x == 0) {
            d.scal[SC_UCONST] = c.uconst;
            d.scal[SC_ULRC] = c.ulrc;
            d.scal[SC_PLRC] = c.plrc;
            d.scal[SC_WBG] = c.wbg;
            d.scal[SC_LAMBDA] = 1.0;
        }
    }
    if (i >= N) return;
    for (int k = 0; k < 3; ++k) {
        d.R[(size_t)k * N + i] = R[3 * i + k];
        d.v[(size_t)k * N + i] = 0.0;
        d.Lm[(size_t)k * N + i] = 0.0;
    }
    for (int k = 0; k < 4; ++k) d.q[(size_t)k * N + i] = q[4 * i + k];
    int m = 0, end = c.counts[0];
    while (m + 1 < c.n_models && i >= end) end += c.counts[++m];
    d.species[i] = m;
}

namespace {
struct DeviceScratch {
    bool ready = false;
    unsigned char *base = nullptr;
    int sms = 0;                 // multiprocessors of the device
    const void *attr_set[16];    // pair kernels whose shared-memory limit is raised on this device
    int n_attr = 0;
};
std::mutex g_noalloc_mu;
DeviceScratch g_noalloc_dev[64];

// once per device, with that device current: the device address of the array,
// the multiprocessor count; the dynamic shared-memory limit of the pair kernel
// `fn` raised to 96 KB once per kernel
ms2_status scratch_base(unsigned char **out, int *sms, const void *fn) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ms2_fail_cuda(e, "cudaGetDevice", __FILE__, __LINE__);
    if (dev < 0 || dev >= 64) return ms2_fail(MS2_EINVAL, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    DeviceScratch &d = g_noalloc_dev[dev];
    if (!d.ready) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return ms2_fail_cuda(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
        d.base = (unsigned char *)p;
        e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return ms2_fail_cuda(e, "cudaDeviceGetAttribute", __FILE__, __LINE__);
        d.ready = true;
    }
    bool set = false;
    for (int k = 0; k < d.n_attr; ++k) set = set || d.attr_set[k] == fn;
    if (!set) {
        e = ms2_allow_smem(fn, 96 * 1024);
        if (e != cudaSuccess) return ms2_fail_cuda(e, "cudaFuncSetAttribute", __FILE__, __LINE__);
        if (d.n_attr < 16) d.attr_set[d.n_attr++] = fn;
    }
    *out = d.base;
    *sms = d.sms;
    return MS2_OK;
}
}  // namespace

extern "C" ms2_status ms2_forces_noalloc(const ms2_model *models, const int *N_per_model, int n_models, double box,
                                         double cutoff, ms2_elec elec, const ms2_options *opt, const double *R_dev,
                                         const double *q_dev, double *F_dev, double *tau_dev, double *UW_dev,
                                         void *stream) {
    ms2_status st = ms2_validate_models(models, n_models, elec);
    if (st != MS2_OK) return st;
    if (elec == MS2_ELEC_EWALD) return ms2_fail(MS2_EINVAL, "ms2_forces_noalloc: Ewald is not available here");
    if (!N_per_model || !R_dev || !q_dev || !F_dev || !tau_dev || !UW_dev)
        return ms2_fail(MS2_EINVAL, "ms2_forces_noalloc: null argument");
    long long Nt = 0;
    for (int m = 0; m < n_models; ++m) {
        if (N_per_model[m] < 0) return ms2_fail(MS2_EINVAL, "negative molecule count");
        Nt += N_per_model[m];
    }
    if (Nt < 2 || Nt > NA_NMAX)
        return ms2_fail(MS2_EINVAL, "ms2_forces_noalloc: %lld molecules outside 2..%d", Nt, NA_NMAX);
    // host side, a per-thread list reserved once (no heap traffic afterwards)
    static thread_local std::vector<int> species;
    if (species.capacity() < (size_t)NA_NMAX) species.reserve(NA_NMAX);
    species.clear();
    for (int m = 0; m < n_models; ++m)
        for (int k = 0; k < N_per_model[m]; ++k) species.push_back(m);
    const int N = (int)Nt;
    if (!(box > 0) || !(cutoff > 0) || !(cutoff < 0.5 * box))
        return ms2_fail(MS2_EINVAL, "ms2_forces_noalloc: need box > 0 and 0 < cutoff < box/2");
    ms2_options o;
    ms2_default_options(&o);
    if (opt) o = *opt;
    if (o.fp64) return ms2_fail(MS2_EINVAL, "ms2_forces_noalloc: FP32 site-pair arithmetic only (opt->fp64 must be 0)");

    SysParams hp;
    ms2_fill_params(hp, models, n_models, species, box, cutoff, elec, o, 1.0);
    unsigned ljm = 0, qm = 0, dm = 0;
    for (int m = 0; m < hp.n_species; ++m)
        for (int a = 0; a < hp.n_sites[m]; ++a) {
            if (hp.ljt[m][a] >= 0) ljm |= 1u << a;
            if (hp.q[m][a] != 0.f) qm |= 1u << a;
            if (hp.bdip[m][a][0] != 0 || hp.bdip[m][a][1] != 0 || hp.bdip[m][a][2] != 0) dm |= 1u << a;
        }
    int ns = 1;
    int tile = 0;
    bool multi = false;
    void *fn = ms2_pick_pair_kernel(hp.ns, ljm, qm, dm, hp.elec, hp.multi != 0, &ns, &tile, &multi, false);
    if (ns > NA_NS) return ms2_fail(MS2_EINVAL, "ms2_forces_noalloc: at most %d site slots", NA_NS);
    hp.ns = ns;
    double coulomb, kconv, uconst, wbg, ulrc, plrc;
    ms2_unit_constants(o.reduced != 0, &coulomb, &kconv);
    ms2_energy_constants(hp, species, 1.0, cutoff, o.lrc != 0, coulomb, &uconst, &wbg, &ulrc, &plrc);

    unsigned char *base = nullptr;
    int sms = 0;
    st = scratch_base(&base, &sms, fn);
    if (st != MS2_OK) return st;
    cudaStream_t sm = (cudaStream_t)stream;

    DevSys d;
    memset(&d, 0, sizeof d);
    d.N = N;
    d.ns = ns;
    const int wpb = 8, iblocks = (N + wpb - 1) / wpb;
    d.jsplit = std::max(1, std::min(NA_JS, (sms * 2) / std::max(iblocks, 1)));
    d.nunits = (N + 7) / 8;
    d.X = (uint32_t *)(base + O_X);
    d.s = (float *)(base + O_S);
    d.mu = hp.has_dipole ? (float *)(base + O_MU) : nullptr;
    d.mum = hp.elec == ELEC_RF ? (float *)(base + O_MUM) : nullptr;
    d.part = (float *)(base + O_PART);
    d.F = (double *)(base + O_F);
    d.tau = (double *)(base + O_TAU);
    d.Ui = (double *)(base + O_UI);
    d.npart = (int *)(base + O_NP);
    d.blk = (double *)(base + O_BLK);
    d.counter = (unsigned int *)(base + O_CNT);
    d.scal = (double *)(base + O_SCAL);
    d.species = (int *)(base + O_SPEC);
    d.R = (double *)(base + O_R);
    d.q = (double *)(base + O_Q);
    d.v = (double *)(base + O_V);
    d.Lm = (double *)(base + O_L);
    const SysParams *dP = (const SysParams *)(base + O_PARAMS);

    // inputs, and what must start at zero (the last-block counter, the
    // velocities and angular momenta the reduction reads, the scalars), all set
    // by one kernel from values passed by value
    NaSetup c;
    memset(&c, 0, sizeof c);
    c.uconst = uconst;
    c.ulrc = ulrc;
    c.plrc = plrc;
    c.wbg = wbg;
    c.n_models = n_models;
    for (int m = 0; m < n_models; ++m) c.counts[m] = N_per_model[m];

    const int range = (N + d.jsplit - 1) / d.jsplit;
    int TJ = std::max(32, range);
    while (ms2_pair_smem_bytes(ns, tile, multi, TJ, wpb) > 96 * 1024 && TJ > 64) TJ = (TJ + 1) / 2;
    const size_t smem = ms2_pair_smem_bytes(ns, tile, multi, TJ, wpb);

    k_noalloc_setup<<<(N + 127) / 128, 128, 0, sm>>>(hp, c, d, (SysParams *)(base + O_PARAMS), R_dev, q_dev);
    k_build<<<(4 * N + 127) / 128, 128, 0, sm>>>(dP, d);
    void (*pair)(const SysParams *, DevSys, int) = (void (*)(const SysParams *, DevSys, int))fn;
    pair<<<dim3(iblocks, d.jsplit), wpb * 32, smem, sm>>>(dP, d, TJ);
    k_reduce<<<(d.nunits + 3) / 4, 128, 0, sm>>>(dP, d, 1 /* sum the partials only */);
    k_aos3<<<(N + 127) / 128, 128, 0, sm>>>(d.F, F_dev, N);
    k_aos3<<<(N + 127) / 128, 128, 0, sm>>>(d.tau, tau_dev, N);
    ms2_count_launches(6);
    MS2_CUDA_OK(cudaGetLastError());
    // U and W are adjacent scalars
    MS2_CUDA_OK(cudaMemcpyAsync(UW_dev, d.scal + SC_UTOT, 2 * sizeof(double), cudaMemcpyDeviceToDevice, sm));
    return MS2_OK;
}

extern "C" size_t ms2_noalloc_scratch_bytes(void) { return NOALLOC_BYTES; }
