// Batched systems: persistent kernels that advance many independent systems,
// one thread block per system for a whole chunk of steps (drift + rotation +
// site build, optional RDF sample, partner search + site-pair forces, fixed-
// order reduction with the isokinetic factor), taking the next system from a
// longest-first work list when done.  A step needs only __syncthreads(): no
// grid-wide barrier.  Each model kind (slot pattern) has its own kernel, so each
// keeps its own register budget; the kinds run concurrently on forked streams.
//
// Every per-system result depends only on the system and its fixed tile (the
// whole system in one shared-memory tile): warps take molecules round-robin,
// and the system sums are taken over fixed chunks of 32 molecules in chunk
// order.  A system therefore gives bit-identical results alone, in any batch,
// and with any block size the autotuner picks.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "integrate_dev.cuh"
#include "ms2_host.h"
#include "pair_engine.cuh"

using namespace pair_engine;
using namespace integ;

namespace {

enum Kind { K_LJ1 = 0, K_W3RF, K_ST3RF, K_G4, K_G4D, K_COUNT };
const char *kKindName[K_COUNT] = {"lj1", "water3_rf", "stockmayer3_rf", "generic4", "generic4_dipole"};

struct BatchEntry {
    const SysParams *P;
    DevSys S;
    int TJ;
    int rdf_every;
    long long step0;  // step counter of the system before this launch
    double *chunk;    // [ceil(N/32)][Q_N] partial sums of the fixed-order reduction
};

constexpr int RDF_SMEM_MAX = 4096;  // histogram cells staged in shared memory

}  // namespace

// ------------------------------------------------------------------ phases
// drift: one quad of lanes per molecule (lanes 0-2 components, lane 3 rotation)
__device__ __forceinline__ void batch_drift(const SysParams *__restrict__ P, const DevSys &S) {
    const int N = S.N, c = threadIdx.x & 3;
    const double dt = P->dt, lam = S.scal[SC_LAMBDA];
    for (int base = 0; base < N; base += blockDim.x >> 2) {
        const int i = base + (threadIdx.x >> 2);
        const bool on = i < N;
        const int ii = on ? i : 0, sp = S.species[ii];
        double q[4] = {S.q[ii], S.q[N + ii], S.q[2 * N + ii], S.q[3 * N + ii]};
        if (c < 3) {
            if (on) {
                const double v = lam * (S.v[c * N + i] + dt * P->kconv * P->inv_mass[sp] * S.F[c * N + i]);
                S.v[c * N + i] = v;
                S.R[c * N + i] += dt * v;
            }
        } else {
            const double ct = dt * P->kconv;
            double L[3];
            for (int k = 0; k < 3; ++k) {
                L[k] = lam * (S.Lm[k * N + ii] + ct * S.tau[k * N + ii]);
                if (on) S.Lm[k * N + i] = L[k];
            }
            const double *Ii = P->Iinv[sp];
            if (Ii[0] != 0.0 || Ii[1] != 0.0 || Ii[2] != 0.0) {
                double q1[4];
                rotate_q(Ii, q, L, dt, P->quat_iters, q1);
                for (int k = 0; k < 4; ++k) {
                    q[k] = q1[k];
                    if (on) S.q[k * N + i] = q1[k];
                }
            }
        }
        for (int k = 0; k < 4; ++k) q[k] = __shfl_sync(0xffffffffu, q[k], (threadIdx.x & 28) | 3);
        if (c < 3 && on) build_row(P, S, i, c, q, S.R[c * N + i], S.species[i]);
    }
}

// RDF sample of the current configuration into a shared-memory histogram
__device__ void batch_rdf(const SysParams *__restrict__ P, const DevSys &S, unsigned *hist) {
    const int N = S.N, NS = S.ns, nb = S.rdf_bins, rows = S.rdf_rows, T = P->n_ljt;
    for (int k = threadIdx.x; k < rows * nb; k += blockDim.x) hist[k] = 0u;
    __syncthreads();
    const float l2l = P->lat_to_len, l2 = P->len_to_lat, rmax2 = S.rdf_rmax2, inv_dr = S.rdf_inv_dr;
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < N; i += nw) {
        const int spi = S.species[i];
        for (int a = 0; a < NS; ++a) {
            const int ta = S.rdf_kind[spi * MS2_MAXS + a];
            if (ta < 0) continue;
            uint32_t Xa[3];
            for (int c = 0; c < 3; ++c)
                Xa[c] = S.X[c * N + i] + (uint32_t)__float2int_rn(S.s[(c * NS + a) * N + i] * l2);
            for (int j = i + 1 + lane; j < N; j += 32) {
                const int spj = S.species[j];
                for (int b = 0; b < NS; ++b) {
                    const int tb = S.rdf_kind[spj * MS2_MAXS + b];
                    if (tb < 0) continue;
                    float r2 = 0.f;
                    for (int c = 0; c < 3; ++c) {
                        const uint32_t Xb = S.X[c * N + j] + (uint32_t)__float2int_rn(S.s[(c * NS + b) * N + j] * l2);
                        const float d = (float)(int)(Xb - Xa[c]) * l2l;
                        r2 += d * d;
                    }
                    if (!(r2 < rmax2)) continue;
                    const int bin = (int)(sqrtf(r2) * inv_dr);
                    if (bin >= nb) continue;
                    const int t1 = min(ta, tb), t2 = max(ta, tb);
                    atomicAdd(&hist[(t1 * T - t1 * (t1 - 1) / 2 + (t2 - t1)) * nb + bin], 1u);
                }
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < rows * nb; k += blockDim.x)
        if (hist[k]) atomicAdd(&S.rdf[k], (unsigned long long)hist[k]);
}

// reduction: lane = molecule within a chunk of 32, chunks round-robin over the
// warps, chunk sums in a fixed shuffle tree, then chunk order; the step scalars
// and the isokinetic factor for the next drift
__device__ void batch_reduce(const SysParams *__restrict__ P, const DevSys &S, double *chunk) {
    const int N = S.N, nch = (N + 31) >> 5;
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double dt = P->dt, kc = P->kconv;
    for (int ch = warp; ch < nch; ch += nw) {
        const int i = ch * 32 + lane;
        double r[Q_N] = {0, 0, 0, 0, 0, 0};
        if (i < N) {
            const int sp = S.species[i];
            const double M = P->mass[sp];
            const double q[4] = {S.q[i], S.q[N + i], S.q[2 * N + i], S.q[3 * N + i]};
            double fm = 0;
            for (int c = 0; c < 3; ++c) {
                double col[3];
                rot_column(q, c, col);
                const double F = S.F[c * N + i], v = S.v[c * N + i];
                fm = fmax(fm, fabs(F));
                const double L0 = S.Lm[i], L1 = S.Lm[N + i], L2 = S.Lm[2 * N + i];
                const double t0 = S.tau[i], t1 = S.tau[N + i], t2 = S.tau[2 * N + i];
                const double lb = col[0] * L0 + col[1] * L1 + col[2] * L2;
                const double lb1 = lb + dt * kc * (col[0] * t0 + col[1] * t1 + col[2] * t2);
                const double Ii = P->Iinv[sp][c];
                const double v1 = v + dt * kc * P->inv_mass[sp] * F;
                r[Q_KTR] += 0.5 * M * v * v;
                r[Q_KROT] += 0.5 * Ii * lb * lb;
                r[Q_K1] += 0.5 * M * v1 * v1 + 0.5 * Ii * lb1 * lb1;
            }
            r[Q_U] = S.Ui[i] + S.Ui[N + i] + S.Ui[2 * N + i];
            r[Q_W] = S.Ui[3 * N + i];
            r[Q_BAD] = fm < 1e30 ? 0.0 : 1.0;
        }
        for (int k = 0; k < Q_N; ++k) {
            const double x = warp_sum(r[k]);
            if (lane == 0) chunk[ch * Q_N + k] = x;
        }
    }
    __syncthreads();
    __shared__ double tot[Q_N];
    if (warp == 0) {
        for (int k = 0; k < Q_N; ++k) {
            double x = 0;
            for (int ch = lane; ch < nch; ch += 32) x += chunk[ch * Q_N + k];
            x = warp_sum(x);
            if (lane == 0) tot[k] = x;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) finish_step(P, S, RED_SUM | RED_RECORD | RED_LAMBDA, tot);
    __syncthreads();
}

template <int NS, unsigned LJM, unsigned QM, unsigned DM, int ELEC, bool MULTI>
__global__ void __launch_bounds__(256) k_batch(const BatchEntry *__restrict__ tab, const int *__restrict__ order,
                                               int n, unsigned int *next, int nsteps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Eng = PairWarp<NS, LJM, QM, DM, ELEC, MULTI>;
    __shared__ int cur;
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) cur = (int)atomicAdd(next, 1u);
        __syncthreads();
        if (cur >= n) return;
        const BatchEntry &e = tab[order[cur]];
        const SysParams *P = e.P;
        const DevSys S = e.S;
        const int N = S.N, TJ = e.TJ;
        Smem sm = carve<NS, Eng::DMU, MULTI>(smem_raw, TJ, nw);
        unsigned *hist = (unsigned *)(smem_raw + pair_engine::smem_bytes(NS, Eng::DMU, MULTI, TJ, nw));
        int *wq = sm.queue + warp * 64;
        load_tables<MULTI>(P, sm);
        Eng eng;
        eng.setup(P);
        for (int st = 0; st < nsteps; ++st) {
            batch_drift(P, S);
            __syncthreads();
            if (S.rdf && e.rdf_every > 0 && ((e.step0 + st + 1) % e.rdf_every) == 0) batch_rdf(P, S, hist);
            stage_tile<NS, Eng::DMU, MULTI>(sm, S, 0, N, TJ, Eng::MOLD && eng.rfq);
            __syncthreads();
            for (int i = warp; i < N; i += nw) {
                eng.begin(P, S, i);
                eng.scan(sm, TJ, 0, N, wq, lane);
                const PairOut o = eng.finish(lane);
                if (lane == 0) {
                    for (int k = 0; k < 3; ++k) {
                        S.F[k * N + i] = (double)o.F[k];
                        S.tau[k * N + i] = (double)o.T[k];
                    }
                    S.Ui[i] = o.ulj;
                    S.Ui[N + i] = o.uqq;
                    S.Ui[2 * N + i] = o.udd;
                    S.Ui[3 * N + i] = o.w;
                    S.npart[i] = o.np;
                }
            }
            __syncthreads();
            batch_reduce(P, S, e.chunk);
        }
    }
}

namespace {
typedef void (*BatchFn)(const BatchEntry *, const int *, int, unsigned int *, int);
const BatchFn kBatchFn[K_COUNT] = {
    &k_batch<1, 1u, 0u, 0u, ELEC_NONE, false>,
    &k_batch<3, 1u, 7u, 0u, ELEC_RF, false>,
    &k_batch<3, 3u, 0u, 4u, ELEC_RF, false>,
    &k_batch<4, 0xFu, 0xFu, 0u, -1, true>,
    &k_batch<4, 0xFu, 0xFu, 0xFu, -1, true>,
};
const int kKindNS[K_COUNT] = {1, 3, 3, 4, 4};
const bool kKindDMU[K_COUNT] = {false, false, true, false, true};
const bool kKindMulti[K_COUNT] = {false, false, false, true, true};

int kind_of(ms2_system s) {
    const SysParams &P = s->hp;
    if (P.ns == 1 && s->ljm == 1u && s->qm == 0 && s->dm == 0 && P.elec == ELEC_NONE && !P.multi) return K_LJ1;
    if (P.ns == 3 && s->ljm == 1u && s->qm == 7u && s->dm == 0 && P.elec == ELEC_RF && !P.multi) return K_W3RF;
    if (P.ns == 3 && s->ljm == 3u && s->qm == 0 && s->dm == 4u && P.elec == ELEC_RF && !P.multi) return K_ST3RF;
    if (P.ns <= 4) return s->dm ? K_G4D : K_G4;
    return -1;
}

size_t batch_smem(int kind, int N, int threads, int rdf_cells) {
    return pair_engine::smem_bytes(kKindNS[kind], kKindDMU[kind], kKindMulti[kind], N, threads / 32) +
           sizeof(unsigned) * (size_t)std::max(rdf_cells, 1);
}

// ---------------------------------------------------------- autotune cache
std::mutex g_tune_mu;
std::string tune_path() {
    const char *p = getenv("MS2_TUNE_CACHE");
    if (p && *p) return p;
    const char *h = getenv("HOME");
    return std::string(h ? h : "/tmp") + "/.cache/ms2_gb300_tune.txt";
}
std::map<std::string, int> load_tune() {
    std::map<std::string, int> m;
    std::ifstream f(tune_path());
    std::string k;
    int v;
    while (f >> k >> v) m[k] = v;
    return m;
}
void store_tune(const std::string &key, int v) {
    std::map<std::string, int> m = load_tune();
    m[key] = v;
    const std::string p = tune_path();
    const std::string dir = p.substr(0, p.find_last_of('/'));
    if (!dir.empty()) {
        std::string cmd = dir;  // create the directory without a shell
        for (size_t k = 1; k <= cmd.size(); ++k)
            if (k == cmd.size() || cmd[k] == '/') {
                std::string sub = cmd.substr(0, k);
                (void)!mkdir(sub.c_str(), 0755);
            }
    }
    std::ofstream f(p + ".tmp");
    for (auto &kv : m) f << kv.first << " " << kv.second << "\n";
    f.close();
    rename((p + ".tmp").c_str(), p.c_str());
}
}  // namespace

struct ms2_batch_s {
    std::vector<ms2_system> sys;
    cudaStream_t stream = nullptr;
    DevAlloc al;
    BatchEntry *dtab = nullptr;
    std::vector<BatchEntry> htab;
    int *dorder[K_COUNT] = {nullptr};
    std::vector<int> order[K_COUNT];
    unsigned *dnext = nullptr;  // one counter per kind
    int threads[K_COUNT] = {0};
    size_t smem[K_COUNT] = {0};
    int grid[K_COUNT] = {0};
    cudaStream_t ks[K_COUNT] = {nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join[K_COUNT] = {nullptr};
    int chunk = 100;
};

// trial = autotuner run: no RDF samples, no step counters
static ms2_status batch_launch(ms2_batch b, int nsteps, bool trial = false) {
    for (size_t k = 0; k < b->sys.size(); ++k) {
        b->htab[k].step0 = b->sys[k]->step;
        b->htab[k].rdf_every = (!trial && b->sys[k]->d.rdf) ? b->sys[k]->rdf_every : 0;
        b->htab[k].S = b->sys[k]->d;
    }
    MS2_CUDA_OK(cudaMemcpyAsync(b->dtab, b->htab.data(), sizeof(BatchEntry) * b->htab.size(), cudaMemcpyHostToDevice,
                                b->stream));
    MS2_CUDA_OK(cudaMemsetAsync(b->dnext, 0, sizeof(unsigned) * K_COUNT, b->stream));
    MS2_CUDA_OK(cudaEventRecord(b->ev_fork, b->stream));
    for (int k = 0; k < K_COUNT; ++k) {
        if (b->order[k].empty()) continue;
        MS2_CUDA_OK(cudaStreamWaitEvent(b->ks[k], b->ev_fork, 0));
        kBatchFn[k]<<<b->grid[k], b->threads[k], b->smem[k], b->ks[k]>>>(b->dtab, b->dorder[k], (int)b->order[k].size(),
                                                                         b->dnext + k, nsteps);
        ms2_count_launches(1);
        MS2_CUDA_OK(cudaGetLastError());
        MS2_CUDA_OK(cudaEventRecord(b->ev_join[k], b->ks[k]));
        MS2_CUDA_OK(cudaStreamWaitEvent(b->stream, b->ev_join[k], 0));
    }
    if (trial) return MS2_OK;
    for (ms2_system s : b->sys) {
        s->step += nsteps;
        if (s->d.rdf && s->rdf_every > 0)
            s->rdf_samples += (int)(s->step / s->rdf_every - (s->step - nsteps) / s->rdf_every);
    }
    return MS2_OK;
}

static ms2_status set_shape(ms2_batch b, int k, int threads) {
    int maxN = 0, rdf = 0;
    for (int idx : b->order[k]) {
        maxN = std::max(maxN, b->sys[idx]->N);
        rdf = std::max(rdf, b->sys[idx]->d.rdf ? b->sys[idx]->d.rdf_rows * b->sys[idx]->d.rdf_bins : 0);
    }
    b->threads[k] = threads;
    b->smem[k] = batch_smem(k, maxN, threads, rdf);
    MS2_CUDA_OK(cudaFuncSetAttribute((const void *)kBatchFn[k], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)std::max<size_t>(b->smem[k], 48 * 1024)));
    int per_sm = 0;
    MS2_CUDA_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kBatchFn[k], threads, b->smem[k]));
    if (per_sm < 1) return ms2_fail(MS2_EINVAL, "batch kind %s: %d threads do not fit one SM", kKindName[k], threads);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->grid[k] = std::min((int)b->order[k].size(), per_sm * sms);
    return MS2_OK;
}

// State the tuner touches, saved and restored around each trial.
static ms2_status snapshot_state(ms2_batch b, std::vector<void *> &buf, bool save) {
    size_t idx = 0;
    for (ms2_system s : b->sys) {
        const int N = s->N;
        struct { void *p; size_t n; } arr[] = {
            {s->d.R, 3 * sizeof(double) * N}, {s->d.v, 3 * sizeof(double) * N}, {s->d.q, 4 * sizeof(double) * N},
            {s->d.Lm, 3 * sizeof(double) * N}, {s->d.F, 3 * sizeof(double) * N}, {s->d.tau, 3 * sizeof(double) * N},
            {s->d.Ui, 4 * sizeof(double) * N}, {s->d.npart, sizeof(int) * N}, {s->d.X, 3 * sizeof(uint32_t) * N},
            {s->d.s, 3 * s->ns * sizeof(float) * N}, {s->d.scal, sizeof(double) * SC_COUNT_},
            {s->d.acc, sizeof(double) * AC_COUNT_}};
        for (auto &a : arr) {
            if (save) {
                void *p = nullptr;
                MS2_CUDA_OK(b->al.alloc(&p, a.n));
                buf.push_back(p);
                MS2_CUDA_OK(cudaMemcpyAsync(p, a.p, a.n, cudaMemcpyDeviceToDevice, b->stream));
            } else {
                MS2_CUDA_OK(cudaMemcpyAsync(a.p, buf[idx++], a.n, cudaMemcpyDeviceToDevice, b->stream));
            }
        }
        if (s->mum_bytes()) {
            if (save) {
                void *p = nullptr;
                MS2_CUDA_OK(b->al.alloc(&p, s->mum_bytes()));
                buf.push_back(p);
                MS2_CUDA_OK(cudaMemcpyAsync(p, s->d.mum, s->mum_bytes(), cudaMemcpyDeviceToDevice, b->stream));
            } else {
                MS2_CUDA_OK(cudaMemcpyAsync(s->d.mum, buf[idx++], s->mum_bytes(), cudaMemcpyDeviceToDevice, b->stream));
            }
        }
        if (s->mu_bytes()) {
            if (save) {
                void *p = nullptr;
                MS2_CUDA_OK(b->al.alloc(&p, s->mu_bytes()));
                buf.push_back(p);
                MS2_CUDA_OK(cudaMemcpyAsync(p, s->d.mu, s->mu_bytes(), cudaMemcpyDeviceToDevice, b->stream));
            } else {
                MS2_CUDA_OK(cudaMemcpyAsync(s->d.mu, buf[idx++], s->mu_bytes(), cudaMemcpyDeviceToDevice, b->stream));
            }
        }
    }
    return MS2_OK;
}

// Autotuner: per model kind, the block size (128 or 256 threads) that runs one
// step of this batch fastest; results cached on disk by (kind, size bucket).
static ms2_status tune(ms2_batch b) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::map<std::string, int> cache = load_tune();
    std::string key[K_COUNT];
    bool need = false;
    for (int k = 0; k < K_COUNT; ++k) {
        if (b->order[k].empty()) continue;
        std::vector<int> ns;
        for (int idx : b->order[k]) ns.push_back(b->sys[idx]->N);
        std::sort(ns.begin(), ns.end());
        int med = ns[ns.size() / 2], bucket = 1;
        while (bucket < med) bucket <<= 1;
        int cnt = 1;
        while (cnt < (int)ns.size()) cnt <<= 1;
        std::ostringstream os;
        os << "v1/" << kKindName[k] << "/N" << bucket << "/S" << cnt;
        key[k] = os.str();
        auto it = cache.find(key[k]);
        if (it != cache.end() && set_shape(b, k, it->second) == MS2_OK) continue;
        need = true;
    }
    if (!need) return MS2_OK;
    std::vector<void *> saved;
    ms2_status st = snapshot_state(b, saved, true);
    if (st != MS2_OK) return st;
    cudaEvent_t e0, e1;
    MS2_CUDA_OK(cudaEventCreate(&e0));
    MS2_CUDA_OK(cudaEventCreate(&e1));
    for (int k = 0; k < K_COUNT; ++k) {
        if (b->order[k].empty() || cache.count(key[k])) continue;
        float best = 1e30f;
        int best_t = 256;
        for (int t : {128, 256}) {
            if (set_shape(b, k, t) != MS2_OK) continue;
            // only kind k runs in a trial
            std::vector<int> keep[K_COUNT];
            for (int j = 0; j < K_COUNT; ++j)
                if (j != k) std::swap(keep[j], b->order[j]);
            MS2_CUDA_OK(cudaEventRecord(e0, b->stream));
            st = batch_launch(b, 1, true);
            MS2_CUDA_OK(cudaEventRecord(e1, b->stream));
            for (int j = 0; j < K_COUNT; ++j)
                if (j != k) std::swap(keep[j], b->order[j]);
            if (st != MS2_OK) return st;
            MS2_CUDA_OK(cudaEventSynchronize(e1));
            float ms = 0;
            MS2_CUDA_OK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                best_t = t;
            }
            st = snapshot_state(b, saved, false);
            if (st != MS2_OK) return st;
        }
        MS2_CUDA_OK(cudaStreamSynchronize(b->stream));
        st = set_shape(b, k, best_t);
        if (st != MS2_OK) return st;
        store_tune(key[k], best_t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    MS2_CUDA_OK(cudaStreamSynchronize(b->stream));
    return MS2_OK;
}

// whether the batch kernels take this system (used by the server)
bool ms2_batch_accepts(ms2_system s) {
    if (!s || s->hp.integrator != MS2_INT_LEAPFROG_Q || s->fp64 || s->hp.elec == ELEC_EWALD || s->hp.massieu ||
        s->d.gk || s->res_every > 0 || s->hf_every > 0)
        return false;
    const int kind = kind_of(s);
    if (kind < 0) return false;
    const int rdf = s->d.rdf ? s->d.rdf_rows * s->d.rdf_bins : 0;
    if (rdf > RDF_SMEM_MAX) return false;
    return batch_smem(kind, s->N, 128, rdf) <= 227 * 1024;
}

extern "C" ms2_status ms2_batch_create(const ms2_system *systems, int n, ms2_batch *out) {
    if (!out || !systems || n < 1) return ms2_fail(MS2_EINVAL, "need n >= 1 systems and an output handle");
    *out = nullptr;
    ms2_batch b = new ms2_batch_s();
    // the batch owns its stream: it must outlive none of the systems' streams
    for (int k = 0; k < n; ++k) {
        ms2_system s = systems[k];
        if (!s) { delete b; return ms2_fail(MS2_EINVAL, "system %d is null", k); }
        if (s->hp.integrator != MS2_INT_LEAPFROG_Q || s->fp64 || s->hp.elec == ELEC_EWALD || s->hp.massieu || s->d.gk ||
            s->res_every > 0 || s->hf_every > 0) {
            delete b;
            return ms2_fail(MS2_EINVAL, "system %d: batches take leapfrog systems with FP32 pair arithmetic and "
                                        "reaction field or no electrostatics, without Massieu, conductivity, "
                                        "residence or heat-flux sampling", k);
        }
        const int kind = kind_of(s);
        if (kind < 0) { delete b; return ms2_fail(MS2_EINVAL, "system %d: more than 4 site slots", k); }
        const int rdf = s->d.rdf ? s->d.rdf_rows * s->d.rdf_bins : 0;
        if (rdf > RDF_SMEM_MAX) { delete b; return ms2_fail(MS2_EINVAL, "system %d: RDF histogram too large for a batch", k); }
        if (batch_smem(kind, s->N, 128, rdf) > 227 * 1024) {
            delete b;
            return ms2_fail(MS2_EINVAL, "system %d: %d molecules do not fit one block's shared memory", k, s->N);
        }
        b->sys.push_back(s);
        b->order[kind].push_back(k);
    }
    // longest first: cost ~ N^2 (all pairs are tested; partners ~ N * const)
    for (int k = 0; k < K_COUNT; ++k)
        std::stable_sort(b->order[k].begin(), b->order[k].end(),
                         [&](int x, int y) { return b->sys[x]->N > b->sys[y]->N; });
    b->htab.resize(n);
    ms2_status st = MS2_OK;
    auto fail = [&](ms2_status s2) { ms2_batch_destroy(b); return s2; };
    {
        cudaError_t e0 = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e0 != cudaSuccess) return fail(ms2_fail_cuda(e0, "batch stream", __FILE__, __LINE__));
    }
    for (int k = 0; k < n; ++k) {
        ms2_system s = b->sys[k];
        BatchEntry &e = b->htab[k];
        e.P = s->dP;
        e.S = s->d;
        e.TJ = s->N;
        e.rdf_every = 0;
        e.step0 = s->step;
        cudaError_t ce = b->al.alloc((void **)&e.chunk, sizeof(double) * Q_N * ((s->N + 31) / 32));
        if (ce != cudaSuccess) return fail(ms2_fail_cuda(ce, "batch scratch", __FILE__, __LINE__));
    }
    cudaError_t ce = b->al.alloc((void **)&b->dtab, sizeof(BatchEntry) * n);
    if (ce == cudaSuccess) ce = b->al.alloc((void **)&b->dnext, sizeof(unsigned) * K_COUNT);
    for (int k = 0; k < K_COUNT && ce == cudaSuccess; ++k) {
        if (b->order[k].empty()) continue;
        ce = b->al.alloc((void **)&b->dorder[k], sizeof(int) * b->order[k].size());
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(b->dorder[k], b->order[k].data(), sizeof(int) * b->order[k].size(),
                                 cudaMemcpyHostToDevice, b->stream);
        if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&b->ks[k], cudaStreamNonBlocking);
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
    }
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (ce != cudaSuccess) return fail(ms2_fail_cuda(ce, "batch set-up", __FILE__, __LINE__));
    for (int k = 0; k < K_COUNT; ++k)
        if (!b->order[k].empty() && (st = set_shape(b, k, 256)) != MS2_OK) return fail(st);
    // the systems' own queued work comes first
    for (ms2_system s : b->sys)
        if (s->stream != b->stream) {
            cudaStreamSynchronize(s->stream);
        }
    st = tune(b);
    if (st != MS2_OK) return fail(st);
    *out = b;
    return MS2_OK;
}

extern "C" ms2_status ms2_batch_step(ms2_batch b, long long n) {
    if (!b) return ms2_fail(MS2_EINVAL, "null batch");
    if (n < 0) return ms2_fail(MS2_EINVAL, "negative step count");
    for (ms2_system s : b->sys)
        if (s->stream != b->stream) cudaStreamSynchronize(s->stream);
    long long done = 0;
    while (done < n) {
        const int m = (int)std::min<long long>(b->chunk, n - done);
        ms2_status st = batch_launch(b, m);
        if (st != MS2_OK) return st;
        done += m;
    }
    // later work of each system on its own stream waits for the batch
    cudaEvent_t ev;
    MS2_CUDA_OK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    MS2_CUDA_OK(cudaEventRecord(ev, b->stream));
    for (ms2_system s : b->sys)
        if (s->stream != b->stream) MS2_CUDA_OK(cudaStreamWaitEvent(s->stream, ev, 0));
    cudaEventDestroy(ev);
    return MS2_OK;
}

extern "C" ms2_status ms2_batch_destroy(ms2_batch b) {
    if (!b) return MS2_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (int k = 0; k < K_COUNT; ++k) {
        if (b->ks[k]) cudaStreamDestroy(b->ks[k]);
        if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    b->al.release_all();
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return MS2_OK;
}
