// Batched systems: many independent systems advanced together by one
// cooperative persistent kernel per model kind (slot pattern), one 512-thread
// block per SM, for a chunk of steps.  Each step runs the phases of the
// single-system path over all systems of the kind at once, with a bounded grid
// barrier between phases:
//   drift      groups of 8 molecules (a quad per molecule), round-robin over all warps
//   pair       molecule items split into equal-cost contiguous ranges, one per
//              block; a block stages each system of its range in shared memory
//              and its warps take that system's items (owner warp per molecule,
//              the whole system as one j-range); RDF samples on the same tile
//   reduction  units of 8 molecules, round-robin over all warps
//   totals     one warp per system: fixed-order unit totals, the step record and
//              the thermostat factor of the next drift
// So work is balanced over the whole GPU at molecule granularity whatever the
// mix of sizes (no system waits on one block), and the kinds run one after the
// other on the batch stream.
//
// Every per-system result depends only on the system: its pair items, its
// reduction units and their orders are fixed by the system alone, not by the
// batch, the grid or the block size.  A system therefore gives bit-identical
// results alone, in any batch, and with any shape the autotuner picks.
#include <algorithm>
#include <chrono>
#include <cmath>
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

#include "ewald_dev.cuh"
#include "grid_dev.cuh"
#include "integrate_dev.cuh"
#include "ms2_host.h"
#include "pair_engine.cuh"

using namespace pair_engine;
using namespace integ;

namespace {

enum Kind { K_LJ1 = 0, K_W3RF, K_ST3RF, K_G4, K_G4D, K_ION3EW, K_COUNT };
const char *kKindName[K_COUNT] = {"lj1", "water3_rf", "stockmayer3_rf", "generic4", "generic4_dipole",
                                  "water_ions3_ewald"};

constexpr int MS_THREADS = 512;   // largest block shape (the autotuner may take 256)
constexpr int UNIT = 8;           // molecules per reduction unit (one quad pass of a warp)
constexpr int VB_PER_BLOCK = 4;   // pair-phase pieces per block of the grid (drawn dynamically), by default
constexpr int RDF_SMEM_MAX = 4096;  // histogram cells staged in shared memory
// candidate-list skin, in units of the cut-off.  Measured on the bench mix over
// 10^4 steps from lattices (ms per step in the first and last 2000 steps):
// 0.15 -> 2.45 / 2.67, 0.2 -> 2.45 / 2.63, 0.25 -> 2.50 / 2.73, 0.3 -> 2.52 / 2.76,
// 0.45 -> 2.65 / 2.87.  Small skins rebuild often while the lattices relax; large
// ones scan long lists once the dilute systems condense.
constexpr double kSkin = 0.2;

struct BatchEntry {
    const SysParams *P;
    DevSys S;         // the system's arrays, with jsplit = 1 and blk -> the batch's unit partials
    int units;        // reduction units: ceil(N / UNIT)
    int rdf_every;
    long long step0;  // step counter of the system before this launch
    // Candidate lists with a skin (kSkin r_c): per molecule, the molecules within r_c + skin
    // at the last build, in ascending order.  The exact centre test runs on them
    // each step until some molecule of the system has moved more than skin / 2
    // since the build (then no other molecule can have come within r_c), so the
    // partners are those of the full scan, in its order.  lcap = 0: full scans.
    uint16_t *nl;                 // [N][lcap]
    int *ncnt;                    // [N] candidates at the build (> lcap: that owner scans all)
    uint32_t *Xb;                 // [3][N] lattice centres at the build
    int *nflag;                   // non-zero: rebuild in this step's pair phase
    int lcap;
    unsigned long long rs2, sk2;  // (r_c + skin)^2 and (skin / 2)^2, lattice units, with margins
    // Ewald (reciprocal space): A(k) S(k) of the step, structure-factor and sum task counts
    float2 *AS;
    int nsb, nkc;
};

// launch arguments of one kind (device tables built on the host)
struct MsArgs {
    const BatchEntry *tab;
    int n_sys;
    const int2 *drift;     // drift groups (entry, first molecule), 8 molecules each
    int n_drift;
    const int4 *seg;       // pair segments (entry, first molecule, end, 0) ...
    const int *seg_off;    // ... of virtual block v: seg[seg_off[v] .. seg_off[v + 1])
    int n_vb;              // virtual blocks (pieces of equal estimated cost, in system order)
    const int2 *unit;      // reduction units (entry, unit)
    int n_unit;
    int Np;                // stride of the staged tile (largest N of the kind, multiple of 4)
    int nsteps;
    unsigned *bar, *err;   // barrier counter (zero at entry) and sticky timeout flag
    unsigned *work;        // pair-phase work counter (zero at entry): n_vb + grid draws a step
    // Ewald kinds: reciprocal-space tasks (entry, task): structure-factor tasks,
    // sum tasks, force tasks (one k chunk of a system, all its site groups)
    const int2 *ew_sk, *ew_sum, *ew_force;
    int n_sk, n_sum, n_force;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

}  // namespace

// ------------------------------------------------------------------ kernel
template <int NS, unsigned LJM, unsigned QM, unsigned DM, int ELEC, bool MULTI, int BT = MS_THREADS>
__global__ void __launch_bounds__(BT, 1) k_mstep(MsArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Eng = PairWarp<NS, LJM, QM, DM, ELEC, MULTI>;
    __shared__ double wtot[BT / 32][MS2_NRED];
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * nw + warp, W = gridDim.x * nw;
    const Smem sm = carve<NS, Eng::TILE, MULTI>(smem_raw, A.Np, nw);
    unsigned *hist = (unsigned *)(smem_raw + al16(pair_engine::smem_bytes(NS, Eng::TILE, MULTI, A.Np, nw)));
    int *wq = sm.queue + warp * QSTRIDE;
    unsigned target = 0, work_base = 0;
    __shared__ int s_vb;
    auto on_timeout = [&]() {
        for (int e = 0; e < A.n_sys; ++e) A.tab[e].S.scal[SC_KERR] = 1.0;
    };
    using grid_dev::grid_sync;
    for (int k = 0; k < A.nsteps; ++k) {
        // ---- drift + site build: kick with the last forces and thermostat factor
        for (int g = gw; g < A.n_drift; g += W) {
            const int2 d = A.drift[g];
            const BatchEntry &en = A.tab[d.x];
            const int i = d.y + (lane >> 2);
            const bool on = i < en.S.N;
            const double lam = __ldcg(en.S.scal + SC_LAMBDA);
            drift_quad<false>(en.P, en.S, global_view(en.S), i, i, on, lane & 3, false, lam);
            if (en.lcap) {  // displacement since the list build (lane c: component c), summed over the quad
                const int c = lane & 3;
                unsigned long long d2 = 0;
                if (on && c < 3) {
                    const int d = (int)(en.S.X[c * en.S.N + i] - __ldcg(en.Xb + c * en.S.N + i));
                    d2 = (unsigned long long)((long long)d * d);
                }
                d2 += __shfl_xor_sync(0xffffffffu, d2, 1);
                d2 += __shfl_xor_sync(0xffffffffu, d2, 2);
                if (c == 0 && d2 > en.sk2) *en.nflag = 1;
            }
        }
        grid_sync(A.bar, A.err, target, on_timeout);
        // ---- pair items (and RDF samples): the virtual blocks, drawn one at a
        // time from the work counter, so that a block that finishes early takes
        // the next piece; every block stops at its first draw past the end, so a
        // step takes exactly n_vb + grid draws.  Which block runs an item does
        // not change its result.
        for (;;) {
            if (threadIdx.x == 0) s_vb = (int)(atomicAdd(A.work, 1u) - work_base);
            __syncthreads();
            const int vb = s_vb;
            __syncthreads();  // read by all before thread 0 draws again
            if (vb >= A.n_vb) break;
        for (int sg = A.seg_off[vb]; sg < A.seg_off[vb + 1]; ++sg) {
            const int4 g = A.seg[sg];
            const BatchEntry &en = A.tab[g.x];
            const SysParams *P = en.P;
            const DevSys &S = en.S;
            const int N = S.N;
            const bool rdf = S.rdf && en.rdf_every > 0 && ((en.step0 + k + 1) % en.rdf_every) == 0;
            Eng e;
            e.setup(P);
            __syncthreads();  // the previous segment's tile is no longer read
            load_tables<MULTI>(P, sm);
            stage_tile<NS, DM, Eng::MOLD, MULTI>(sm, S, 0, N, A.Np, Eng::MOLD && e.rfq);
            if (rdf)
                for (int c = threadIdx.x; c < S.rdf_rows * S.rdf_bins; c += blockDim.x) hist[c] = 0u;
            __syncthreads();
            const bool build = en.lcap && __ldcg(en.nflag) != 0;  // the same in every block this step
            for (int i = g.y + warp; i < g.z; i += nw) {
                e.begin_tile(P, sm, A.Np, i);
                if (!en.lcap) {
                    e.scan(sm, A.Np, 0, N, wq, lane);
                } else if (build) {
                    const int nc = e.scan_build(sm, A.Np, N, wq, lane, en.nl + (size_t)i * en.lcap, en.lcap, en.rs2);
                    if (lane == 0) {
                        en.ncnt[i] = nc;
                        en.Xb[i] = e.Xi;
                        en.Xb[N + i] = e.Yi;
                        en.Xb[2 * N + i] = e.Zi;
                    }
                } else {
                    const int nc = __ldcg(en.ncnt + i);
                    if (nc > en.lcap)
                        e.scan(sm, A.Np, 0, N, wq, lane);
                    else
                        e.scan_list(sm, A.Np, en.nl + (size_t)i * en.lcap, nc, wq, lane);
                }
                const PairOut o = e.finish(lane);
                if (lane == 0) {
                    float *q = S.part + i;
                    q[PV_FX * N] = o.F[0]; q[PV_FY * N] = o.F[1]; q[PV_FZ * N] = o.F[2];
                    q[PV_TX * N] = o.T[0]; q[PV_TY * N] = o.T[1]; q[PV_TZ * N] = o.T[2];
                    q[PV_ULJ * N] = o.ulj; q[PV_UQQ * N] = o.uqq; q[PV_UDD * N] = o.udd; q[PV_W * N] = o.w;
                    q[PV_NP * N] = (float)o.np;
                    q[PV_VV * N] = o.vv;
                }
                if (rdf) rdf_molecule<NS, MULTI>(P, S, sm, A.Np, i, i + 1 + lane, 32, N, hist);
            }
            if (rdf) {  // uniform over the block
                __syncthreads();
                for (int c = threadIdx.x; c < S.rdf_rows * S.rdf_bins; c += blockDim.x)
                    if (hist[c]) atomicAdd(&S.rdf[c], (unsigned long long)hist[c]);
            }
        }
        }
        work_base += (unsigned)(A.n_vb + gridDim.x);
        grid_sync(A.bar, A.err, target, on_timeout);
        // ---- Ewald reciprocal space of every system of the kind: the tasks of
        // the single-system path (structure factor, sums, forces), each a function
        // of its system and index alone, a grid barrier after each kind of task
        constexpr int EWM = ELEC == ELEC_EWALD ? RED_EWALD : 0;
        if constexpr (ELEC == ELEC_EWALD) {
            for (int t = blockIdx.x; t < A.n_sk; t += gridDim.x) {
                const int2 w = A.ew_sk[t];
                const BatchEntry &en = A.tab[w.x];
                ewald::sk_task(en.P, en.S, w.y, smem_raw, threadIdx.x, blockDim.x);
            }
            grid_sync(A.bar, A.err, target, on_timeout);
            for (int t = blockIdx.x; t < A.n_sum; t += gridDim.x) {
                const int2 w = A.ew_sum[t];
                const BatchEntry &en = A.tab[w.x];
                ewald::sum_task(en.S, en.AS, w.y, en.nsb, smem_raw, threadIdx.x, blockDim.x);
            }
            grid_sync(A.bar, A.err, target, on_timeout);
            for (int e = gw; e < A.n_sys; e += W) {  // U_rec and W_rec of each system (one warp)
                const BatchEntry &en = A.tab[e];
                ewald::sum_finish(en.P, en.S, en.nkc, lane);
            }
            for (int t = blockIdx.x; t < A.n_force; t += gridDim.x) {
                const int2 w = A.ew_force[t];
                const BatchEntry &en = A.tab[w.x];
                const int M = en.S.nsite_q;
                for (int s0 = 0; s0 < M; s0 += blockDim.x) {
                    if (en.S.kx == 8)
                        ewald::force_task<9>(en.P, en.S, en.AS, s0, w.y, 1, smem_raw, threadIdx.x, blockDim.x);
                    else
                        ewald::force_task<0>(en.P, en.S, en.AS, s0, w.y, 1, smem_raw, threadIdx.x, blockDim.x);
                }
            }
            grid_sync(A.bar, A.err, target, on_timeout);
        }
        // ---- reduction units: F, tau, energies, kinetic energies (before and after the kick)
        for (int g = gw; g < A.n_unit; g += W) {
            const int2 u = A.unit[g];
            const BatchEntry &en = A.tab[u.x];
            reduce_unit<false>(en.P, en.S, global_io(en.S), RED_SUM | RED_LAMBDA | EWM, u.y, en.units, lane);
            if (u.y == 0 && lane == 0 && en.lcap) *en.nflag = 0;  // the pair phase has read it
        }
        grid_sync(A.bar, A.err, target, on_timeout);
        // ---- per system: totals (lane l sums units l, l + 32, ... in order, then
        // one fixed 8-value tree), the record, the next thermostat factor
        for (int s = gw; s < A.n_sys; s += W) {
            const BatchEntry &en = A.tab[s];
            double x[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int u = lane; u < en.units; u += 32)
#pragma unroll
                for (int q = 0; q < Q_N; ++q) x[q] += __ldcg(en.S.blk + (size_t)u * MS2_NRED + q);
            const double t = warp_sum8(x, lane);
            if ((lane & 3) == 0 && (lane >> 2) < Q_N) wtot[warp][lane >> 2] = t;
            __syncwarp();
            finish_step_warp(en.P, en.S, RED_SUM | RED_RECORD | RED_LAMBDA | EWM, wtot[warp], lane, en.S.acc,
                             global_consts(en.S));
            __syncwarp();
        }
        grid_sync(A.bar, A.err, target, on_timeout);
    }
}

namespace {
typedef void (*BatchFn)(MsArgs);
const BatchFn kBatchFn[K_COUNT] = {
    &k_mstep<1, 1u, 0u, 0u, ELEC_NONE, false>,
    &k_mstep<3, 1u, 7u, 0u, ELEC_RF, false>,
    &k_mstep<3, 3u, 0u, 4u, ELEC_RF, false>,
    &k_mstep<4, 0xFu, 0xFu, 0u, -1, true>,
    &k_mstep<4, 0xFu, 0xFu, 0xFu, -1, true>,
    &k_mstep<3, 1u, 7u, 0u, ELEC_EWALD, true>,
};
// 1024-thread shapes (64 registers a thread) where the pair work needs few
// registers and the scan's latency wants more warps: the point-LJ kind
const BatchFn kBatchFnWide[K_COUNT] = {&k_mstep<1, 1u, 0u, 0u, ELEC_NONE, false, 2 * MS_THREADS>, nullptr, nullptr,
                                       nullptr, nullptr, nullptr};
BatchFn kernel_of(int kind, int threads) { return threads > MS_THREADS ? kBatchFnWide[kind] : kBatchFn[kind]; }
const int kKindNS[K_COUNT] = {1, 3, 3, 4, 4, 3};
// tile layout of each kind's kernel (dipole slots kept, molecular dipoles kept)
const int kKindTile[K_COUNT] = {pair_engine::tile_code(0, false), pair_engine::tile_code(0, true),
                                 pair_engine::tile_code(1, false), pair_engine::tile_code(0, true),
                                 pair_engine::tile_code(4, true), pair_engine::tile_code(0, false)};
const bool kKindMulti[K_COUNT] = {false, false, false, true, true, true};

static_assert(PairWarp<1, 1u, 0u, 0u, ELEC_NONE, false>::TILE == tile_code(0, false) &&
                  PairWarp<3, 1u, 7u, 0u, ELEC_RF, false>::TILE == tile_code(0, true) &&
                  PairWarp<3, 3u, 0u, 4u, ELEC_RF, false>::TILE == tile_code(1, false) &&
                  PairWarp<4, 0xFu, 0xFu, 0u, -1, true>::TILE == tile_code(0, true) &&
                  PairWarp<4, 0xFu, 0xFu, 0xFu, -1, true>::TILE == tile_code(4, true) &&
                  PairWarp<3, 1u, 7u, 0u, ELEC_EWALD, true>::TILE == tile_code(0, false),
              "kKindTile matches the kinds' kernels");

// A batch launches one kernel per group: the systems of one model kind and one
// size class (up to BIG_N molecules, or more).  A kind's block shape and
// shared memory follow its largest system; the class split keeps a few large
// systems from setting them for all the small ones.  Which group runs a system
// never changes its results (they depend on the system alone).
constexpr int BIG_N = 2048;
constexpr int G_COUNT = 2 * K_COUNT;
inline int kind_of_group(int g) { return g >> 1; }
inline int group_of(int kind, int N) { return 2 * kind + (N > BIG_N ? 1 : 0); }

int kind_of(ms2_system s) {
    const SysParams &P = s->hp;
    if (P.ns == 1 && s->ljm == 1u && s->qm == 0 && s->dm == 0 && P.elec == ELEC_NONE && !P.multi) return K_LJ1;
    if (P.ns == 3 && s->ljm == 1u && s->qm == 7u && s->dm == 0 && P.elec == ELEC_RF && !P.multi) return K_W3RF;
    if (P.ns == 3 && s->ljm == 3u && s->qm == 0 && s->dm == 4u && P.elec == ELEC_RF && !P.multi) return K_ST3RF;
    if (P.elec == ELEC_EWALD)  // water and single-site ions (or water alone), |n| <= kmax per axis
        return (P.ns == 3 && s->ljm == 1u && s->qm == 7u && s->dm == 0) ? K_ION3EW : -1;
    if (P.ns == 4) return s->dm ? K_G4D : K_G4;
    return -1;
}

size_t batch_smem(int kind, int Np, int threads, int rdf_cells) {
    return al16(pair_engine::smem_bytes(kKindNS[kind], kKindTile[kind], kKindMulti[kind], Np, threads / 32)) +
           sizeof(unsigned) * (size_t)std::max(rdf_cells, 1);
}

// scratch of the reciprocal-space tasks of one Ewald system (they reuse the
// pair tile's shared memory after the pair phase)
size_t ewald_smem(ms2_system s, int threads) {
    if (s->hp.elec != ELEC_EWALD) return 0;
    const DevSys &d = s->d;
    return std::max({ewald::sk_smem(d.kx, d.ky, d.kz, d.sk_sites), ewald::sum_smem(),
                     ewald::force_smem(d.kx, d.kz, 1, threads)});
}

// relative cost of one pair item of system s (warp instructions, rough): the
// candidate scan over all N molecules plus the expected partners times the
// site pairs each evaluates
// (with candidate lists: the list, (1 + skin)^3 x the partners, at a higher
// cost per entry, plus a full scan about every 16 steps)
double item_cost(ms2_system s, bool lists) {
    const double L = s->hp.L, rc = s->rc;
    const double frac = std::min(1.0, 4.0 / 3.0 * M_PI * rc * rc * rc / (L * L * L));
    int sp = 0;
    for (int a = 0; a < 8; ++a)
        for (int c = 0; c < 8; ++c)
            if ((((s->ljm >> a) & (s->ljm >> c)) | ((s->qm >> a) & (s->qm >> c)) | ((s->dm >> a) & (s->dm >> c))) & 1u)
                ++sp;
    const double grow = (1.0 + kSkin) * (1.0 + kSkin) * (1.0 + kSkin);
    const double scan = lists ? 25.0 * std::min(1.0, grow * frac) + 20.0 / 16.0 : 20.0;
    return (double)s->N * (scan + frac * (25.0 * sp + 30.0));
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
    std::vector<int> order[G_COUNT];       // member systems of each group, in creation order
    std::vector<BatchEntry> htab[G_COUNT];
    BatchEntry *dtab[G_COUNT] = {nullptr};
    int2 *ddrift[G_COUNT] = {nullptr}, *dunit[G_COUNT] = {nullptr};
    int n_drift[G_COUNT] = {0}, n_unit[G_COUNT] = {0};
    int4 *dseg[G_COUNT] = {nullptr};
    int *dsegoff[G_COUNT] = {nullptr};
    int Np[G_COUNT] = {0}, rdf_cells[G_COUNT] = {0};
    // Ewald kinds: reciprocal-space task tables
    int2 *dew_sk[G_COUNT] = {nullptr}, *dew_sum[G_COUNT] = {nullptr}, *dew_force[G_COUNT] = {nullptr};
    int n_ew_sk[G_COUNT] = {0}, n_ew_sum[G_COUNT] = {0}, n_ew_force[G_COUNT] = {0};
    int threads[G_COUNT] = {0}, grid[G_COUNT] = {0};
    size_t smem[G_COUNT] = {0};
    unsigned *dbar = nullptr;  // [G_COUNT][3]: barrier counter, timeout flag, pair-phase work counter
    int nvb[G_COUNT] = {0};    // virtual blocks of each group's pair phase
    int vbpb[G_COUNT] = {0};   // ... per block of the grid (the tuned piece size)
    int *dnflag[G_COUNT] = {nullptr};  // candidate-list rebuild flags, one per system of the kind
    int chunk = 100;
    bool tune_shapes = true;  // false: cached shape or the default, no trial launches
};

// trial = autotuner run: no RDF samples, no step counters
static ms2_status set_shape(ms2_batch b, int k, int threads, int vb = VB_PER_BLOCK);

static ms2_status batch_launch(ms2_batch b, int nsteps, bool trial = false) {
    for (int k = 0; k < G_COUNT; ++k) {
        if (b->order[k].empty()) continue;
        std::vector<BatchEntry> &t = b->htab[k];
        int cells = b->rdf_cells[k];
        for (size_t e = 0; e < t.size(); ++e) {
            ms2_system s = b->sys[b->order[k][e]];
            // the system's current arrays (an RDF set up after the batch was made),
            // with the batch's own decomposition
            double *ublk = t[e].S.blk;
            t[e].S = s->d;
            t[e].S.jsplit = 1;
            t[e].S.nunits = t[e].units;
            t[e].S.blk = ublk;
            t[e].step0 = s->step;
            t[e].rdf_every = (!trial && s->d.rdf) ? s->rdf_every : 0;
            if (s->d.rdf) cells = std::max(cells, s->d.rdf_rows * s->d.rdf_bins);
        }
        if (cells > b->rdf_cells[k]) {  // a larger histogram than the shape reserves
            if (cells > RDF_SMEM_MAX) return ms2_fail(MS2_EINVAL, "RDF histogram too large for a batch");
            b->rdf_cells[k] = cells;
            ms2_status st = set_shape(b, k, b->threads[k], b->vbpb[k]);
            if (st != MS2_OK) st = set_shape(b, k, 256, b->vbpb[k]);
            if (st != MS2_OK) return st;
        }
        MS2_CUDA_OK(cudaMemcpyAsync(b->dtab[k], t.data(), sizeof(BatchEntry) * t.size(), cudaMemcpyHostToDevice,
                                    b->stream));
        MS2_CUDA_OK(cudaMemsetAsync(b->dbar + 3 * k, 0, 3 * sizeof(unsigned), b->stream));
        // the lists are rebuilt at the start of every launch (the states may have been set or stepped since)
        MS2_CUDA_OK(cudaMemsetAsync(b->dnflag[k], 1, sizeof(int) * t.size(), b->stream));
        MsArgs A;
        A.tab = b->dtab[k];
        A.n_sys = (int)t.size();
        A.drift = b->ddrift[k];
        A.n_drift = b->n_drift[k];
        A.seg = b->dseg[k];
        A.seg_off = b->dsegoff[k];
        A.n_vb = b->nvb[k];
        A.unit = b->dunit[k];
        A.n_unit = b->n_unit[k];
        A.Np = b->Np[k];
        A.nsteps = nsteps;
        A.bar = b->dbar + 3 * k;
        A.err = b->dbar + 3 * k + 1;
        A.work = b->dbar + 3 * k + 2;
        A.ew_sk = b->dew_sk[k];
        A.ew_sum = b->dew_sum[k];
        A.ew_force = b->dew_force[k];
        A.n_sk = b->n_ew_sk[k];
        A.n_sum = b->n_ew_sum[k];
        A.n_force = b->n_ew_force[k];
        void *args[] = {(void *)&A};
        MS2_CUDA_OK(cudaLaunchCooperativeKernel((const void *)kernel_of(kind_of_group(k), b->threads[k]), b->grid[k], b->threads[k], args, b->smem[k],
                                                b->stream));
        ms2_count_launches(1);
    }
    if (trial) return MS2_OK;
    for (ms2_system s : b->sys) {
        s->step += nsteps;
        if (s->d.rdf && s->rdf_every > 0)
            s->rdf_samples += (int)(s->step / s->rdf_every - (s->step - nsteps) / s->rdf_every);
    }
    return MS2_OK;
}

// block shape of kind k and the pair segments of each block: the kind's items
// (molecules, system by system) cut into grid ranges of equal estimated cost
static ms2_status set_shape(ms2_batch b, int k, int threads, int vb) {
    const int kind = kind_of_group(k);
    const BatchFn fn = kernel_of(kind, threads);
    if (!fn) return ms2_fail(MS2_EINVAL, "batch kind %s has no %d-thread shape", kKindName[kind], threads);
    b->threads[k] = threads;
    b->smem[k] = batch_smem(kind, b->Np[k], threads, b->rdf_cells[k]);
    for (int idx : b->order[k]) b->smem[k] = std::max(b->smem[k], ewald_smem(b->sys[idx], threads));
    MS2_CUDA_OK(ms2_allow_smem((const void *)fn, b->smem[k]));
    int per_sm = 0, sms = 0, dev = 0, coop = 0;
    MS2_CUDA_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, b->smem[k]));
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (per_sm < 1 || !coop)
        return ms2_fail(MS2_EINVAL, "batch kind %s: %d threads with %zu B of shared memory do not fit one SM",
                        kKindName[kind], threads, b->smem[k]);
    const int G = per_sm * sms;
    b->grid[k] = G;
    double total = 0;
    std::vector<double> cost;
    for (size_t e = 0; e < b->order[k].size(); ++e) {
        const int idx = b->order[k][e];
        cost.push_back(item_cost(b->sys[idx], b->htab[k][e].lcap > 0));
        total += cost.back() * b->sys[idx]->N;
    }
    // vb virtual blocks of equal estimated cost per block of the grid, drawn
    // dynamically by the blocks (the estimate need not be exact)
    const int GV = vb * G;
    b->vbpb[k] = vb;
    b->nvb[k] = GV;
    std::vector<int4> seg;
    std::vector<int> off(GV + 1, 0);
    double acc = 0;
    int blk = 0;
    for (size_t e = 0; e < b->order[k].size(); ++e) {
        const int N = b->sys[b->order[k][e]]->N;
        int first = 0;
        for (int i = 0; i < N; ++i) {
            const double mid = acc + (i + 0.5) * cost[e];
            const int bi = std::min(GV - 1, (int)(mid * GV / total));
            if (bi != blk) {
                if (i > first) seg.push_back(make_int4((int)e, first, i, 0));
                for (int q = blk + 1; q <= bi; ++q) off[q] = (int)seg.size();
                blk = bi;
                first = i;
            }
        }
        if (N > first) seg.push_back(make_int4((int)e, first, N, 0));
        acc += cost[e] * N;
    }
    for (int q = blk + 1; q <= GV; ++q) off[q] = (int)seg.size();
    MS2_CUDA_OK(b->al.alloc((void **)&b->dseg[k], sizeof(int4) * std::max<size_t>(seg.size(), 1)));
    MS2_CUDA_OK(b->al.alloc((void **)&b->dsegoff[k], sizeof(int) * (GV + 1)));
    MS2_CUDA_OK(cudaMemcpyAsync(b->dseg[k], seg.data(), sizeof(int4) * seg.size(), cudaMemcpyHostToDevice, b->stream));
    MS2_CUDA_OK(cudaMemcpyAsync(b->dsegoff[k], off.data(), sizeof(int) * (GV + 1), cudaMemcpyHostToDevice, b->stream));
    MS2_CUDA_OK(cudaStreamSynchronize(b->stream));  // the host vectors go out of scope
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

// Autotuner: per group (model kind and size class), the decomposition that runs
// this batch fastest over a list build and two steps on the lists: the block
// shape (256 threads, two blocks per SM where they fit; 512 threads, one block
// per SM; 1024 threads with 64 registers where the kind has that kernel) times
// the size of the pair-phase pieces (1, 4 or 16 pieces per block of the grid:
// larger pieces stage fewer systems, smaller ones balance better); results
// cached on disk by (kind, size class, size bucket, count bucket).  The shape
// changes only the work split, never a system's results.
static ms2_status tune(ms2_batch b) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::map<std::string, int> cache = load_tune();
    std::string key[G_COUNT];
    bool need = false;
    for (int k = 0; k < G_COUNT; ++k) {
        if (b->order[k].empty()) continue;
        std::vector<int> ns;
        for (int idx : b->order[k]) ns.push_back(b->sys[idx]->N);
        std::sort(ns.begin(), ns.end());
        int med = ns[ns.size() / 2], bucket = 1;
        while (bucket < med) bucket <<= 1;
        int cnt = 1;
        while (cnt < (int)ns.size()) cnt <<= 1;
        std::ostringstream os;
        os << "v5/" << kKindName[kind_of_group(k)] << "/C" << (k & 1) << "/N" << bucket << "/S" << cnt;
        key[k] = os.str();
        auto it = cache.find(key[k]);  // shape code: threads x 64 + pieces per block
        if (it != cache.end() && set_shape(b, k, it->second / 64, it->second % 64) == MS2_OK) continue;
        need = true;
    }
    if (!need || !b->tune_shapes) return MS2_OK;  // (untuned kinds keep the default shape)
    std::vector<void *> saved;
    ms2_status st = snapshot_state(b, saved, true);
    if (st != MS2_OK) return st;
    cudaEvent_t e0, e1;
    MS2_CUDA_OK(cudaEventCreate(&e0));
    MS2_CUDA_OK(cudaEventCreate(&e1));
    for (int k = 0; k < G_COUNT; ++k) {
        if (b->order[k].empty() || cache.count(key[k])) continue;
        float best = 1e30f;
        int best_t = MS_THREADS, best_vb = VB_PER_BLOCK;
        for (int trial = 0; trial < 9; ++trial) {
            const int t = (trial / 3 == 0) ? 256 : (trial / 3 == 1 ? MS_THREADS : 2 * MS_THREADS);
            const int vb = trial % 3 == 0 ? 1 : (trial % 3 == 1 ? 4 : 16);
            if (!kernel_of(kind_of_group(k), t) || set_shape(b, k, t, vb) != MS2_OK) continue;
            // only group k runs in a trial
            std::vector<int> keep[G_COUNT];
            for (int j = 0; j < G_COUNT; ++j)
                if (j != k) std::swap(keep[j], b->order[j]);
            // an untimed launch first (module loading, cold caches), then the state back
            st = batch_launch(b, 1, true);
            if (st == MS2_OK) st = snapshot_state(b, saved, false);
            if (st == MS2_OK) {  // a list build and two steps on the lists
                MS2_CUDA_OK(cudaEventRecord(e0, b->stream));
                st = batch_launch(b, 3, true);
                MS2_CUDA_OK(cudaEventRecord(e1, b->stream));
            }
            for (int j = 0; j < G_COUNT; ++j)
                if (j != k) std::swap(keep[j], b->order[j]);
            if (st != MS2_OK) return st;
            MS2_CUDA_OK(cudaEventSynchronize(e1));
            float ms = 0;
            MS2_CUDA_OK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                best_t = t;
                best_vb = vb;
            }
            st = snapshot_state(b, saved, false);
            if (st != MS2_OK) return st;
        }
        MS2_CUDA_OK(cudaStreamSynchronize(b->stream));
        st = set_shape(b, k, best_t, best_vb);
        if (st != MS2_OK) return st;
        store_tune(key[k], best_t * 64 + best_vb);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    MS2_CUDA_OK(cudaStreamSynchronize(b->stream));
    return MS2_OK;
}

// dynamic shared memory a block of kind k's kernel can have at most on this
// device: the opt-in per-block limit less the kernel's static shared memory
static size_t batch_smem_limit(int kind, int threads) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, (const void *)kernel_of(kind, threads)) != cudaSuccess) return 0;
    return optin > (int)fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
}

// whether the batch kernels take this system (used by the server)
bool ms2_batch_accepts(ms2_system s) {
    if (!s || s->hp.integrator != MS2_INT_LEAPFROG_Q || s->fp64 || s->hp.massieu || s->d.gk || s->res_every > 0 ||
        s->hf_every > 0)
        return false;
    const int kind = kind_of(s);
    if (kind < 0) return false;
    const int rdf = s->d.rdf ? s->d.rdf_rows * s->d.rdf_bins : 0;
    if (rdf > RDF_SMEM_MAX) return false;
    return std::max(batch_smem(kind, (s->N + 3) & ~3, 256, rdf), ewald_smem(s, 256)) <= batch_smem_limit(kind, 256);
}

// Batch creation with options (the server's batches): tune = false takes the
// cached block shape or the default without trial launches; fa/ff/ctx, if set,
// allocate the batch's device memory (a server's block cache, so that the
// batches it rebuilds as jobs come and go do not call cudaMalloc/cudaFree).
ms2_status ms2_batch_create_opt(const ms2_system *systems, int n, ms2_batch *out, bool tune_shapes,
                                void *(*fa)(size_t, void *), void (*ff)(void *, void *), void *ctx) {
    if (!out || !systems || n < 1) return ms2_fail(MS2_EINVAL, "need n >= 1 systems and an output handle");
    *out = nullptr;
    ms2_batch b = new ms2_batch_s();
    b->al.fa = fa;
    b->al.ff = ff;
    b->al.ctx = ctx;
    b->tune_shapes = tune_shapes;
    // the batch owns its stream: it must outlive none of the systems' streams
    for (int k = 0; k < n; ++k) {
        ms2_system s = systems[k];
        if (!s) { delete b; return ms2_fail(MS2_EINVAL, "system %d is null", k); }
        if (s->hp.integrator != MS2_INT_LEAPFROG_Q || s->fp64 || s->hp.massieu || s->d.gk || s->res_every > 0 ||
            s->hf_every > 0) {
            delete b;
            return ms2_fail(MS2_EINVAL, "system %d: batches take leapfrog systems with FP32 pair arithmetic, "
                                        "without Massieu, conductivity, residence or heat-flux sampling", k);
        }
        const int kind = kind_of(s);
        if (kind < 0) {
            delete b;
            return ms2_fail(MS2_EINVAL, "system %d: more than 4 site slots, or an Ewald system other than "
                                        "3-site water with single-site ions", k);
        }
        const int rdf = s->d.rdf ? s->d.rdf_rows * s->d.rdf_bins : 0;
        if (rdf > RDF_SMEM_MAX) { delete b; return ms2_fail(MS2_EINVAL, "system %d: RDF histogram too large for a batch", k); }
        if (std::max(batch_smem(kind, (s->N + 3) & ~3, 256, rdf), ewald_smem(s, 256)) > batch_smem_limit(kind, 256)) {
            delete b;
            return ms2_fail(MS2_EINVAL, "system %d: %d molecules do not fit one block's shared memory", k, s->N);
        }
        b->sys.push_back(s);
        b->order[group_of(kind, s->N)].push_back(k);
    }
    ms2_status st = MS2_OK;
    auto fail = [&](ms2_status s2) { ms2_batch_destroy(b); return s2; };
    {
        cudaError_t e0 = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e0 != cudaSuccess) return fail(ms2_fail_cuda(e0, "batch stream", __FILE__, __LINE__));
    }
    cudaError_t ce = b->al.alloc((void **)&b->dbar, sizeof(unsigned) * 3 * G_COUNT);
    for (int k = 0; k < G_COUNT && ce == cudaSuccess; ++k) {
        if (b->order[k].empty()) continue;
        std::vector<int2> drift, unit, ew_sk, ew_sum, ew_force;
        ce = b->al.alloc((void **)&b->dnflag[k], sizeof(int) * b->order[k].size());
        // candidate lists of the kind's systems in one allocation (a server re-creates
        // batches as jobs come and go): skin kSkin r_c; only where the expected list
        // (1.3 x the ideal-gas count within r_c + skin) is shorter than 3N/4
        std::vector<int> lcaps(b->order[k].size(), 0);
        std::vector<size_t> nl_off(b->order[k].size(), 0);
        size_t nl_bytes = 0;
        for (size_t e = 0; e < b->order[k].size(); ++e) {
            ms2_system s = b->sys[b->order[k][e]];
            const int N = s->N;
            const double L = s->hp.L, rc = s->rc, skin = kSkin * rc;
            const double frac = std::min(1.0, 4.18879020478639098 * std::pow(rc + skin, 3.0) / (L * L * L));  // 4 pi / 3
            const int lexp = (int)std::ceil(1.3 * frac * N + 32.0);  // the expected list, with a margin
            // capacity MS2_LIST_CAP x the ideal-gas count (dilute systems condense into
            // droplets over long runs: a molecule there has 2-3 x the average
            // neighbours; an owner whose list overflows scans in full)
            const int lcap = std::min(((N + 31) & ~31), ((int)std::ceil(MS2_LIST_CAP * frac * N + 64.0) + 31) & ~31);
            if (N <= 65535 && lexp < (3 * N) / 4) {
                lcaps[e] = lcap;
                nl_off[e] = nl_bytes;
                nl_bytes += al16(sizeof(uint16_t) * (size_t)N * lcap) + al16(sizeof(int) * N) + al16(sizeof(uint32_t) * 3 * N);
            }
        }
        unsigned char *nl_base = nullptr;
        if (ce == cudaSuccess && nl_bytes) ce = b->al.alloc((void **)&nl_base, nl_bytes);
        for (size_t e = 0; e < b->order[k].size() && ce == cudaSuccess; ++e) {
            ms2_system s = b->sys[b->order[k][e]];
            const int N = s->N;
            BatchEntry en;
            memset(&en, 0, sizeof en);
            en.P = s->dP;
            en.S = s->d;
            en.S.jsplit = 1;
            en.units = (N + UNIT - 1) / UNIT;
            en.S.nunits = en.units;
            ce = b->al.alloc((void **)&en.S.blk, sizeof(double) * MS2_NRED * en.units);
            if (ce == cudaSuccess && lcaps[e]) {
                const int lcap = lcaps[e];
                const double rc = s->rc, skin = kSkin * rc, sc = s->hp.lat_scale;
                unsigned char *q = nl_base + nl_off[e];
                en.nl = (uint16_t *)q;
                q += al16(sizeof(uint16_t) * (size_t)N * lcap);
                en.ncnt = (int *)q;
                q += al16(sizeof(int) * N);
                en.Xb = (uint32_t *)q;
                const double rl = (rc + skin) * sc + 2.0, hl = std::max(0.0, 0.5 * skin * sc - 2.0);
                en.rs2 = (unsigned long long)std::ceil(rl * rl);
                en.sk2 = (unsigned long long)std::floor(hl * hl);
                en.lcap = lcap;
            }
            en.nflag = b->dnflag[k] + e;
            en.step0 = s->step;
            if (s->hp.elec == ELEC_EWALD) {
                en.AS = s->AS;
                en.nsb = ewald::n_site_tasks(s->d.nsite_q, s->d.sk_sites);
                en.nkc = ewald::n_sum_tasks(ewald::n_k(s->d.kx, s->d.ky, s->d.kz));
                for (int t = 0; t < en.nsb; ++t) ew_sk.push_back(make_int2((int)e, t));
                for (int t = 0; t < en.nkc; ++t) ew_sum.push_back(make_int2((int)e, t));
                for (int t = 0; t < s->d.kchunks; ++t) ew_force.push_back(make_int2((int)e, t));
            }
            b->htab[k].push_back(en);
            for (int m = 0; m < N; m += 8) drift.push_back(make_int2((int)e, m));
            for (int u = 0; u < en.units; ++u) unit.push_back(make_int2((int)e, u));
            b->Np[k] = std::max(b->Np[k], (N + 3) & ~3);
            b->rdf_cells[k] = std::max(b->rdf_cells[k], s->d.rdf ? s->d.rdf_rows * s->d.rdf_bins : 0);
        }
        if (ce == cudaSuccess) ce = b->al.alloc((void **)&b->dtab[k], sizeof(BatchEntry) * b->htab[k].size());
        if (ce == cudaSuccess) ce = b->al.alloc((void **)&b->ddrift[k], sizeof(int2) * drift.size());
        if (ce == cudaSuccess) ce = b->al.alloc((void **)&b->dunit[k], sizeof(int2) * unit.size());
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(b->ddrift[k], drift.data(), sizeof(int2) * drift.size(), cudaMemcpyHostToDevice, b->stream);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(b->dunit[k], unit.data(), sizeof(int2) * unit.size(), cudaMemcpyHostToDevice, b->stream);
        const std::vector<int2> *ew[3] = {&ew_sk, &ew_sum, &ew_force};
        int2 **dew[3] = {&b->dew_sk[k], &b->dew_sum[k], &b->dew_force[k]};
        for (int q = 0; q < 3 && ce == cudaSuccess; ++q)
            if (!ew[q]->empty()) {
                ce = b->al.alloc((void **)dew[q], sizeof(int2) * ew[q]->size());
                if (ce == cudaSuccess)
                    ce = cudaMemcpyAsync(*dew[q], ew[q]->data(), sizeof(int2) * ew[q]->size(), cudaMemcpyHostToDevice,
                                         b->stream);
            }
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);  // the host vectors go out of scope
        b->n_drift[k] = (int)drift.size();
        b->n_unit[k] = (int)unit.size();
        b->n_ew_sk[k] = (int)ew_sk.size();
        b->n_ew_sum[k] = (int)ew_sum.size();
        b->n_ew_force[k] = (int)ew_force.size();
    }
    if (ce != cudaSuccess) return fail(ms2_fail_cuda(ce, "batch set-up", __FILE__, __LINE__));
    for (int k = 0; k < G_COUNT; ++k)
        if (!b->order[k].empty() && set_shape(b, k, MS_THREADS) != MS2_OK && (st = set_shape(b, k, 256)) != MS2_OK)
            return fail(st);
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

extern "C" ms2_status ms2_batch_create(const ms2_system *systems, int n, ms2_batch *out) {
    return ms2_batch_create_opt(systems, n, out, true, nullptr, nullptr, nullptr);
}

extern "C" ms2_status ms2_batch_step(ms2_batch b, long long n) {
    if (!b) return ms2_fail(MS2_EINVAL, "null batch");
    if (n < 0) return ms2_fail(MS2_EINVAL, "negative step count");
    for (ms2_system s : b->sys)  // forces of a state set since the last step
        if (ms2_status e = ms2_ensure_forces(s)) return e;
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
    b->al.release_all();
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return MS2_OK;
}
