// Fused MD step of one system: a cooperative persistent kernel, one block of
// 512 threads per SM, runs a whole chunk of leapfrog steps (paper, Sec. "Hybrid
// MPI & OpenMP Parallelization": the partner search, energy and force loops over
// molecules; the rigid-body leapfrog with isokinetic scaling and the thermo
// reduction as in k_integrate.cu).
//
// Block b owns the molecules [N b / G, N (b+1) / G) for the whole launch; their
// FP64 state (R, v, q, L, F, tau) stays in its shared memory and goes back to
// global memory at the end.  Per step:
//
//   stage the whole system's lattice coordinates and site offsets in shared
//   memory; pair items (own molecule i, j-range p), one per warp; every
//   'rdf_every' steps the RDF; the partials stay in shared memory
//   reduction unit b (the own molecules, one warp): F, tau, energies, kinetic
//   energies; its totals to global memory
//   -- grid barrier --
//   every block sums the G units in fixed order and derives the thermostat
//   factor itself; drift and site build of the own molecules; their lattice
//   coordinates and offsets to global memory (block 0 records the step during
//   the next pair phase, on a warp without a pair item)
//   -- grid barrier --
//
// The phases are the device functions of the per-phase kernels (drift_quad,
// PairWarp, reduce_unit, reduce_totals, finish_step_warp) and the per-phase path of a
// fusable system uses the same decomposition (j-ranges, tile segmentation,
// reduction units = the G block ranges), so a chunk run here is bitwise
// identical to the same chunk run as separate kernels.  What the fusion saves
// is the kernel boundaries (a launch costs ~5 us event to event, a bounded grid
// barrier ~1.2 us on GB300), the state round trips through L2 and the last-block
// tail of the reduction.
//
// Every grid-barrier wait is bounded (2 s of %globaltimer).  A block that gives
// up sets a sticky flag that ends every other wait at once and marks the system
// (SC_KERR); the kernel then runs to its end without waiting and the host
// reports MS2_ETIMEOUT at its next read.
#include <algorithm>

#include "ms2_internal.cuh"

#include "ewald_dev.cuh"
#include "grid_dev.cuh"
#include "integrate_dev.cuh"
#include "pair_engine.cuh"

using namespace pair_engine;
using namespace integ;
using grid_dev::global_ns;

namespace {

constexpr int STEP_THREADS = 512;
constexpr int STEP_WARPS = STEP_THREADS / 32;
// the quantity of block 0's record totals that warp w forms (-1: none), up to
// Q_N + 3 of them: warps 6-15, those that share no scheduler (warp % 4) with
// warp 1 first (a switch: no table in memory, which a step after an L2 flush
// would read from DRAM)
__device__ __forceinline__ int tot_quantity(int w) {
    switch (w) {
        case 6: return 0;
        case 7: return 1;
        case 8: return 2;
        case 10: return 3;
        case 11: return 4;
        case 12: return 5;
        case 14: return 6;
        case 15: return 7;
        case 9: return 8;
        case 13: return 9;
        default: return -1;
    }
}
// site-site RDF of the staged configuration (the k_rdf arithmetic, reading
// the shared-memory tile): molecules i = block, block + grid, ...; threads over j > i
template <int NS, bool MULTI>
__device__ void rdf_tile(const SysParams *__restrict__ P, const DevSys &S, const Smem &sm, int TJ, unsigned *hist) {
    const int N = S.N, cells = S.rdf_rows * S.rdf_bins;
    for (int k = threadIdx.x; k < cells; k += blockDim.x) hist[k] = 0u;
    __syncthreads();
    for (int i = blockIdx.x; i < N; i += gridDim.x)
        rdf_molecule<NS, MULTI>(P, S, sm, TJ, i, i + 1 + threadIdx.x, blockDim.x, N, hist);
    __syncthreads();
    for (int k = threadIdx.x; k < cells; k += blockDim.x)
        if (hist[k]) atomicAdd(&S.rdf[k], (unsigned long long)hist[k]);
}

// step k of the launch samples the electric current flux
__device__ __forceinline__ bool gk_step(const StepArgs &A, int k) {
    return A.gk_every > 0 && ((A.s0 + k + 1) % A.gk_every) == 0;
}

// step k of the launch samples the heat flux
__device__ __forceinline__ bool hf_step(const StepArgs &A, int k) {
    return A.hf_every > 0 && ((A.s0 + k + 1) % A.hf_every) == 0;
}

}  // namespace

static_assert(sizeof(SysParams) % 16 == 0, "the parameter copy moves 16-byte words");

// per-block region after the staged system: parameters, own state and partials
struct OwnLayout {
    size_t params, state, ui, np, sp, part, hpart, ews, hist;  // byte offsets from the region start
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// (ews: bytes of the reciprocal-space task scratch, Ewald systems; the RDF
// histogram follows)
__host__ __device__ inline OwnLayout own_layout(int mcap, int js, size_t ews) {
    OwnLayout o;
    o.params = 0;                                                     // a copy of the system parameters
    o.state = al16(o.params + sizeof(SysParams));                     // 19 doubles per slot
    o.ui = al16(o.state + sizeof(double) * 19 * (size_t)mcap);        // 4 doubles per slot
    o.np = al16(o.ui + sizeof(double) * 4 * (size_t)mcap);            // 1 int per slot
    o.sp = al16(o.np + sizeof(int) * (size_t)mcap);                   // species, 1 int per slot
    o.part = al16(o.sp + sizeof(int) * (size_t)mcap);                 // [js][NPV][mcap] floats
    o.hpart = al16(o.part + sizeof(float) * MS2_NPV * (size_t)js * mcap);  // [js][3][mcap] heat partials
    o.ews = al16(o.hpart + sizeof(float) * 3 * (size_t)js * mcap);
    o.hist = al16(o.ews + ews);
    return o;
}

// HEAT: the variant that also runs the heat-flux power pass and heat unit of
// k_heat / k_heat_reduce on the sampled steps (after the totals, before the next
// drift); their record (block 0) follows at the next step's pair phase, or after
// one more grid barrier at the end of the launch.
template <int NS, unsigned LJM, unsigned QM, unsigned DM, int ELEC, bool MULTI, bool MASS = false, bool HEAT = false>
__global__ void __launch_bounds__(STEP_THREADS, 1) k_step(const SysParams *__restrict__ P, DevSys S, StepArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Eng = PairWarp<NS, LJM, QM, DM, ELEC, MULTI, MASS>;
    constexpr int EWM = ELEC == ELEC_EWALD ? RED_EWALD : 0;  // reduction mode bit of the reciprocal space
    __shared__ double tot[MS2_NRED];
    __shared__ double lam_s;                    // thermostat factor for the next drift
    __shared__ double kin_s[6 * 32];            // kinetic terms of the reduction unit (kin_pre)
    __shared__ double od_s[4 * 32];             // site offsets of the split site build (build_site)
    __shared__ unsigned long long tph[6];       // timing: entry, then the phase marks of the last step
    const int N = S.N, G = gridDim.x, b = blockIdx.x, JS = S.jsplit, MC = A.mcap;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lo = (int)((long long)N * b / G), hi = (int)((long long)N * (b + 1) / G), nm = hi - lo;
    if (A.timing && b == 0 && threadIdx.x == 0) tph[5] = global_ns();  // kernel entry
    Smem sm = carve<NS, Eng::TILE, MULTI>(smem_raw, A.Np, STEP_WARPS);
    unsigned char *own = smem_raw + al16(smem_bytes(NS, Eng::TILE, MULTI, A.Np, STEP_WARPS));
    // the own region's arrays, rebuilt where needed (short live ranges: the
    // pair loop keeps its registers)
    auto view = [&]() {
        const OwnLayout l = own_layout(MC, JS, (size_t)A.ews);
        double *st = (double *)(own + l.state);
        return StateView{st, st + 3 * MC, st + 6 * MC, st + 10 * MC, st + 13 * MC, st + 16 * MC,
                         (const int *)(own + l.sp), MC};
    };
    // the system parameters, copied into shared memory once: the per-step phases
    // then read no parameter through L2 after a grid barrier
    const SysParams *Ps = (const SysParams *)(own + own_layout(MC, JS, (size_t)A.ews).params);
    auto part_at = [&]() { return (float *)(own + own_layout(MC, JS, (size_t)A.ews).part); };
    auto hpart_at = [&]() { return (float *)(own + own_layout(MC, JS, (size_t)A.ews).hpart); };
    int *wq = sm.queue + warp * QSTRIDE;
    // prologue: every load is issued before anything waits on one (after an L2
    // flush each dependent round trip goes to DRAM): the thermostat factor, the
    // parameter copy and the own state; the tables then come from the copy
    double lam0 = 0.0;
    if (threadIdx.x == 0) lam0 = __ldcg(S.scal + SC_LAMBDA);
    // block 0 records the steps: its running sums and the launch constants stay
    // in shared memory for the launch (written back at the end)
    __shared__ double acc_s[AC_COUNT_];
    __shared__ StepConsts kc_s;
    if (b == 0) {
        if (threadIdx.x < AC_COUNT_) acc_s[threadIdx.x] = __ldcg(S.acc + threadIdx.x);
        if (threadIdx.x == 32) kc_s = global_consts(S);
    }
    {
        const int4 *src = (const int4 *)P;
        int4 *dst = (int4 *)(own + own_layout(MC, JS, (size_t)A.ews).params);
        for (int k = threadIdx.x; k < (int)(sizeof(SysParams) / sizeof(int4)); k += blockDim.x) dst[k] = src[k];
    }
    // own state into shared memory
    for (int t = threadIdx.x; t < nm; t += blockDim.x) {
        const StateView sv = view();
        const int i = lo + t;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sv.R[c * MC + t] = __ldcg(S.R + c * N + i);
            sv.v[c * MC + t] = __ldcg(S.v + c * N + i);
            sv.L[c * MC + t] = __ldcg(S.Lm + c * N + i);
            sv.F[c * MC + t] = __ldcg(S.F + c * N + i);
            sv.tau[c * MC + t] = __ldcg(S.tau + c * N + i);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) sv.q[c * MC + t] = __ldcg(S.q + c * N + i);
        ((int *)sv.spc)[t] = S.species[i];
    }
    __syncthreads();
    load_tables<MULTI>(Ps, sm);
    Eng e;
    e.setup(Ps);
    if (b == 0 && threadIdx.x == 0) *A.bar_next = 0u;
    unsigned target = A.bar_extra;
    auto on_timeout = [&]() { S.scal[SC_KERR] = 1.0; };
    using grid_dev::grid_sync;
    const bool rfq = Eng::MOLD && e.rfq;
    const bool rec = A.timing && b == 0 && threadIdx.x == 0;
    // timing of the last step: every block marks the end of its compute phases
    auto mark = [&](int k, int slot) {
        if (A.timing && k == A.nsteps - 1) {  // uniform over the grid
            __syncthreads();
            if (threadIdx.x == 0) atomicMax(A.tmax + slot, global_ns());
        }
    };
    if (threadIdx.x == 0) lam_s = lam0;
    __syncthreads();
    // the thermostat factor of the next drift, per thread: the drift warps form
    // it themselves after each step's reduction (no block barrier on it)
    double lam_r = lam_s;
    // one reduction pass (1 to 8 molecules) and a warp left without a pair item
    const bool kin_early = nm >= 1 && nm <= 8 && nm * JS <= STEP_WARPS - 2;
    // one drift pass (1 to 8 molecules, warp 1) and 2 to 4 site slots: the site
    // build runs a warp per site
    const bool site_split = NS >= 2 && NS <= 4 && nm >= 1 && nm <= 8;
    // k = -1 (after ms2_set_state): the state as set is evaluated first -- site
    // build instead of the drift, then partner search, forces, unit reduction,
    // totals and the configuration's scalars (ms2_eval_forces' k_build, k_pair
    // and k_reduce on the same decomposition), no record and no sampling
    for (int k = A.init ? -1 : 0; k < A.nsteps; ++k) {
        const bool ev = k < 0;
        const bool tm = rec && k == A.nsteps - 1;
        if (tm) tph[0] = global_ns();
        // ---- drift + site build of the own molecules (k = -1: the site build alone, as k_build)
        if (warp >= 1)
            for (int m0 = 8 * (warp - 1); m0 < nm; m0 += 8 * (STEP_WARPS - 1)) {
                const int m = m0 + (lane >> 2), c = lane & 3;
                if (!ev) {
                    if (site_split)
                        drift_quad<true, false>(Ps, S, view(), m, lo + m, m < nm, c, false, lam_r);
                    else
                        drift_quad<true>(Ps, S, view(), m, lo + m, m < nm, c, false, lam_r);
                } else if (m < nm && c < 3) {
                    const StateView sv = view();
                    const double q[4] = {sv.q[m], sv.q[MC + m], sv.q[2 * MC + m], sv.q[3 * MC + m]};
                    build_row(Ps, S, lo + m, c, q, sv.R[c * MC + m], sv.spc[m]);
                }
            }
        if (!ev && site_split) {
            // the site build of the drifted molecules split by site: warp 1 + a
            // builds site a's rows (and warp 1 the lattice centres), each FP64
            // chain on a scheduler of its own; then warp 1 sums the molecular
            // dipole from their offsets in site order (build_row's arithmetic)
            __syncthreads();
            const int m = lane >> 2, c = lane & 3;
            if (warp >= 1 && warp <= NS && m < nm && c < 3) {
                const StateView sv = view();
                const double q[4] = {sv.q[m], sv.q[MC + m], sv.q[2 * MC + m], sv.q[3 * MC + m]};
                const int a = warp - 1;
                if (a == 0) S.X[c * N + lo + m] = lattice_coord(sv.R[c * MC + m], Ps->lat_scale);
                od_s[a * 32 + lane] = build_site(Ps, S, lo + m, c, q, sv.spc[m], a);
            }
            __syncthreads();
            if (warp == 1 && m < nm && c < 3) build_md(Ps, S, lo + m, c, view().spc[m], od_s + lane, 32);
        }
        mark(k, 0);
        grid_sync(A.bar, A.err, target, on_timeout, A.wait_ns);
        if (tm) tph[1] = global_ns();
        // ---- stage the whole system; pair items of the own molecules; RDF
        stage_tile<NS, DM, Eng::MOLD, MULTI>(sm, S, 0, N, A.Np, rfq);
        __syncthreads();
        // the previous step's record (U, W, T, P, averages, a conductivity
        // sample), off the critical path: block 0's last warp, which has no pair
        // item unless 16 are due
        if (k > 0 && b == 0 && warp == STEP_WARPS - 1) {
            const int gk = gk_step(A, k - 1) ? RED_GK : 0;
            finish_step_warp(Ps, S, RED_SUM | RED_RECORD | RED_LAMBDA | EWM | gk, tot, lane, acc_s, kc_s);
            if (gk) gk_update(S, tot, lane);
            if (HEAT && hf_step(A, k - 1)) heat_record(S, G, lane);
        }
        // the kinetic terms of the reduction unit need no forces: a warp without
        // a pair item (nor block 0's record) forms them beside the pair phase
        if (kin_early && warp == STEP_WARPS - 2) {
            const OwnLayout ol = own_layout(MC, JS, (size_t)A.ews);
            const RedIO io{part_at(), nullptr, MC, view(), (double *)(own + ol.ui), (int *)(own + ol.np), MC, lo};
            kin_pre<true>(Ps, S, io, b, G, lane, kin_s);
        }
        for (int t = warp; t < nm * JS; t += STEP_WARPS) {
            const int m = t % nm, p = t / nm, i = lo + m;
            const int j0 = (int)(((long long)N * p) / JS), j1 = (int)(((long long)N * (p + 1)) / JS);
            e.begin_tile(Ps, sm, A.Np, i);
            for (int t0 = j0; t0 < j1; t0 += A.TJ) e.scan(shifted(sm, t0), A.Np, t0, min(A.TJ, j1 - t0), wq, lane);
            const PairOut o = e.finish(lane);
            if (lane == 0) {
                float *q = part_at() + (size_t)p * MS2_NPV * MC + m;
                q[PV_FX * MC] = o.F[0]; q[PV_FY * MC] = o.F[1]; q[PV_FZ * MC] = o.F[2];
                q[PV_TX * MC] = o.T[0]; q[PV_TY * MC] = o.T[1]; q[PV_TZ * MC] = o.T[2];
                q[PV_ULJ * MC] = o.ulj; q[PV_UQQ * MC] = o.uqq; q[PV_UDD * MC] = o.udd; q[PV_W * MC] = o.w;
                q[PV_NP * MC] = (float)o.np;
                q[PV_VV * MC] = o.vv;
            }
        }
        if (!ev && A.rdf_every > 0 && ((A.s0 + k + 1) % A.rdf_every) == 0) {
            __syncthreads();
            rdf_tile<NS, MULTI>(Ps, S, sm, A.Np, (unsigned *)(own + own_layout(MC, JS, (size_t)A.ews).hist));
        }
        __syncthreads();
        mark(k, 1);
        if (tm) {
            tph[2] = global_ns();
            S.scal[SC_TPAIR] = (double)(tph[2] - tph[1]);
        }
        // ---- Ewald reciprocal space: the tasks of the per-phase kernels, spread
        // over the blocks (structure-factor tasks, sum tasks, force tasks), a grid
        // barrier after each kind; the reduction then sums the force chunks
        if constexpr (ELEC == ELEC_EWALD) {
            unsigned char *ews = own + own_layout(MC, JS, (size_t)A.ews).ews;
            const int M = S.nsite_q, nsb = ewald::n_site_tasks(M, S.sk_sites);
            const int nkc = ewald::n_sum_tasks(ewald::n_k(S.kx, S.ky, S.kz));
            unsigned long long te = tm ? global_ns() : 0ull;  // timing (block 0): each phase until its barrier ends
            for (int sb = b; sb < nsb; sb += G) ewald::sk_task(Ps, S, sb, ews, threadIdx.x, STEP_THREADS);
            grid_sync(A.bar, A.err, target, on_timeout, A.wait_ns);
            if (tm) { const unsigned long long t = global_ns(); S.scal[SC_TPH9] = (double)(t - te); te = t; }
            for (int kc = b; kc < nkc; kc += G) ewald::sum_task(S, A.AS, kc, nsb, ews, threadIdx.x, STEP_THREADS);
            grid_sync(A.bar, A.err, target, on_timeout, A.wait_ns);
            if (tm) { const unsigned long long t = global_ns(); S.scal[SC_TPH10] = (double)(t - te); te = t; }
            const int ng = (M + STEP_THREADS - 1) / STEP_THREADS, nft = ng * S.kchunks;
            // U_rec and W_rec: the last block, which has no force task when there are fewer than G
            if (b == G - 1 && warp == 0) ewald::sum_finish(Ps, S, nkc, lane);
            for (int t = b; t < nft; t += G) {
                if (S.kx == 8)
                    ewald::force_task<9>(Ps, S, A.AS, (t % ng) * STEP_THREADS, t / ng, A.ny_per_chunk, ews, threadIdx.x,
                                         STEP_THREADS);
                else
                    ewald::force_task<0>(Ps, S, A.AS, (t % ng) * STEP_THREADS, t / ng, A.ny_per_chunk, ews, threadIdx.x,
                                         STEP_THREADS);
            }
            grid_sync(A.bar, A.err, target, on_timeout, A.wait_ns);
            if (tm) S.scal[SC_TPH11] = (double)(global_ns() - te);
        }
        // ---- reduction unit b: the own molecules
        if (warp == 0) {
            const OwnLayout ol = own_layout(MC, JS, (size_t)A.ews);
            const RedIO io{part_at(), nullptr, MC, view(), (double *)(own + ol.ui), (int *)(own + ol.np), MC, lo};
            reduce_unit<true>(Ps, S, io, RED_SUM | RED_LAMBDA | EWM | (!ev && gk_step(A, k) ? RED_GK : 0), b, G, lane,
                              kin_early ? kin_s : nullptr);
        }
        mark(k, 2);
        grid_sync(A.bar, A.err, target, on_timeout, A.wait_ns);
        if (tm) tph[3] = global_ns();
        // ---- totals.  The warps that drift the block's molecules form the
        // kinetic energy after the kick and from it the thermostat factor of
        // their next drift (the same fixed-order sum in each); block 0 forms
        // every step scalar for its record on warps 6-15, which the drift
        // leaves idle (its molecules take warps 1-4 at most), beside the next
        // drift.  The next grid barrier orders them before the record reads them.
        {
            const int nq = !ev && gk_step(A, k) ? Q_N + 3 : Q_N;
            // (none after the launch's last step: the next launch takes the factor
            // from block 0's record)
            if (k < A.nsteps - 1 && warp >= 1 && 8 * (warp - 1) < nm) lam_r = lambda_k1(Ps, unit_total(S, G, Q_K1, lane));
            // quantity q on warp tot_quantity^-1(q): warps 6-15, those that
            // share no scheduler (warp % 4) with warp 1, which drifts up to 8
            // molecules, first (the FP64 unit is per scheduler)
            if (b == 0) {
                const int q = tot_quantity(warp);
                if (q >= 0 && q < nq) {
                    const double x = unit_total(S, G, q, lane);
                    if (lane == 0) tot[q] = x;
                }
            }
            if (ev && b == 0) {  // the scalars of the state as set, at once
                __syncthreads();
                if (warp == 0) finish_step_warp(Ps, S, RED_SUM | RED_LAMBDA | EWM, tot, lane, acc_s, kc_s);
            }
        }
        // ---- heat flux of this configuration (sampled steps): power pass over
        // the staged system, then heat unit b
        if constexpr (HEAT) {
            if (!ev && hf_step(A, k)) {
                for (int t = warp; t < nm * JS; t += STEP_WARPS) {
                    const int m = t % nm, p = t / nm, i = lo + m;
                    const int j0 = (int)(((long long)N * p) / JS), j1 = (int)(((long long)N * (p + 1)) / JS);
                    e.begin_tile(Ps, sm, A.Np, i);
                    float hv[3], hw[3];
                    heat_velocities<true>(Ps, view(), m, hv, hw);
                    e.begin_heat(hv, hw);
                    for (int t0 = j0; t0 < j1; t0 += A.TJ)
                        e.template scan<true>(shifted(sm, t0), A.Np, t0, min(A.TJ, j1 - t0), wq, lane);
                    float jh[3];
                    e.finish_heat(jh);
                    if (lane == 0)
#pragma unroll
                        for (int c = 0; c < 3; ++c) hpart_at()[((size_t)p * 3 + c) * MC + m] = jh[c];
                }
                __syncthreads();
                if (warp == 0) {
                    const OwnLayout ol = own_layout(MC, JS, (size_t)A.ews);
                    heat_unit<true>(Ps, S, hpart_at(), MC, view(), (const double *)(own + ol.ui), MC, lo, b, G, lane);
                }
                __syncthreads();
            }
        }
        if (tm) {
            const unsigned long long t4 = global_ns();
            const unsigned long long m0 = __ldcg(A.tmax), m1 = __ldcg(A.tmax + 1), m2 = __ldcg(A.tmax + 2);
            S.scal[SC_TPH0] = (double)(m0 - tph[0]);     // drift + site build (slowest block)
            S.scal[SC_TPH1] = (double)(tph[1] - m0);     // grid barrier after it
            S.scal[SC_TPH2] = (double)(m1 - tph[1]);     // staging + pair + RDF (slowest block)
            S.scal[SC_TPH3] = (double)(m2 - m1);         // unit reduction (slowest block)
            S.scal[SC_TPH4] = (double)(tph[3] - m2);     // grid barrier after it
            S.scal[SC_TPH5] = (double)(t4 - tph[3]);     // totals and thermostat factor (block 0)
            S.scal[SC_TPH6] = (double)(tph[0] - tph[5]); // kernel entry to the last step
            S.scal[SC_TPH7] = (double)(t4 - tph[0]);     // the last step
            tph[4] = t4;
            // every mark of this step came before the last barrier: zero for the next launch
            A.tmax[0] = A.tmax[1] = A.tmax[2] = 0ull;
        }
    }
    // ---- the last step's record; own state, forces and per-molecule results
    // back to global memory (after block 0's last totals are written)
    __syncthreads();
    if (A.nsteps > 0 && b == 0 && warp == 0) {
        const int gk = gk_step(A, A.nsteps - 1) ? RED_GK : 0;
        finish_step_warp(Ps, S, RED_SUM | RED_RECORD | RED_LAMBDA | EWM | gk, tot, lane, acc_s, kc_s);
        if (gk) gk_update(S, tot, lane);
    }
    if (b == 0 && warp == 0 && lane < AC_COUNT_) S.acc[lane] = acc_s[lane];  // the launch's running sums
    if (HEAT && A.nsteps > 0 && hf_step(A, A.nsteps - 1)) {  // uniform over the grid
        grid_sync(A.bar, A.err, target, on_timeout, A.wait_ns);
        if (b == 0 && warp == 0) heat_record(S, G, lane);
    }
    // the write-back starts at warp 1, so that block 0's record (warp 0) runs
    // beside it; it reads only block-held data the last barrier ordered
    const OwnLayout ol = own_layout(MC, JS, (size_t)A.ews);
    const double *ui_s = (const double *)(own + ol.ui);
    const int *np_s = (const int *)(own + ol.np);
    for (int t = (threadIdx.x + STEP_THREADS - 32) % STEP_THREADS; t < nm; t += blockDim.x) {
        const StateView sv = view();
        const int i = lo + t;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            S.R[c * N + i] = sv.R[c * MC + t];
            S.v[c * N + i] = sv.v[c * MC + t];
            S.Lm[c * N + i] = sv.L[c * MC + t];
            S.F[c * N + i] = sv.F[c * MC + t];
            S.tau[c * N + i] = sv.tau[c * MC + t];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            S.q[c * N + i] = sv.q[c * MC + t];
            S.Ui[c * N + i] = ui_s[c * MC + t];
        }
        S.npart[i] = np_s[t];
    }
    if (A.timing && b == 0) {  // uniform within block 0
        __syncthreads();
        if (threadIdx.x == 0) S.scal[SC_TPH8] = (double)(global_ns() - tph[4]);  // last step end to exit
    }
}

// ------------------------------------------------------------ host side
// shared memory of the fused step: the staged system, the partner queues of 16
// warps, the parameter tables, then the own region (state and partials of at
// most mcap molecules, j-split js) and an RDF histogram of rdf_cells counters
size_t ms2_step_smem_bytes(int NS, int tile, bool multi, int Np, int mcap, int js, int rdf_cells, size_t ews) {
    const size_t own = own_layout(mcap, js, ews).hist;
    return al16(pair_engine::smem_bytes(NS, tile, multi, Np, STEP_WARPS)) + own + sizeof(unsigned) * (size_t)rdf_cells;
}

int ms2_step_threads() { return STEP_THREADS; }

// fused-step kernel of a pair-kernel variant, or null where the per-phase
// kernels are used (FP64, 8 site slots, other mixtures)
// (heat: the variant with the heat-flux pass; Massieu sampling and heat flux
// together run on the per-phase kernels)
void *ms2_pick_step_kernel(int ns, unsigned ljm, unsigned qm, unsigned dm, int elec, bool multi, bool mass, bool heat) {
    if (mass && heat) return nullptr;
    if (elec == ELEC_EWALD) {  // water with single-site ions (several species); no Massieu or heat flux with Ewald
        if (multi && ns == 3 && ljm == 1 && qm == 7 && dm == 0 && !mass && !heat)
            return (void *)&k_step<3, 1u, 7u, 0u, ELEC_EWALD, true>;
        return nullptr;
    }
    if (multi) return nullptr;
    if (ns == 1 && ljm == 1 && qm == 0 && dm == 0 && elec == ELEC_NONE)
        return mass ? (void *)&k_step<1, 1u, 0u, 0u, ELEC_NONE, false, true>
                    : heat ? (void *)&k_step<1, 1u, 0u, 0u, ELEC_NONE, false, false, true>
                           : (void *)&k_step<1, 1u, 0u, 0u, ELEC_NONE, false>;
    if (ns == 3 && ljm == 1 && qm == 7 && dm == 0 && elec == ELEC_RF)
        return mass ? (void *)&k_step<3, 1u, 7u, 0u, ELEC_RF, false, true>
                    : heat ? (void *)&k_step<3, 1u, 7u, 0u, ELEC_RF, false, false, true>
                           : (void *)&k_step<3, 1u, 7u, 0u, ELEC_RF, false>;
    if (ns == 3 && ljm == 3 && qm == 0 && dm == 4 && elec == ELEC_RF && !mass)
        return heat ? (void *)&k_step<3, 3u, 0u, 4u, ELEC_RF, false, false, true>
                    : (void *)&k_step<3, 3u, 0u, 4u, ELEC_RF, false>;
    return nullptr;
}

// launch: grid = one block per SM (cooperative: all blocks resident)
cudaError_t ms2_launch_step(void *fn, int grid, size_t smem, cudaStream_t st, const SysParams *P, const DevSys &S,
                            const StepArgs &A) {
    void *args[] = {(void *)&P, (void *)&S, (void *)&A};
    return cudaLaunchCooperativeKernel(fn, grid, STEP_THREADS, args, smem, st);
}

// bytes of the reciprocal-space task scratch of a fused Ewald block
size_t ms2_step_ewald_scratch(int kx, int ky, int kz, int ny_per_chunk, int skc) {
    return std::max(std::max(ewald::sk_smem(kx, ky, kz, skc), ewald::sum_smem()),
                    ewald::force_smem(kx, kz, ny_per_chunk, STEP_THREADS));
}
