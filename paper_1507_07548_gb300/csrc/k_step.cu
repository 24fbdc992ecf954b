// Fused MD step of one system: a cooperative persistent kernel, one block of
// 512 threads per SM, runs a whole chunk of leapfrog steps (paper, Sec. "Hybrid
// MPI & OpenMP Parallelization": the partner search, energy and force loops over
// molecules; the rigid-body leapfrog with isokinetic scaling and the thermo
// reduction as in k_integrate.cu).  Per step:
//
//   drift + site build   (molecules spread over all blocks, a quad each)
//   -- grid barrier --
//   stage the whole system in shared memory; pair items (molecule i, j-range p)
//   spread over all warps of the grid; every 'rdf_every' steps the RDF
//   -- grid barrier --
//   reduction units (8 molecules per warp): F, tau, energies, kinetic energies
//   -- grid barrier --
//   every block sums the units in fixed order and derives the thermostat
//   factor itself; block 0 records the step scalars.
//
// The phases are the device functions of the per-phase kernels (drift_quad,
// PairWarp, reduce_unit, reduce_totals, finish_step) on the same work
// decomposition (j-ranges, tile segmentation, reduction units), so a chunk run
// here is bitwise identical to the same chunk run as separate kernels.  What the
// fusion saves is the kernel boundaries (a launch costs ~2 us, a bounded grid
// barrier ~1.2 us on GB300), the last-block tail of the reduction and the
// re-staging of tiles per block.
//
// Every grid-barrier wait is bounded (2 s of %globaltimer).  A block that gives
// up sets a sticky flag that ends every other wait at once and marks the system
// (SC_KERR); the kernel then runs to its end without waiting and the host
// reports MS2_ETIMEOUT at its next read.
#include "ms2_internal.cuh"

#include "integrate_dev.cuh"
#include "pair_engine.cuh"

using namespace pair_engine;
using namespace integ;

namespace {

constexpr int STEP_THREADS = 512;
constexpr int STEP_WARPS = STEP_THREADS / 32;
constexpr unsigned long long WAIT_NS = 2000000000ull;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_u32(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// monotone-counter grid barrier: the k-th barrier of a launch waits for
// count >= k * gridDim.x
__device__ __forceinline__ void grid_sync(unsigned *count, unsigned *err, unsigned &target, double *scal) {
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
        __threadfence();
        red_release_u32(count, 1u);
        const unsigned long long t0 = global_ns();
        while (ld_acquire_u32(count) < target) {
            if (ld_acquire_u32(err) != 0u) break;  // another block gave up
            if (global_ns() - t0 > WAIT_NS) {
                atomicExch(err, 1u);
                scal[SC_KERR] = 1.0;
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// site-site RDF of the staged configuration (the k_rdf arithmetic, reading
// the shared-memory tile): molecules i = block, block + grid, ...; threads over j > i
template <int NS, bool MULTI>
__device__ void rdf_tile(const SysParams *__restrict__ P, const DevSys &S, const Smem &sm, int TJ, unsigned *hist) {
    const int N = S.N, nb = S.rdf_bins, rows = S.rdf_rows, T = P->n_ljt;
    for (int k = threadIdx.x; k < rows * nb; k += blockDim.x) hist[k] = 0u;
    __syncthreads();
    const float l2l = P->lat_to_len, l2 = P->len_to_lat;
    const float rmax2 = S.rdf_rmax2, inv_dr = S.rdf_inv_dr;
    const uint32_t *tx[3] = {sm.tX, sm.tY, sm.tZ};
    for (int i = blockIdx.x; i < N; i += gridDim.x) {
        const int spi = MULTI ? sm.tsp[i] : 0;
        for (int a = 0; a < NS; ++a) {
            const int ta = S.rdf_kind[spi * MS2_MAXS + a];
            if (ta < 0) continue;
            uint32_t Xa[3];
            for (int c = 0; c < 3; ++c) Xa[c] = tx[c][i] + (uint32_t)__float2int_rn(sm.ts[(c * NS + a) * TJ + i] * l2);
            for (int j = i + 1 + threadIdx.x; j < N; j += blockDim.x) {
                const int spj = MULTI ? sm.tsp[j] : 0;
                for (int b = 0; b < NS; ++b) {
                    const int tb = S.rdf_kind[spj * MS2_MAXS + b];
                    if (tb < 0) continue;
                    float r2 = 0.f;
                    for (int c = 0; c < 3; ++c) {
                        const uint32_t Xb = tx[c][j] + (uint32_t)__float2int_rn(sm.ts[(c * NS + b) * TJ + j] * l2);
                        const float d = (float)(int)(Xb - Xa[c]) * l2l;
                        r2 += d * d;
                    }
                    if (!(r2 < rmax2)) continue;
                    const int bin = (int)(sqrtf(r2) * inv_dr);
                    if (bin >= nb) continue;
                    const int t1 = min(ta, tb), t2 = max(ta, tb);
                    const int row = t1 * T - t1 * (t1 - 1) / 2 + (t2 - t1);
                    atomicAdd(&hist[row * nb + bin], 1u);
                }
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < rows * nb; k += blockDim.x)
        if (hist[k]) atomicAdd(&S.rdf[k], (unsigned long long)hist[k]);
}

}  // namespace

template <int NS, unsigned LJM, unsigned QM, unsigned DM, int ELEC, bool MULTI>
__global__ void __launch_bounds__(STEP_THREADS, 1) k_step(const SysParams *__restrict__ P, DevSys S, StepArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Eng = PairWarp<NS, LJM, QM, DM, ELEC, MULTI>;
    __shared__ double tot[MS2_NRED];
    __shared__ double lam_s;
    const int N = S.N, G = gridDim.x, b = blockIdx.x, JS = S.jsplit;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Smem sm = carve<NS, Eng::DMU, MULTI>(smem_raw, A.Np, STEP_WARPS);
    unsigned *hist = (unsigned *)(smem_raw + ((smem_bytes(NS, Eng::DMU, MULTI, A.Np, STEP_WARPS) + 15) & ~(size_t)15));
    int *wq = sm.queue + warp * 64;
    load_tables<MULTI>(P, sm);
    Eng e;
    e.setup(P);
    if (b == 0 && threadIdx.x == 0) *A.bar_next = 0u;
    unsigned target = 0;
    double lam = __ldcg(S.scal + SC_LAMBDA);
    // drift share of this block: molecules [lo, hi), by warps 1.. (warp 0 of
    // block 0 records the previous step meanwhile)
    const int lo = (int)((long long)N * b / G), hi = (int)((long long)N * (b + 1) / G);
    const bool rfq = Eng::MOLD && e.rfq;
    const int nitems = N * JS;
    const unsigned long long t_entry = (A.timing && b == 0 && threadIdx.x == 0) ? global_ns() : 0ull;
    unsigned long long t_ph[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < A.nsteps; ++k) {
        if (A.timing && b == 0 && threadIdx.x == 0 && k == A.nsteps - 1) t_ph[0] = global_ns();
        // ---- drift + site build
        if (warp >= 1)
            for (int m0 = lo + 8 * (warp - 1); m0 < hi; m0 += 8 * (STEP_WARPS - 1)) {
                const int i = m0 + (lane >> 2);
                drift_quad(P, S, i, i < hi, lane & 3, false, lam);
            }
        grid_sync(A.bar, A.err, target, S.scal);
        const bool tm = A.timing && b == 0 && threadIdx.x == 0 && k == A.nsteps - 1;
        const unsigned long long tp0 = tm ? global_ns() : 0ull;
        if (tm) t_ph[1] = tp0;
        // ---- stage the whole system, pair items, RDF
        stage_tile<NS, Eng::DMU, MULTI>(sm, S, 0, N, A.Np, rfq);
        __syncthreads();
        for (int it = b + G * warp; it < nitems; it += G * STEP_WARPS) {
            const int i = it % N, p = it / N;
            const int j0 = (int)(((long long)N * p) / JS), j1 = (int)(((long long)N * (p + 1)) / JS);
            e.begin_tile(P, sm, A.Np, i);
            for (int t0 = j0; t0 < j1; t0 += A.TJ) e.scan(shifted(sm, t0), A.Np, t0, min(A.TJ, j1 - t0), wq, lane);
            const PairOut o = e.finish(lane);
            if (lane == 0) {
                float *q = S.part + (size_t)p * MS2_NPV * N + i;
                q[PV_FX * N] = o.F[0]; q[PV_FY * N] = o.F[1]; q[PV_FZ * N] = o.F[2];
                q[PV_TX * N] = o.T[0]; q[PV_TY * N] = o.T[1]; q[PV_TZ * N] = o.T[2];
                q[PV_ULJ * N] = o.ulj; q[PV_UQQ * N] = o.uqq; q[PV_UDD * N] = o.udd; q[PV_W * N] = o.w;
                q[PV_NP * N] = (float)o.np;
            }
        }
        if (A.rdf_every > 0 && ((A.s0 + k + 1) % A.rdf_every) == 0) {
            __syncthreads();
            rdf_tile<NS, MULTI>(P, S, sm, A.Np, hist);
        }
        grid_sync(A.bar, A.err, target, S.scal);
        if (tm) {
            t_ph[2] = global_ns();
            S.scal[SC_TPAIR] = (double)(t_ph[2] - tp0);
        }
        // ---- reduction units
        for (int vb = b + G * warp; vb < S.nvb; vb += G * STEP_WARPS)
            reduce_unit(P, S, RED_SUM | RED_LAMBDA, vb, lane);
        grid_sync(A.bar, A.err, target, S.scal);
        if (tm) t_ph[3] = global_ns();
        // ---- totals in every block; thermostat factor for the next drift
        reduce_totals(S, S.nvb, tot);
        __syncthreads();
        if (threadIdx.x == 0) lam_s = lambda_of(P, tot);
        __syncthreads();
        lam = lam_s;
        if (b == 0 && threadIdx.x == 0) finish_step(P, S, RED_SUM | RED_RECORD | RED_LAMBDA, tot);
        if (tm) {
            t_ph[4] = global_ns();
            S.scal[SC_TPH0] = (double)(t_ph[1] - t_ph[0]);  // drift + site build + barrier
            S.scal[SC_TPH1] = (double)(t_ph[2] - t_ph[1]);  // staging + pair + RDF + barrier
            S.scal[SC_TPH2] = (double)(t_ph[3] - t_ph[2]);  // reduction units + barrier
            S.scal[SC_TPH3] = (double)(t_ph[4] - t_ph[3]);  // totals, thermostat factor, step record
            S.scal[SC_TPH4] = (double)(t_ph[0] - t_entry);  // kernel entry to the last step
        }
    }
}

// ------------------------------------------------------------ host side
// shared memory of the fused step: the staged system, the partner queues of 16
// warps, the parameter tables and an RDF histogram of rdf_cells counters
size_t ms2_step_smem_bytes(int NS, bool dmu, bool multi, int Np, int rdf_cells) {
    return ((pair_engine::smem_bytes(NS, dmu, multi, Np, STEP_WARPS) + 15) & ~(size_t)15) +
           sizeof(unsigned) * (size_t)rdf_cells;
}

int ms2_step_threads() { return STEP_THREADS; }

// fused-step kernel of a pair-kernel variant, or null where the per-phase
// kernels are used (Ewald, FP64, 8 site slots)
void *ms2_pick_step_kernel(int ns, unsigned ljm, unsigned qm, unsigned dm, int elec, bool multi) {
    if (elec == ELEC_EWALD) return nullptr;
    if (!multi) {
        if (ns == 1 && ljm == 1 && qm == 0 && dm == 0 && elec == ELEC_NONE)
            return (void *)&k_step<1, 1u, 0u, 0u, ELEC_NONE, false>;
        if (ns == 3 && ljm == 1 && qm == 7 && dm == 0 && elec == ELEC_RF)
            return (void *)&k_step<3, 1u, 7u, 0u, ELEC_RF, false>;
        if (ns == 3 && ljm == 3 && qm == 0 && dm == 4 && elec == ELEC_RF)
            return (void *)&k_step<3, 3u, 0u, 4u, ELEC_RF, false>;
    }
    return nullptr;
}

// launch: grid = one block per SM (cooperative: all blocks resident)
cudaError_t ms2_launch_step(void *fn, int grid, size_t smem, cudaStream_t st, const SysParams *P, const DevSys &S,
                            const StepArgs &A) {
    void *args[] = {(void *)&P, (void *)&S, (void *)&A};
    return cudaLaunchCooperativeKernel(fn, grid, STEP_THREADS, args, smem, st);
}
