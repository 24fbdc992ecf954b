// K2: interaction partner search fused with site-pair energy, force, torque and
// molecular virial (paper, Sec. "Hybrid MPI & OpenMP Parallelization": the
// partner search, energy and force loops over molecules; Sec. "Massieu potential
// derivatives": LJ and Coulomb pair potentials, reaction field; Sec. "Algorithmic
// Developments": Ewald real-space part).
//
// Design (owner computes, no atomics): one warp owns molecule i and one j-range
// (grid.y splits the j loop into JSPLIT ranges).  The block stages its j-range in
// shared memory tile by tile; lanes test 32 candidates at a time on the integer
// centre lattice (exact minimum image by 32-bit wrap-around), partners are
// compacted into a per-warp queue with a ballot, and each full batch of 32
// partners is evaluated one partner per lane with all site pairs unrolled.
// Reaction field with point charges (neutral molecules) uses the exact identity
//   sum_ab q_a q_b (1/r_ab + k_RF r_ab^2 - c_RF) = sum_ab q_a q_b / r_ab - 2 mu_i.mu_j
// (mu = sum_a q_a s_a, the molecular charge dipole): the c_RF terms cancel and
// the k_RF part is a molecular dipole term with zero force, torque
// 2 C k_RF mu_i x mu_j and zero molecular virial.  The site-pair terms are then
// bare Coulomb; the k_RF site forces, which grow with r and cancel exactly over a
// neutral pair, never meet FP32 rounding.
// Site-pair arithmetic is FP32; each lane accumulates its partners in FP32
// registers, the warp reduces with shuffles in a fixed tree, and lane 0 writes
// one FP32 partial per (j-range, i).  The reduction over j-ranges is FP64 and in
// range order, so results are bitwise reproducible.
#include "ms2_internal.cuh"

#include "integrate_dev.cuh"
#include "pair_engine.cuh"

using namespace pair_engine;

// bytes of dynamic shared memory the pair kernel needs
size_t ms2_pair_smem_bytes(int NS, int tile, bool multi, int TJ, int wpb) {
    return pair_engine::smem_bytes(NS, tile, multi, TJ, wpb);
}

// grid: x = blocks of wpb molecules (one warp each), y = j-range; one FP32
// partial per (j-range, molecule)
template <int NS, unsigned LJM, unsigned QM, unsigned DM, int ELEC, bool MULTI, bool MASS = false>
__global__ void __launch_bounds__(256) k_pair(const SysParams *__restrict__ P, DevSys S, int TJ) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Eng = PairWarp<NS, LJM, QM, DM, ELEC, MULTI, MASS>;
    const int N = S.N;
    const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * wpb + warp;
    const int JS = gridDim.y, p = blockIdx.y;
    const int j0 = (int)(((long long)N * p) / JS), j1 = (int)(((long long)N * (p + 1)) / JS);
    Smem sm = carve<NS, Eng::TILE, MULTI>(smem_raw, TJ, wpb);
    int *wq = sm.queue + warp * QSTRIDE;
    load_tables<MULTI>(P, sm);
    Eng e;
    e.setup(P);
    const bool active = i < N;
    e.begin(P, S, active ? i : 0);
    for (int t0 = j0; t0 < j1; t0 += TJ) {
        const int tn = min(TJ, j1 - t0);
        __syncthreads();
        stage_tile<NS, DM, Eng::MOLD, MULTI>(sm, S, t0, tn, TJ, Eng::MOLD && e.rfq);
        __syncthreads();
        if (active) e.scan(sm, TJ, t0, tn, wq, lane);
    }
    if (!active) return;
    const PairOut o = e.finish(lane);
    if (lane == 0) {
        float *q = S.part + (size_t)p * MS2_NPV * N + i;
        q[PV_FX * N] = o.F[0]; q[PV_FY * N] = o.F[1]; q[PV_FZ * N] = o.F[2];
        q[PV_TX * N] = o.T[0]; q[PV_TY * N] = o.T[1]; q[PV_TZ * N] = o.T[2];
        q[PV_ULJ * N] = o.ulj; q[PV_UQQ * N] = o.uqq; q[PV_UDD * N] = o.udd; q[PV_W * N] = o.w;
        q[PV_NP * N] = (float)o.np;
        q[PV_VV * N] = o.vv;
    }
}

// Heat-flux power pass (Sec. 4, Eq. 6) after the reduction of a sampled step:
// the decomposition of k_pair, each warp's molecule i moving with its
// integer-time velocities (integ::heat_velocities); one FP32 partial
// sum_l d_kl P_kl per (j-range, i, component) into hpart.
template <int NS, unsigned LJM, unsigned QM, unsigned DM, int ELEC, bool MULTI>
__global__ void __launch_bounds__(256) k_heat(const SysParams *__restrict__ P, DevSys S, int TJ) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Eng = PairWarp<NS, LJM, QM, DM, ELEC, MULTI>;
    const int N = S.N;
    const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * wpb + warp;
    const int JS = gridDim.y, p = blockIdx.y;
    const int j0 = (int)(((long long)N * p) / JS), j1 = (int)(((long long)N * (p + 1)) / JS);
    Smem sm = carve<NS, Eng::TILE, MULTI>(smem_raw, TJ, wpb);
    int *wq = sm.queue + warp * QSTRIDE;
    load_tables<MULTI>(P, sm);
    Eng e;
    e.setup(P);
    const bool active = i < N;
    const int ii = active ? i : 0;
    e.begin(P, S, ii);
    float v[3], w[3];
    integ::heat_velocities<false>(P, integ::global_view(S), ii, v, w);
    e.begin_heat(v, w);
    for (int t0 = j0; t0 < j1; t0 += TJ) {
        const int tn = min(TJ, j1 - t0);
        __syncthreads();
        stage_tile<NS, DM, Eng::MOLD, MULTI>(sm, S, t0, tn, TJ, Eng::MOLD && e.rfq);
        __syncthreads();
        if (active) e.template scan<true>(sm, TJ, t0, tn, wq, lane);
    }
    if (!active) return;
    float jh[3];
    e.finish_heat(jh);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 3; ++k) S.hpart[((size_t)p * 3 + k) * N + i] = jh[k];
}

// FP64 variant for point LJ molecules (site-pair arithmetic in FP64 too):
// same owner/warp/ballot structure; partials are FP64.
__global__ void __launch_bounds__(256) k_pair_lj64(const SysParams *__restrict__ P, DevSys S, int TJ) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = S.N;
    const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * wpb + warp;
    const int JS = gridDim.y, p = blockIdx.y;
    const int j0 = (int)(((long long)N * p) / JS), j1 = (int)(((long long)N * (p + 1)) / JS);
    uint32_t *tX = (uint32_t *)smem_raw, *tY = tX + TJ, *tZ = tY + TJ;
    double *tR = (double *)(((uintptr_t)(tZ + TJ) + 15) & ~(uintptr_t)15);  // [3][TJ]
    int *wq = (int *)(tR + 3 * TJ) + warp * 64;
    const double L = P->L, c6 = P->c6d[0][0], c12 = P->c12d[0][0];
    const unsigned long long rc2 = P->rc2;
    const bool active = i < N;
    const int ii = active ? i : 0;
    const uint32_t Xi = S.X[ii], Yi = S.X[N + ii], Zi = S.X[2 * N + ii];
    const double Rxi = S.R[ii], Ryi = S.R[N + ii], Rzi = S.R[2 * N + ii];
    double fx = 0, fy = 0, fz = 0, u = 0, w = 0, vv = 0;
    int np = 0;
    for (int t0 = j0; t0 < j1; t0 += TJ) {
        const int tn = min(TJ, j1 - t0);
        __syncthreads();
        for (int k = threadIdx.x; k < tn; k += blockDim.x) {
            const int j = t0 + k;
            tX[k] = S.X[j]; tY[k] = S.X[N + j]; tZ[k] = S.X[2 * N + j];
            tR[k] = S.R[j]; tR[TJ + k] = S.R[N + j]; tR[2 * TJ + k] = S.R[2 * N + j];
        }
        __syncthreads();
        if (!active) continue;
        int qn = 0;
        auto interact = [&](int jl) {
            double d[3] = {tR[jl] - Rxi, tR[TJ + jl] - Ryi, tR[2 * TJ + jl] - Rzi};
#pragma unroll
            for (int k = 0; k < 3; ++k) d[k] -= L * rint(d[k] / L);
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], ri2 = 1.0 / r2;
            const double r6 = ri2 * ri2 * ri2, t6 = c6 * r6, t12 = c12 * r6 * r6;
            const double g = (6.0 * t6 - 12.0 * t12) * ri2;  // force on i = g * d
            u += t12 - t6;
            fx += g * d[0]; fy += g * d[1]; fz += g * d[2];
            w -= g * r2;
            vv += 180.0 * t12 - 54.0 * t6;  // u'' r^2 - 2 u' r of a point pair (Massieu derivatives)
            ++np;
        };
        for (int base = 0; base < tn; base += 32) {
            const int jl = base + lane;
            bool partner = false;
            if (jl < tn && t0 + jl != i) {
                const int dx = (int)(tX[jl] - Xi), dy = (int)(tY[jl] - Yi), dz = (int)(tZ[jl] - Zi);
                partner = lattice_d2(dx, dy, dz) < rc2;
            }
            const unsigned m = __ballot_sync(0xffffffffu, partner);
            if (partner) wq[qn + __popc(m & ((1u << lane) - 1u))] = jl;
            qn += __popc(m);
            __syncwarp();
            if (qn >= 32) {
                interact(wq[lane]);
                __syncwarp();
                qn -= 32;
                if (lane < qn) wq[lane] = wq[32 + lane];
                __syncwarp();
            }
        }
        if (qn > 0) {
            if (lane < qn) interact(wq[lane]);
            __syncwarp();
        }
    }
    if (!active) return;
    fx = warp_sum(fx); fy = warp_sum(fy); fz = warp_sum(fz);
    u = warp_sum(u); w = warp_sum(w); vv = warp_sum(vv); np = warp_sum(np);
    if (lane == 0) {
        double *o = S.part64 + (size_t)p * MS2_NPV * N + i;
        o[PV_FX * N] = fx; o[PV_FY * N] = fy; o[PV_FZ * N] = fz;
        o[PV_TX * N] = 0; o[PV_TY * N] = 0; o[PV_TZ * N] = 0;
        o[PV_ULJ * N] = u; o[PV_UQQ * N] = 0; o[PV_UDD * N] = 0; o[PV_W * N] = w;
        o[PV_NP * N] = (double)np;
        o[PV_VV * N] = vv;
    }
}

size_t ms2_pair64_smem_bytes(int TJ, int wpb) {
    return 3 * sizeof(uint32_t) * TJ + 16 + 3 * sizeof(double) * TJ + sizeof(int) * wpb * 64;
}

// ------------------------------------------------------------- dispatch
struct PairVariant {
    int ns;
    unsigned ljm, qm, dm;
    int elec;
    bool multi;
    void (*fn)(const SysParams *, DevSys, int);
    void (*mass)(const SysParams *, DevSys, int);  // variant that also sums d2U/dV2, or null
    void (*heat)(const SysParams *, DevSys, int);  // heat-flux power pass, or null (Ewald)
};

#define V(NS, LJM, QM, DM, E, M) {NS, LJM, QM, DM, E, M, &k_pair<NS, LJM, QM, DM, E, M>, nullptr, nullptr}
#define VH(NS, LJM, QM, DM, E, M) \
    {NS, LJM, QM, DM, E, M, &k_pair<NS, LJM, QM, DM, E, M>, nullptr, &k_heat<NS, LJM, QM, DM, E, M>}
#define VMH(NS, LJM, QM, DM, E, M)                                                                   \
    {NS, LJM, QM, DM, E, M, &k_pair<NS, LJM, QM, DM, E, M>, &k_pair<NS, LJM, QM, DM, E, M, true>, \
     &k_heat<NS, LJM, QM, DM, E, M>}
static const PairVariant kVariants[] = {
    VMH(1, 1u, 0u, 0u, ELEC_NONE, false),    // point LJ
    VMH(3, 1u, 7u, 0u, ELEC_RF, false),      // 3-site water, reaction field
    V(3, 1u, 7u, 0u, ELEC_EWALD, false),     // 3-site water, Ewald
    V(3, 1u, 7u, 0u, ELEC_EWALD, true),      // water + single-site ions, Ewald
    VH(3, 3u, 0u, 4u, ELEC_RF, false),       // 2 LJ + dipole (Stockmayer-like)
};
#undef V
#undef VH
#undef VMH

// generic fallbacks: runtime electrostatics, all slots may carry everything
static void (*const kGeneric[2][2])(const SysParams *, DevSys, int) = {
    {&k_pair<4, 0xFu, 0xFu, 0u, -1, true>, &k_pair<4, 0xFu, 0xFu, 0xFu, -1, true>},
    {&k_pair<8, 0xFFu, 0xFFu, 0u, -1, true>, &k_pair<8, 0xFFu, 0xFFu, 0xFFu, -1, true>},
};
static void (*const kGenericMass)(const SysParams *, DevSys, int) = &k_pair<4, 0xFu, 0xFu, 0u, -1, true, true>;
static void (*const kGenericHeat[2])(const SysParams *, DevSys, int) = {&k_heat<4, 0xFu, 0xFu, 0u, -1, true>,
                                                                        &k_heat<4, 0xFu, 0xFu, 0xFu, -1, true>};

// The heat-flux pass matching the pair kernel ms2_pick_pair_kernel returned for
// the same arguments (same slot padding and decomposition), or null (Ewald, FP64
// path, 8 site slots).
void *ms2_pick_heat_kernel(int ns, unsigned ljm, unsigned qm, unsigned dm, int elec, bool multi, const void *pair_fn) {
    if (elec == ELEC_EWALD) return nullptr;
    for (const PairVariant &v : kVariants)
        if ((const void *)v.fn == pair_fn || (const void *)v.mass == pair_fn) return (void *)v.heat;
    for (int d = 0; d < 2; ++d)
        if ((const void *)kGeneric[0][d] == pair_fn) return (void *)kGenericHeat[d];
    if ((const void *)kGenericMass == pair_fn) return (void *)kGenericHeat[0];
    (void)ns; (void)ljm; (void)qm; (void)dm; (void)multi;
    return nullptr;
}

// Picks the kernel for a system's slot pattern.  Returns the padded slot count
// the kernel expects in *ns_used (the site arrays must be laid out with it).
// With mass, the variant that also sums the second volume derivative (null where
// none is built: dipoles, Ewald, 8 site slots).
void *ms2_pick_pair_kernel(int ns, unsigned ljm, unsigned qm, unsigned dm, int elec, bool multi, int *ns_used,
                           int *tile, bool *mult_used, bool mass) {
    for (const PairVariant &v : kVariants) {
        if (v.ns == ns && v.ljm == ljm && v.qm == qm && v.dm == dm && v.elec == elec && v.multi == multi &&
            (!mass || v.mass)) {
            *ns_used = ns;
            *tile = pair_engine::tile_code(pair_engine::popc_c(v.dm), v.qm != 0 && v.elec == ELEC_RF);
            *mult_used = multi;
            return (void *)(mass ? v.mass : v.fn);
        }
        if (mass) continue;
        // a single-species system can use the multi-species variant of its pattern
        if (v.ns == ns && v.ljm == ljm && v.qm == qm && v.dm == dm && v.elec == elec && v.multi && !multi) {
            bool exact_single = false;
            for (const PairVariant &u : kVariants)
                if (u.ns == ns && u.ljm == ljm && u.qm == qm && u.dm == dm && u.elec == elec && !u.multi)
                    exact_single = true;
            if (!exact_single) {
                *ns_used = ns;
                *tile = pair_engine::tile_code(pair_engine::popc_c(v.dm), v.qm != 0 && v.elec == ELEC_RF);
                *mult_used = true;
                return (void *)v.fn;
            }
        }
    }
    const int g = ns <= 4 ? 0 : 1;
    *ns_used = g ? 8 : 4;
    // the generic kernels keep every slot's dipole (when they take dipoles) and the
    // molecular dipoles (their electrostatics are chosen at run time)
    *tile = pair_engine::tile_code(dm != 0 ? *ns_used : 0, true);
    *mult_used = true;
    if (mass) return (g == 0 && dm == 0 && elec != ELEC_EWALD) ? (void *)kGenericMass : nullptr;
    return (void *)kGeneric[g][dm != 0];
}
