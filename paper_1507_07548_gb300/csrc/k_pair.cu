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

namespace {

constexpr unsigned FULL = 0xffffffffu;

struct Smem {
    uint32_t *tX, *tY, *tZ;
    float *ts, *tmu, *tmd;
    int *tsp, *queue;
    float *sq, *sql, *sc6, *sc12, *sc6l, *sc12l;
    int *sljt;
};

template <int NS, bool DMU, bool MULTI, bool MOLD>
__device__ __forceinline__ Smem carve(unsigned char *base, int TJ, int wpb) {
    Smem m;
    m.tX = (uint32_t *)base;
    m.tY = m.tX + TJ;
    m.tZ = m.tY + TJ;
    m.ts = (float *)(m.tZ + TJ);
    m.tmu = m.ts + 3 * NS * TJ;
    m.tmd = m.tmu + (DMU ? 3 * NS * TJ : 0);
    m.tsp = (int *)(m.tmd + (MOLD ? 3 * TJ : 0));
    m.queue = m.tsp + (MULTI ? TJ : 0);
    m.sq = (float *)(m.queue + wpb * 64);
    m.sql = m.sq + MS2_MAXSP * MS2_MAXS;
    m.sljt = (int *)(m.sql + MS2_MAXSP * MS2_MAXS);
    m.sc6 = (float *)(m.sljt + MS2_MAXSP * MS2_MAXS);
    m.sc12 = m.sc6 + MS2_MAXT * MS2_MAXT;
    m.sc6l = m.sc12 + MS2_MAXT * MS2_MAXT;
    m.sc12l = m.sc6l + MS2_MAXT * MS2_MAXT;
    return m;
}

}  // namespace

// bytes of dynamic shared memory the pair kernel needs
size_t ms2_pair_smem_bytes(int NS, bool dmu, bool multi, int TJ, int wpb) {
    size_t n = 3 * sizeof(uint32_t) * TJ + sizeof(float) * 3 * NS * TJ;
    if (dmu) n += sizeof(float) * 3 * NS * TJ;
    n += sizeof(float) * 3 * TJ;  // molecular dipoles (reaction field; reserved always)
    if (multi) n += sizeof(int) * TJ;
    n += sizeof(int) * wpb * 64;
    n += 2 * sizeof(float) * MS2_MAXSP * MS2_MAXS + sizeof(int) * MS2_MAXSP * MS2_MAXS;
    n += 4 * sizeof(float) * MS2_MAXT * MS2_MAXT;
    return n;
}

// NS: site slots per molecule; LJM/QM/DM: slot bit masks that may carry LJ,
// charge, dipole; ELEC: ELEC_NONE/RF/EWALD or -1 = read from the parameters;
// MULTI: several species (per-molecule parameter lookup).
template <int NS, unsigned LJM, unsigned QM, unsigned DM, int ELEC, bool MULTI>
__global__ void __launch_bounds__(256) k_pair(const SysParams *__restrict__ P, DevSys S, int TJ) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool DMU = DM != 0;
    constexpr bool MOLD = QM != 0 && (ELEC == ELEC_RF || ELEC < 0);  // molecular-dipole RF term
    const int N = S.N;
    const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * wpb + warp;
    const int JS = gridDim.y, p = blockIdx.y;
    const int j0 = (int)(((long long)N * p) / JS), j1 = (int)(((long long)N * (p + 1)) / JS);
    Smem sm = carve<NS, DMU, MULTI, true>(smem_raw, TJ, wpb);
    const bool rfq = MOLD && P->elec == ELEC_RF;
    int *wq = sm.queue + warp * 64;

    const int elec = ELEC >= 0 ? ELEC : P->elec;
    const float C = P->coulomb, Clo = P->coulomb_lo, krf = P->krf, crf = P->crf, alpha = P->alpha,
                tasp = P->two_alpha_sqrtpi;
    const float l2l = P->lat_to_len, l2l_lo = P->lat_to_len_lo;
    const unsigned long long rc2 = P->rc2;

    if (MULTI) {
        for (int k = threadIdx.x; k < MS2_MAXSP * MS2_MAXS; k += blockDim.x) {
            sm.sq[k] = P->q[k / MS2_MAXS][k % MS2_MAXS];
            sm.sql[k] = P->qlo[k / MS2_MAXS][k % MS2_MAXS];
            sm.sljt[k] = P->ljt[k / MS2_MAXS][k % MS2_MAXS];
        }
        for (int k = threadIdx.x; k < MS2_MAXT * MS2_MAXT; k += blockDim.x) {
            sm.sc6[k] = P->c6[k / MS2_MAXT][k % MS2_MAXT];
            sm.sc12[k] = P->c12[k / MS2_MAXT][k % MS2_MAXT];
            sm.sc6l[k] = P->c6lo[k / MS2_MAXT][k % MS2_MAXT];
            sm.sc12l[k] = P->c12lo[k / MS2_MAXT][k % MS2_MAXT];
        }
    }

    const bool active = i < N;
    const int ii = active ? i : 0;
    const uint32_t Xi = S.X[ii], Yi = S.X[N + ii], Zi = S.X[2 * N + ii];
    float si[NS][3], mui[NS][3];
#pragma unroll
    for (int a = 0; a < NS; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            si[a][k] = S.s[(k * NS + a) * N + ii];
            mui[a][k] = DMU && ((DM >> a) & 1) ? S.mu[(k * NS + a) * N + ii] : 0.f;
        }
    const int spi = MULTI ? S.species[ii] : 0;
    // Coefficient products are kept as hi + lo float pairs: a single FP32
    // rounding of C q_a q_b or 4 eps sigma^12 would scale every term of that
    // site-pair kind the same way and bias the (strongly cancelling) sums.
    float qi[NS], qih[NS], qil[NS], hq[NS][NS], hql[NS][NS], hc6[NS][NS], hc12[NS][NS], hc6l[NS][NS], hc12l[NS][NS];
    int ljti[NS];
#pragma unroll
    for (int a = 0; a < NS; ++a) {
        qi[a] = P->q[spi][a];
        ljti[a] = P->ljt[spi][a];
        qih[a] = P->cq[spi][a];                         // (C q_a) as hi + lo, from FP64
        qil[a] = P->cqlo[spi][a];
    }
    if (!MULTI) {
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
            for (int b = 0; b < NS; ++b) {
                const float qb = P->q[0][b], qbl = P->qlo[0][b];
                hq[a][b] = qih[a] * qb;
                hql[a][b] = fmaf(qih[a], qb, -hq[a][b]) + fmaf(qih[a], qbl, qil[a] * qb);
                const int ta = P->ljt[0][a], tb = P->ljt[0][b];
                const bool on = ta >= 0 && tb >= 0;
                const int ia = on ? ta : 0, ib = on ? tb : 0;
                hc6[a][b] = on ? P->c6[ia][ib] : 0.f;
                hc12[a][b] = on ? P->c12[ia][ib] : 0.f;
                hc6l[a][b] = on ? P->c6lo[ia][ib] : 0.f;
                hc12l[a][b] = on ? P->c12lo[ia][ib] : 0.f;
            }
    }

    float fa[NS][3], ea[NS][3];
#pragma unroll
    for (int a = 0; a < NS; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) fa[a][k] = ea[a][k] = 0.f;
    float ulj = 0.f, uqq = 0.f, udd = 0.f, w = 0.f;
    int np = 0;
    float mdi[3] = {0.f, 0.f, 0.f}, erf_[3] = {0.f, 0.f, 0.f};  // mu_i and sum_j mu_j
    if (MOLD && rfq)
#pragma unroll
        for (int k = 0; k < 3; ++k) mdi[k] = S.mum[k * N + ii];

    // evaluate one partner (tile-local index jl) into the lane's accumulators
    auto interact = [&](int jl) {
        const int dxi = (int)(sm.tX[jl] - Xi), dyi = (int)(sm.tY[jl] - Yi), dzi = (int)(sm.tZ[jl] - Zi);
        // lattice difference -> length with the scale split in two floats, so the
        // FP32 rounding of L/2^32 does not scale every displacement the same way
        const float fxi = (float)dxi, fyi = (float)dyi, fzi = (float)dzi;
        const float dx = fmaf(fxi, l2l, fxi * l2l_lo), dy = fmaf(fyi, l2l, fyi * l2l_lo),
                    dz = fmaf(fzi, l2l, fzi * l2l_lo);
        const int TJl = TJ;
        const int spj = MULTI ? sm.tsp[jl] : 0;
        float pj[NS][3], muj[NS][3];
#pragma unroll
        for (int b = 0; b < NS; ++b) {
            pj[b][0] = dx + sm.ts[(0 * NS + b) * TJl + jl];
            pj[b][1] = dy + sm.ts[(1 * NS + b) * TJl + jl];
            pj[b][2] = dz + sm.ts[(2 * NS + b) * TJl + jl];
#pragma unroll
            for (int k = 0; k < 3; ++k)
                muj[b][k] = DMU && ((DM >> b) & 1) ? sm.tmu[(k * NS + b) * TJl + jl] : 0.f;
        }
        // Molecular virial -d.F_ij, written with d = r_ab - (s_jb - s_ia) as
        //   -sum_ab f_ab.r_ab + sum_b s_jb.G_b - sum_a s_ia.A_a,
        //   G_b = sum_a f_ab, A_a = sum_b f_ab   (per pair),
        // so that no FP32 force sum is multiplied by the long lever arm d and no
        // long accumulation of site forces meets a lever arm at all.
        float Gb[NS][3], Aa[NS][3];
#pragma unroll
        for (int b = 0; b < NS; ++b) Gb[b][0] = Gb[b][1] = Gb[b][2] = Aa[b][0] = Aa[b][1] = Aa[b][2] = 0.f;
        float wsite = 0.f;
#pragma unroll
        for (int a = 0; a < NS; ++a) {
#pragma unroll
            for (int b = 0; b < NS; ++b) {
                const bool mlj = (LJM >> a) & (LJM >> b) & 1u;
                const bool mq = (QM >> a) & (QM >> b) & 1u;
                const bool md = (DM >> a) & (DM >> b) & 1u;
                if (!(mlj || (mq && elec != ELEC_NONE) || (md && elec != ELEC_NONE))) continue;
                const float rx = pj[b][0] - si[a][0], ry = pj[b][1] - si[a][1], rz = pj[b][2] - si[a][2];
                float r2 = rx * rx + ry * ry + rz * rz;
                if (MULTI) r2 = fmaxf(r2, 1e-12f);
                // rsqrt approximation + one Newton step: unbiased to ~1 ulp
                float rinv = rsqrtf(r2);
                rinv = fmaf(rinv, fmaf(-0.5f * r2 * rinv, rinv, 0.5f), rinv);
                const float rinv2 = rinv * rinv;
                float g = 0.f;
                if (mlj) {
                    float c6, c12, c6l, c12l;
                    if (MULTI) {
                        const int ta = ljti[a], tb = sm.sljt[spj * MS2_MAXS + b];
                        const bool on = ta >= 0 && tb >= 0;
                        const int idx = on ? ta * MS2_MAXT + tb : 0;
                        c6 = on ? sm.sc6[idx] : 0.f;
                        c12 = on ? sm.sc12[idx] : 0.f;
                        c6l = on ? sm.sc6l[idx] : 0.f;
                        c12l = on ? sm.sc12l[idx] : 0.f;
                    } else {
                        c6 = hc6[a][b];
                        c12 = hc12[a][b];
                        c6l = hc6l[a][b];
                        c12l = hc12l[a][b];
                    }
                    const float r6 = rinv2 * rinv2 * rinv2, r12 = r6 * r6;
                    const float t6 = fmaf(c6, r6, c6l * r6), t12 = fmaf(c12, r12, c12l * r12);
                    ulj += t12 - t6;
                    g += (6.f * t6 - 12.f * t12) * rinv2;
                }
                if (mq && elec != ELEC_NONE) {
                    float cqq, cql;
                    if (MULTI) {
                        const float qb = sm.sq[spj * MS2_MAXS + b], qbl = sm.sql[spj * MS2_MAXS + b];
                        cqq = qih[a] * qb;
                        cql = fmaf(qih[a], qb, -cqq) + fmaf(qih[a], qbl, qil[a] * qb);
                    } else {
                        cqq = hq[a][b];
                        cql = hql[a][b];
                    }
                    float bu, bg;  // energy and force brackets
                    if (elec == ELEC_RF) {  // bare Coulomb; the RF part is a molecular term
                        bu = rinv;
                        bg = -rinv * rinv2;
                    } else {
                        const float ar = alpha * r2 * rinv;
                        const float ec = erfcf(ar), ex = expf(-ar * ar);
                        bu = ec * rinv;
                        bg = -(ec * rinv + tasp * ex) * rinv2;
                    }
                    uqq += fmaf(cqq, bu, cql * bu);
                    g += fmaf(cqq, bg, cql * bg);
                }
                if (md && elec != ELEC_NONE) {
                    const float rinv3 = rinv * rinv2, rinv5 = rinv3 * rinv2, rinv7 = rinv5 * rinv2;
                    const float mab = mui[a][0] * muj[b][0] + mui[a][1] * muj[b][1] + mui[a][2] * muj[b][2];
                    const float mar = mui[a][0] * rx + mui[a][1] * ry + mui[a][2] * rz;
                    const float mbr = muj[b][0] * rx + muj[b][1] * ry + muj[b][2] * rz;
                    const float kd = elec == ELEC_RF ? 2.f * krf : 0.f;
                    udd += C * (mab * rinv3 - 3.f * mar * mbr * rinv5 - kd * mab);
                    const float cr = C * (15.f * mar * mbr * rinv7 - 3.f * mab * rinv5);
                    const float cma = -3.f * C * mbr * rinv5, cmb = -3.f * C * mar * rinv5;
                    const float fx = cr * rx + cma * mui[a][0] + cmb * muj[b][0];
                    const float fy = cr * ry + cma * mui[a][1] + cmb * muj[b][1];
                    const float fz = cr * rz + cma * mui[a][2] + cmb * muj[b][2];
                    Aa[a][0] += fx; Aa[a][1] += fy; Aa[a][2] += fz;
                    Gb[b][0] += fx; Gb[b][1] += fy; Gb[b][2] += fz;
                    wsite -= fx * rx + fy * ry + fz * rz;
                    const float ce = 3.f * C * mbr * rinv5, cm = -C * (rinv3 - kd);
                    ea[a][0] += ce * rx + cm * muj[b][0];
                    ea[a][1] += ce * ry + cm * muj[b][1];
                    ea[a][2] += ce * rz + cm * muj[b][2];
                }
                Aa[a][0] = fmaf(g, rx, Aa[a][0]); Aa[a][1] = fmaf(g, ry, Aa[a][1]); Aa[a][2] = fmaf(g, rz, Aa[a][2]);
                Gb[b][0] = fmaf(g, rx, Gb[b][0]); Gb[b][1] = fmaf(g, ry, Gb[b][1]); Gb[b][2] = fmaf(g, rz, Gb[b][2]);
                wsite = fmaf(-g, r2, wsite);
            }
        }
#pragma unroll
        for (int b = 0; b < NS; ++b)
            wsite += sm.ts[(0 * NS + b) * TJl + jl] * Gb[b][0] + sm.ts[(1 * NS + b) * TJl + jl] * Gb[b][1] +
                     sm.ts[(2 * NS + b) * TJl + jl] * Gb[b][2];
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            wsite -= si[a][0] * Aa[a][0] + si[a][1] * Aa[a][1] + si[a][2] * Aa[a][2];
            fa[a][0] += Aa[a][0]; fa[a][1] += Aa[a][1]; fa[a][2] += Aa[a][2];
        }
        w += wsite;
        if (MOLD && rfq) {
            erf_[0] += sm.tmd[jl];
            erf_[1] += sm.tmd[TJl + jl];
            erf_[2] += sm.tmd[2 * TJl + jl];
        }
        ++np;
    };

    for (int t0 = j0; t0 < j1; t0 += TJ) {
        const int tn = min(TJ, j1 - t0);
        __syncthreads();
        for (int k = threadIdx.x; k < tn; k += blockDim.x) {
            const int j = t0 + k;
            sm.tX[k] = S.X[j];
            sm.tY[k] = S.X[N + j];
            sm.tZ[k] = S.X[2 * N + j];
#pragma unroll
            for (int c = 0; c < 3 * NS; ++c) sm.ts[c * TJ + k] = S.s[c * N + j];
            if (DMU) {
#pragma unroll
                for (int c = 0; c < 3 * NS; ++c) sm.tmu[c * TJ + k] = S.mu[c * N + j];
            }
            if (MULTI) sm.tsp[k] = S.species[j];
            if (MOLD && rfq) {
                sm.tmd[k] = S.mum[j];
                sm.tmd[TJ + k] = S.mum[N + j];
                sm.tmd[2 * TJ + k] = S.mum[2 * N + j];
            }
        }
        __syncthreads();
        if (!active) continue;
        int qn = 0;
        for (int base = 0; base < tn; base += 32) {
            const int jl = base + lane;
            bool partner = false;
            if (jl < tn && t0 + jl != i) {
                const int dx = (int)(sm.tX[jl] - Xi), dy = (int)(sm.tY[jl] - Yi), dz = (int)(sm.tZ[jl] - Zi);
                partner = lattice_d2(dx, dy, dz) < rc2;
            }
            const unsigned m = __ballot_sync(FULL, partner);
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

    // fixed-tree warp reduction, then one partial per (j-range, molecule)
#pragma unroll
    for (int a = 0; a < NS; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            fa[a][k] = warp_sum(fa[a][k]);
            if (DMU && ((DM >> a) & 1)) ea[a][k] = warp_sum(ea[a][k]);
        }
    if (MOLD && rfq)
#pragma unroll
        for (int k = 0; k < 3; ++k) erf_[k] = warp_sum(erf_[k]);
    ulj = warp_sum(ulj);
    uqq = warp_sum(uqq);
    udd = warp_sum(udd);
    w = warp_sum(w);
    np = warp_sum(np);
    if (lane == 0) {
        float F[3] = {0.f, 0.f, 0.f}, T[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            F[0] += fa[a][0]; F[1] += fa[a][1]; F[2] += fa[a][2];
            T[0] += si[a][1] * fa[a][2] - si[a][2] * fa[a][1];
            T[1] += si[a][2] * fa[a][0] - si[a][0] * fa[a][2];
            T[2] += si[a][0] * fa[a][1] - si[a][1] * fa[a][0];
            if (DMU && ((DM >> a) & 1)) {
                T[0] += mui[a][1] * ea[a][2] - mui[a][2] * ea[a][1];
                T[1] += mui[a][2] * ea[a][0] - mui[a][0] * ea[a][2];
                T[2] += mui[a][0] * ea[a][1] - mui[a][1] * ea[a][0];
            }
        }
        if (MOLD && rfq) {  // -2 C k_RF mu_i.mu_j and its torque 2 C k_RF mu_i x mu_j
            const float c2 = 2.f * C * krf;
            uqq -= c2 * (mdi[0] * erf_[0] + mdi[1] * erf_[1] + mdi[2] * erf_[2]);
            T[0] += c2 * (mdi[1] * erf_[2] - mdi[2] * erf_[1]);
            T[1] += c2 * (mdi[2] * erf_[0] - mdi[0] * erf_[2]);
            T[2] += c2 * (mdi[0] * erf_[1] - mdi[1] * erf_[0]);
        }
        float *o = S.part + (size_t)p * MS2_NPV * N + i;
        o[PV_FX * N] = F[0]; o[PV_FY * N] = F[1]; o[PV_FZ * N] = F[2];
        o[PV_TX * N] = T[0]; o[PV_TY * N] = T[1]; o[PV_TZ * N] = T[2];
        o[PV_ULJ * N] = ulj; o[PV_UQQ * N] = uqq; o[PV_UDD * N] = udd; o[PV_W * N] = w;
        o[PV_NP * N] = (float)np;
    }
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
    double fx = 0, fy = 0, fz = 0, u = 0, w = 0;
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
    u = warp_sum(u); w = warp_sum(w); np = warp_sum(np);
    if (lane == 0) {
        double *o = S.part64 + (size_t)p * MS2_NPV * N + i;
        o[PV_FX * N] = fx; o[PV_FY * N] = fy; o[PV_FZ * N] = fz;
        o[PV_TX * N] = 0; o[PV_TY * N] = 0; o[PV_TZ * N] = 0;
        o[PV_ULJ * N] = u; o[PV_UQQ * N] = 0; o[PV_UDD * N] = 0; o[PV_W * N] = w;
        o[PV_NP * N] = (double)np;
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
};

#define V(NS, LJM, QM, DM, E, M) {NS, LJM, QM, DM, E, M, &k_pair<NS, LJM, QM, DM, E, M>}
static const PairVariant kVariants[] = {
    V(1, 1u, 0u, 0u, ELEC_NONE, false),      // point LJ
    V(3, 1u, 7u, 0u, ELEC_RF, false),        // 3-site water, reaction field
    V(3, 1u, 7u, 0u, ELEC_EWALD, false),     // 3-site water, Ewald
    V(3, 1u, 7u, 0u, ELEC_EWALD, true),      // water + single-site ions, Ewald
    V(3, 3u, 0u, 4u, ELEC_RF, false),        // 2 LJ + dipole (Stockmayer-like)
};
#undef V

// generic fallbacks: runtime electrostatics, all slots may carry everything
static void (*const kGeneric[2][2])(const SysParams *, DevSys, int) = {
    {&k_pair<4, 0xFu, 0xFu, 0u, -1, true>, &k_pair<4, 0xFu, 0xFu, 0xFu, -1, true>},
    {&k_pair<8, 0xFFu, 0xFFu, 0u, -1, true>, &k_pair<8, 0xFFu, 0xFFu, 0xFFu, -1, true>},
};

// Picks the kernel for a system's slot pattern.  Returns the padded slot count
// the kernel expects in *ns_used (the site arrays must be laid out with it).
void *ms2_pick_pair_kernel(int ns, unsigned ljm, unsigned qm, unsigned dm, int elec, bool multi, int *ns_used,
                           bool *dmu, bool *mult_used) {
    for (const PairVariant &v : kVariants) {
        if (v.ns == ns && v.ljm == ljm && v.qm == qm && v.dm == dm && v.elec == elec && v.multi == multi) {
            *ns_used = ns;
            *dmu = dm != 0;
            *mult_used = multi;
            return (void *)v.fn;
        }
        // a single-species system can use the multi-species variant of its pattern
        if (v.ns == ns && v.ljm == ljm && v.qm == qm && v.dm == dm && v.elec == elec && v.multi && !multi) {
            bool exact_single = false;
            for (const PairVariant &u : kVariants)
                if (u.ns == ns && u.ljm == ljm && u.qm == qm && u.dm == dm && u.elec == elec && !u.multi)
                    exact_single = true;
            if (!exact_single) {
                *ns_used = ns;
                *dmu = dm != 0;
                *mult_used = true;
                return (void *)v.fn;
            }
        }
    }
    const int g = ns <= 4 ? 0 : 1;
    *ns_used = g ? 8 : 4;
    *dmu = dm != 0;
    *mult_used = true;
    return (void *)kGeneric[g][dm != 0];
}
