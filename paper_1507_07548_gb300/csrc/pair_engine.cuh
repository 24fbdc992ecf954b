// Per-warp pair engine shared by the single-system pair kernel and the batched
// per-system kernel: one warp owns molecule i, scans a shared-memory tile of
// candidates j on the integer centre lattice, compacts partners with a ballot
// into a per-warp queue and evaluates full batches of 32 partners one per lane
// with all site pairs unrolled (FP32 site math, coefficient products as hi+lo
// floats, bare Coulomb + molecular-dipole term for the reaction field, the
// molecular virial as the owner share).  See k_pair.cu for the method.
#pragma once
#include "ms2_internal.cuh"
#include "dfloat.cuh"

namespace pair_engine {

constexpr unsigned FULL = 0xffffffffu;
// partner queue of a warp: a ring of QCAP tile slots (the scan adds up to 64
// partners to fewer than 32 waiting ones)
constexpr int QCAP = 128;
// close-contact queue of a warp: a ring of CQCAP entries (tile slot, owner site,
// partner site) after the partner ring; QSTRIDE ints per warp in all
constexpr int CQCAP = 64;
constexpr int QSTRIDE = QCAP + CQCAP;

// Tile arrays: tP[j] = (lattice centre X, Y, Z, species) of tile molecule j
// (one 16-byte load), site offsets ts[(k NS + b) TJ + j], the point dipoles of
// the ND dipole slots tmu[(k ND + d) TJ + j] (d: the slot's rank among them) and,
// for the reaction field with point charges (MD), molecular dipoles tmd[k TJ + j].
// A tile layout is coded as ND + 256 MD.
struct Smem {
    uint4 *tP;
    float *ts, *tmu, *tmd;
    int *queue;
    float *sq, *sql, *sc6, *sc12, *sc6l, *sc12l;
    int *sljt;
};

__host__ __device__ constexpr int popc_c(unsigned x) { return x ? (int)(x & 1u) + popc_c(x >> 1) : 0; }
// rank of slot b among the dipole slots of mask DM
__host__ __device__ constexpr int dip_rank(unsigned DM, int b) { return popc_c(DM & ((1u << b) - 1u)); }
__host__ __device__ constexpr int tile_code(int nd, bool md) { return nd + (md ? 256 : 0); }

// tile arrays of TJ molecules, the per-warp queues and the parameter tables
template <int NS, int TILE, bool MULTI>
__device__ __forceinline__ Smem carve(unsigned char *base, int TJ, int wpb) {
    constexpr int ND = TILE & 255;
    constexpr bool MD = (TILE >> 8) != 0;
    Smem m;
    m.tP = (uint4 *)base;
    m.ts = (float *)(m.tP + TJ);
    m.tmu = m.ts + 3 * NS * TJ;
    m.tmd = m.tmu + 3 * ND * TJ;
    m.queue = (int *)(m.tmd + (MD ? 3 * TJ : 0));
    m.sq = (float *)(m.queue + wpb * QSTRIDE);
    m.sql = m.sq + MS2_MAXSP * MS2_MAXS;
    m.sljt = (int *)(m.sql + MS2_MAXSP * MS2_MAXS);
    m.sc6 = (float *)(m.sljt + MS2_MAXSP * MS2_MAXS);
    m.sc12 = m.sc6 + MS2_MAXT * MS2_MAXT;
    m.sc6l = m.sc12 + MS2_MAXT * MS2_MAXT;
    m.sc12l = m.sc6l + MS2_MAXT * MS2_MAXT;
    return m;
}

// bytes of carve's arrays (tile: the layout code ND + 256 MD)
__host__ __device__ inline size_t smem_bytes(int NS, int tile, bool multi, int TJ, int wpb) {
    (void)multi;
    const int nd = tile & 255;
    const bool md = (tile >> 8) != 0;
    size_t n = sizeof(uint4) * TJ + sizeof(float) * 3 * NS * TJ;
    n += sizeof(float) * 3 * nd * TJ;
    if (md) n += sizeof(float) * 3 * TJ;
    n += sizeof(int) * wpb * QSTRIDE;
    n += 2 * sizeof(float) * MS2_MAXSP * MS2_MAXS + sizeof(int) * MS2_MAXSP * MS2_MAXS;
    n += 4 * sizeof(float) * MS2_MAXT * MS2_MAXT;
    return n;
}

// block-level: tables of several species into shared memory
template <bool MULTI>
__device__ __forceinline__ void load_tables(const SysParams *__restrict__ P, const Smem &sm) {
    if constexpr (MULTI) {
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
}

// block-level: molecules [t0, t0+tn) of S into tile slots [0, tn); DM: the
// dipole slots of the kernel, MD: molecular dipoles kept (read when rfq)
template <int NS, unsigned DM, bool MD, bool MULTI>
__device__ __forceinline__ void stage_tile(const Smem &sm, const DevSys &S, int t0, int tn, int TJ, bool rfq) {
    constexpr int ND = popc_c(DM);
    const int N = S.N;
    for (int k = threadIdx.x; k < tn; k += blockDim.x) {
        const int j = t0 + k;
        // L2 loads (the data may come from another block of the same persistent kernel)
        sm.tP[k] = make_uint4(__ldcg(S.X + j), __ldcg(S.X + N + j), __ldcg(S.X + 2 * N + j),
                              MULTI ? (uint32_t)S.species[j] : 0u);
#pragma unroll
        for (int c = 0; c < 3 * NS; ++c) sm.ts[c * TJ + k] = __ldcg(S.s + c * N + j);
        if constexpr (ND > 0) {
#pragma unroll
            for (int b = 0; b < NS; ++b)
                if ((DM >> b) & 1u)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        sm.tmu[(c * ND + dip_rank(DM, b)) * TJ + k] = __ldcg(S.mu + (c * NS + b) * N + j);
        }
        if (MD && rfq) {
            sm.tmd[k] = __ldcg(S.mum + j);
            sm.tmd[TJ + k] = __ldcg(S.mum + N + j);
            sm.tmd[2 * TJ + k] = __ldcg(S.mum + 2 * N + j);
        }
    }
}

// the tile arrays seen from slot t0 on (same stride): a j-range inside a tile
// that holds the whole system
__device__ __forceinline__ Smem shifted(const Smem &m, int t0) {
    Smem v = m;
    v.tP += t0;
    v.ts += t0;
    v.tmu += t0;
    v.tmd += t0;
    return v;
}

// Site-site RDF counts (Sec. 3, Eq. 2) of tile molecule i against tile molecules
// j = j0, j0 + jstep, ... < n (the caller picks j > i so that every pair counts
// once): LJ-site kinds, site positions on the integer lattice (site minimum
// image), bins of width 1/inv_dr below r_max; integer shared-memory atomics.
template <int NS, bool MULTI>
__device__ __forceinline__ void rdf_molecule(const SysParams *__restrict__ P, const DevSys &S, const Smem &sm, int TJ,
                                             int i, int j0, int jstep, int n, unsigned *hist) {
    const int nb = S.rdf_bins, T = P->n_ljt;
    const float l2l = P->lat_to_len, l2 = P->len_to_lat;
    const float rmax2 = S.rdf_rmax2, inv_dr = S.rdf_inv_dr;
    auto coord = [&](int m, int c) { const uint4 p = sm.tP[m]; return c == 0 ? p.x : (c == 1 ? p.y : p.z); };
    const int spi = MULTI ? (int)sm.tP[i].w : 0;
    for (int a = 0; a < NS; ++a) {
        const int ta = S.rdf_kind[spi * MS2_MAXS + a];
        if (ta < 0) continue;
        uint32_t Xa[3];
        for (int c = 0; c < 3; ++c) Xa[c] = coord(i, c) + (uint32_t)__float2int_rn(sm.ts[(c * NS + a) * TJ + i] * l2);
        for (int j = j0; j < n; j += jstep) {
            const int spj = MULTI ? (int)sm.tP[j].w : 0;
            for (int b = 0; b < NS; ++b) {
                const int tb = S.rdf_kind[spj * MS2_MAXS + b];
                if (tb < 0) continue;
                float r2 = 0.f;
                for (int c = 0; c < 3; ++c) {
                    const uint32_t Xb = coord(j, c) + (uint32_t)__float2int_rn(sm.ts[(c * NS + b) * TJ + j] * l2);
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

// result of one molecule (valid in lane 0): F, tau, U_lj, U_qq, U_dd, W,
// the second-volume-derivative sum vv (MASS) and the partner count
struct PairOut {
    float F[3], T[3], ulj, uqq, udd, w, vv;
    int np;
};

// NS: site slots per molecule; LJM/QM/DM: slot bit masks that may carry LJ,
// charge, dipole; ELEC: ELEC_NONE/RF/EWALD or -1 = read from the parameters;
// MULTI: several species (per-molecule parameter lookup); MASS: also the
// second volume derivative of U for the Massieu derivatives (Sec. 2, Eq. 1):
// per site pair h (r.d)^2 + g (d^2 - 2 r.d), with g = u'(r)/r and
// h = (u''(r) - g)/r^2, whose owner sums over partners, halved and divided by
// 9 V^2, give d2U/dV2 at fixed scaled centres (LJ and bare Coulomb; the
// reaction-field k_RF and c_RF terms drop out of neutral molecule pairs).
template <int NS, unsigned LJM, unsigned QM, unsigned DM, int ELEC, bool MULTI, bool MASS = false>
struct PairWarp {
    static_assert(!MASS || (DM == 0 && ELEC != ELEC_EWALD), "volume derivatives: LJ and point charges, no Ewald");
    static constexpr bool DMU = DM != 0;
    static constexpr bool MOLD = QM != 0 && (ELEC == ELEC_RF || ELEC < 0);  // molecular-dipole RF term
    static constexpr int ND = popc_c(DM);                 // dipole slots kept in the tile
    static constexpr int TILE = tile_code(ND, MOLD);      // the tile layout of this variant
    // First site PA of an adjacent pair (PA, PA + 1) that meets every partner site
    // with the same kinds of term (LJ and/or charge, no point dipole), or -1.  In
    // the force pass of a single-species LJ / reaction-field kernel the two rows of
    // site pairs are evaluated together in packed FP32x2 arithmetic (PKF).
    static constexpr int pair_site() {
        for (int a = 0; a + 1 < NS; ++a) {
            const unsigned l0 = (LJM >> a) & 1u, l1 = (LJM >> (a + 1)) & 1u;
            const unsigned q0 = (QM >> a) & 1u, q1 = (QM >> (a + 1)) & 1u;
            const unsigned d0 = (DM >> a) & 1u, d1 = (DM >> (a + 1)) & 1u;
            if (l0 == l1 && q0 == q1 && !d0 && !d1 && (l0 || q0)) return a;
        }
        return -1;
    }
    static constexpr int PA = pair_site(), PB = PA + 1;
    static constexpr bool PKF = PA >= 0 && !MULTI && !MASS && (ELEC == ELEC_RF || ELEC == ELEC_NONE);
    // close-contact LJ site pairs in double-float (not in the heat-flux power
    // pass): compiled where a slot may carry a charge, the systems the host
    // switches it on for (SysParams::close_k6)
    static constexpr bool CLOSE = LJM != 0 && QM != 0;
    int elec;
    bool rfq;
    float C, krf, alpha, tasp, tasp_lo, l2l, l2l_lo, ck6;
    unsigned long long rc2;
    // coefficient tables of a single-species system (hi + lo floats: a single
    // FP32 rounding of C q_a q_b or 4 eps sigma^12 would scale every term of that
    // site-pair kind the same way and bias the strongly cancelling sums)
    float hq[NS][NS], hql[NS][NS], hc6[NS][NS], hc12[NS][NS], hc6l[NS][NS], hc12l[NS][NS];
    // molecule i
    int i, spi;
    uint32_t Xi, Yi, Zi;
    float si[NS][3], mui[NS][3], qih[NS], qil[NS], mdi[3];
    int ljti[NS];
    // the packed pair (PKF): offsets (s_PA, s_PB) per component, coefficients
    // (PA, b), (PB, b) per partner site b, and the lane sums of the NEGATED site
    // forces (-f_PA, -f_PB) per component (no sign flips in the packed terms)
    float2 sp2[3], pq[NS], pql[NS], pc6[NS], pc12[NS], pc6l[NS], pc12l[NS], fp[3];
    // lane accumulators
    float fa[NS][3], ea[NS][3], ulj, uqq, udd, w, vv, erf_[3];
    int np;
    // close-contact sums (double-float energy and virial) and the close ring state
    dfl::df ucl, wcl;
    int cqh, cqn;
    // heat-flux power pass (HP): site velocities v_i + w_i x s_ia, w_i x mu_ia,
    // w_i x mu_i (reaction field) and the lane sums of d_kl P_kl
    float vs[NS][3], wmu[NS][3], wmd[3], jh[3];

    __device__ __forceinline__ void setup(const SysParams *__restrict__ P) {
        elec = ELEC >= 0 ? ELEC : P->elec;
        rfq = MOLD && P->elec == ELEC_RF;
        C = P->coulomb;
        krf = P->krf;
        alpha = P->alpha;
        tasp = P->two_alpha_sqrtpi;
        l2l = P->lat_to_len;
        l2l_lo = P->lat_to_len_lo;
        ck6 = P->close_k6;
        tasp_lo = P->two_alpha_sqrtpi_lo;
        rc2 = P->rc2;
        if (!MULTI) {
#pragma unroll
            for (int a = 0; a < NS; ++a)
#pragma unroll
                for (int b = 0; b < NS; ++b) {
                    const float qa = P->cq[0][a], qal = P->cqlo[0][a];
                    const float qb = P->q[0][b], qbl = P->qlo[0][b];
                    hq[a][b] = qa * qb;
                    hql[a][b] = fmaf(qa, qb, -hq[a][b]) + fmaf(qa, qbl, qal * qb);
                    const int ta = P->ljt[0][a], tb = P->ljt[0][b];
                    const bool on = ta >= 0 && tb >= 0;
                    const int ia = on ? ta : 0, ib = on ? tb : 0;
                    hc6[a][b] = on ? P->c6[ia][ib] : 0.f;
                    hc12[a][b] = on ? P->c12[ia][ib] : 0.f;
                    hc6l[a][b] = on ? P->c6lo[ia][ib] : 0.f;
                    hc12l[a][b] = on ? P->c12lo[ia][ib] : 0.f;
                }
            if constexpr (PKF) {
#pragma unroll
                for (int b = 0; b < NS; ++b) {
                    pq[b] = make_float2(hq[PA][b], hq[PB][b]);
                    pql[b] = make_float2(hql[PA][b], hql[PB][b]);
                    pc6[b] = make_float2(hc6[PA][b], hc6[PB][b]);
                    pc12[b] = make_float2(hc12[PA][b], hc12[PB][b]);
                    pc6l[b] = make_float2(hc6l[PA][b], hc6l[PB][b]);
                    pc12l[b] = make_float2(hc12l[PA][b], hc12l[PB][b]);
                }
            }
        }
    }

    // molecule i of S (all lanes of the warp)
    __device__ __forceinline__ void begin(const SysParams *__restrict__ P, const DevSys &S, int i_) {
        const int N = S.N;
        i = i_;
        Xi = S.X[i];
        Yi = S.X[N + i];
        Zi = S.X[2 * N + i];
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                si[a][k] = S.s[(k * NS + a) * N + i];
                mui[a][k] = DMU && ((DM >> a) & 1) ? S.mu[(k * NS + a) * N + i] : 0.f;
            }
        spi = MULTI ? S.species[i] : 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) mdi[k] = (MOLD && rfq) ? S.mum[k * N + i] : 0.f;
        begin_common(P);
    }

    // molecule i from a tile that holds the whole system with stride TJ
    __device__ __forceinline__ void begin_tile(const SysParams *__restrict__ P, const Smem &sm, int TJ, int i_) {
        i = i_;
        const uint4 p = sm.tP[i];
        Xi = p.x;
        Yi = p.y;
        Zi = p.z;
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                si[a][k] = sm.ts[(k * NS + a) * TJ + i];
                mui[a][k] = DMU && ((DM >> a) & 1) ? sm.tmu[(k * ND + dip_rank(DM, a)) * TJ + i] : 0.f;
            }
        spi = MULTI ? (int)p.w : 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) mdi[k] = (MOLD && rfq) ? sm.tmd[k * TJ + i] : 0.f;
        begin_common(P);
    }

    __device__ __forceinline__ void begin_common(const SysParams *__restrict__ P) {
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            ljti[a] = P->ljt[spi][a];
            qih[a] = P->cq[spi][a];  // (C q_a) as hi + lo, from FP64
            qil[a] = P->cqlo[spi][a];
        }
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) fa[a][k] = ea[a][k] = 0.f;
        if constexpr (PKF) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                sp2[k] = make_float2(si[PA][k], si[PB][k]);
                fp[k] = make_float2(0.f, 0.f);
            }
        }
        ulj = uqq = udd = w = vv = 0.f;
        erf_[0] = erf_[1] = erf_[2] = 0.f;
        np = 0;
        ucl = wcl = dfl::df{0.f, 0.f};
        cqh = cqn = 0;
    }

    // Heat-flux power pass (Sec. 4, Eqs. 5-6) of molecule i, after begin or
    // begin_tile: v and w are its velocity and angular velocity.  The pass sums,
    // over partners l, d_kl P_kl with P_kl = F_kl.v_k + tau_kl.w_k, taken per site
    // as sum_a f_a.(v + w x s_a) + e_a.(w x mu_a) (the dipole torque mu_a x e_a)
    // + 2 C k_RF mu_l.(w x mu_i) (the reaction-field molecular torque); the site
    // forces are those of the force pass, term for term.
    __device__ __forceinline__ void begin_heat(const float v[3], const float wv[3]) {
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            vs[a][0] = v[0] + (wv[1] * si[a][2] - wv[2] * si[a][1]);
            vs[a][1] = v[1] + (wv[2] * si[a][0] - wv[0] * si[a][2]);
            vs[a][2] = v[2] + (wv[0] * si[a][1] - wv[1] * si[a][0]);
            wmu[a][0] = wv[1] * mui[a][2] - wv[2] * mui[a][1];
            wmu[a][1] = wv[2] * mui[a][0] - wv[0] * mui[a][2];
            wmu[a][2] = wv[0] * mui[a][1] - wv[1] * mui[a][0];
        }
        wmd[0] = wv[1] * mdi[2] - wv[2] * mdi[1];
        wmd[1] = wv[2] * mdi[0] - wv[0] * mdi[2];
        wmd[2] = wv[0] * mdi[1] - wv[1] * mdi[0];
        jh[0] = jh[1] = jh[2] = 0.f;
    }

    // one partner, tile-local index jl, into this lane's accumulators (HP: the
    // heat-flux power pass; the force-pass accumulators are then dead).  Returns
    // the LJ site pairs (bit a NS + b) at close contact, whose LJ terms are left
    // out here and evaluated in double-float by close_pair.
    template <bool HP = false>
    __device__ __forceinline__ unsigned long long interact(const Smem &sm, int TJ, int jl) {
    unsigned long long cmask = 0ull;
    const uint4 pjl = sm.tP[jl];
    const int dxi = (int)(pjl.x - Xi), dyi = (int)(pjl.y - Yi), dzi = (int)(pjl.z - Zi);
    // lattice difference -> length with the scale split in two floats, so the
    // FP32 rounding of L/2^32 does not scale every displacement the same way
    const float fxi = (float)dxi, fyi = (float)dyi, fzi = (float)dzi;
    const float dx = fmaf(fxi, l2l, fxi * l2l_lo), dy = fmaf(fyi, l2l, fyi * l2l_lo),
                dz = fmaf(fzi, l2l, fzi * l2l_lo);
    const int spj = MULTI ? (int)pjl.w : 0;
    float pj[NS][3], muj[NS][3];
#pragma unroll
    for (int b = 0; b < NS; ++b) {
        pj[b][0] = dx + sm.ts[(0 * NS + b) * TJ + jl];
        pj[b][1] = dy + sm.ts[(1 * NS + b) * TJ + jl];
        pj[b][2] = dz + sm.ts[(2 * NS + b) * TJ + jl];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            muj[b][k] = DMU && ((DM >> b) & 1) ? sm.tmu[(k * ND + dip_rank(DM, b)) * TJ + jl] : 0.f;
    }
    // Molecular virial, owner share: the site-pair part -sum_ab f_ab.r_ab here
    // (short levers, no FP32 force sum meets the long lever d), the
    // intramolecular part -2 sum_a s_ia.F_ia once per molecule in finish().
    float wsite = 0.f, wvv = 0.f, pw = 0.f;  // pw: the power P_kl (HP)
    const float dd2 = MASS ? dx * dx + dy * dy + dz * dz : 0.f;
    constexpr bool PK = PKF && !HP;
#pragma unroll
    for (int a = 0; a < NS; ++a) {
        if (PK && a == PB) continue;
        if (PK && a == PA) {
            // rows PA and PB together (FP32x2, lane .x = PA, .y = PB): the scalar
            // operations below term by term, the force factor negated; row PB's
            // energy and virial terms are added after row PA's, in partner-site order
            const float2 m1 = make_float2(-1.f, -1.f);
            float dl[NS], dq[NS], dgv[NS];
#pragma unroll
            for (int b = 0; b < NS; ++b) {
                const bool mlj = (LJM >> PA) & (LJM >> b) & 1u;
                const bool mq = ((QM >> PA) & (QM >> b) & 1u) && elec != ELEC_NONE;
                if (!(mlj || mq)) continue;
                const float2 rx = __ffma2_rn(sp2[0], m1, make_float2(pj[b][0], pj[b][0]));
                const float2 ry = __ffma2_rn(sp2[1], m1, make_float2(pj[b][1], pj[b][1]));
                const float2 rz = __ffma2_rn(sp2[2], m1, make_float2(pj[b][2], pj[b][2]));
                const float2 r2 = __ffma2_rn(rz, rz, __ffma2_rn(ry, ry, __fmul2_rn(rx, rx)));
                float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                const float2 nt = __fmul2_rn(__fmul2_rn(make_float2(-0.5f, -0.5f), r2), rinv);
                rinv = __ffma2_rn(rinv, __ffma2_rn(nt, rinv, make_float2(0.5f, 0.5f)), rinv);
                const float2 rinv2 = __fmul2_rn(rinv, rinv);
                float2 ng = make_float2(0.f, 0.f);  // -g
                if (mlj) {
                    const float2 r6 = __fmul2_rn(__fmul2_rn(rinv2, rinv2), rinv2), r12 = __fmul2_rn(r6, r6);
                    float2 t6 = __ffma2_rn(pc6[b], r6, __fmul2_rn(pc6l[b], r6));
                    float2 t12 = __ffma2_rn(pc12[b], r12, __fmul2_rn(pc12l[b], r12));
                    if constexpr (CLOSE && !HP) {
                        const bool c0 = t12.x > ck6 * t6.x, c1 = t12.y > ck6 * t6.y;
                        cmask |= ((unsigned long long)c0 << (PA * NS + b)) | ((unsigned long long)c1 << (PB * NS + b));
                        t6 = make_float2(c0 ? 0.f : t6.x, c1 ? 0.f : t6.y);
                        t12 = make_float2(c0 ? 0.f : t12.x, c1 ? 0.f : t12.y);
                    }
                    const float2 tl = __ffma2_rn(t6, m1, t12);
                    ulj += tl.x;
                    dl[b] = tl.y;
                    // virial term -g r^2 = 12 t12 - 6 t6 directly (no r^-2 r^2 round trip)
                    const float2 tw = __ffma2_rn(make_float2(12.f, 12.f), t12, __fmul2_rn(make_float2(-6.f, -6.f), t6));
                    ng = __fmul2_rn(tw, rinv2);
                    wsite += tw.x;
                    dgv[b] = tw.y;
                }
                if (mq) {  // bare Coulomb (reaction field)
                    const float2 eq = __ffma2_rn(pq[b], rinv, __fmul2_rn(pql[b], rinv));
                    uqq += eq.x;
                    dq[b] = eq.y;
                    const float2 ngq = __fmul2_rn(eq, rinv2);
                    ng = mlj ? __fadd2_rn(ng, ngq) : ngq;
                }
                fp[0] = __ffma2_rn(ng, rx, fp[0]);
                fp[1] = __ffma2_rn(ng, ry, fp[1]);
                fp[2] = __ffma2_rn(ng, rz, fp[2]);
            }
#pragma unroll
            for (int b = 0; b < NS; ++b) {
                const bool mlj = (LJM >> PA) & (LJM >> b) & 1u;
                const bool mq = ((QM >> PA) & (QM >> b) & 1u) && elec != ELEC_NONE;
                if (mlj) ulj += dl[b];
                if (mq) uqq += dq[b];
                if (mlj) wsite += dgv[b];
            }
            continue;
        }
#pragma unroll
        for (int b = 0; b < NS; ++b) {
            const bool mlj = (LJM >> a) & (LJM >> b) & 1u;
            const bool mq = (QM >> a) & (QM >> b) & 1u;
            const bool md = (DM >> a) & (DM >> b) & 1u;
            if (!(mlj || (mq && elec != ELEC_NONE) || (md && elec != ELEC_NONE))) continue;
            const float rx = pj[b][0] - si[a][0], ry = pj[b][1] - si[a][1], rz = pj[b][2] - si[a][2];
            // (explicit operation order, shared with the packed rows above)
            float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
            if (MULTI) r2 = fmaxf(r2, 1e-12f);
            // rsqrt approximation + one Newton step: unbiased to ~1 ulp
            float rinv = rsqrtf(r2);
            rinv = fmaf(rinv, fmaf(-0.5f * r2 * rinv, rinv, 0.5f), rinv);
            const float rinv2 = rinv * rinv;
            // g = u'/r of the site pair; wv the virial term -g r^2 of the parts
            // summed here, formed directly from the terms (bare reaction-field
            // Coulomb has -g r^2 = its energy term, summed as U_qq); hh = (u'' -
            // u'/r)/r^2 (MASS)
            float g = 0.f, wv = 0.f, hh = 0.f;
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
                float t6 = fmaf(c6, r6, c6l * r6), t12 = fmaf(c12, r12, c12l * r12);
                if (MASS) hh += (168.f * t12 - 48.f * t6) * (rinv2 * rinv2);
                if constexpr (CLOSE && !HP) {
                    const bool cl = t12 > ck6 * t6;
                    cmask |= (unsigned long long)cl << (a * NS + b);
                    t6 = cl ? 0.f : t6;
                    t12 = cl ? 0.f : t12;
                }
                ulj += t12 - t6;
                const float t6x = 6.f * t6;
                g = fmaf(-12.f, t12, t6x) * rinv2;
                wv = fmaf(12.f, t12, -t6x);
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
                float gq;
                if (elec == ELEC_RF) {  // bare Coulomb (the RF part is a molecular term): g = -E / r^2
                    const float eq = fmaf(cqq, rinv, cql * rinv);
                    uqq += eq;
                    gq = -eq * rinv2;
                } else {
                    // alpha is exact in FP32; 2 alpha / sqrt(pi) as hi + lo (one rounding of it
                    // would scale every exp term of the molecular virial the same way)
                    const float ar = alpha * r2 * rinv;
                    const float ec = erfcf(ar), ex = expf(-ar * ar);
                    const float bu = ec * rinv, bx = fmaf(tasp, ex, tasp_lo * ex), bg = -(bu + bx) * rinv2;
                    const float eu = fmaf(cqq, bu, cql * bu);
                    uqq += eu;
                    gq = fmaf(cqq, bg, cql * bg);
                    // -gq r^2 = C q q (erfc(a r)/r + 2a/sqrt(pi) exp(-a^2 r^2)), formed directly
                    wv += eu + fmaf(cqq, bx, cql * bx);
                }
                g = mlj ? g + gq : gq;
                if (MASS) hh -= 3.f * gq * rinv2;  // bare Coulomb: h = 3 C q q / r^5
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
                fa[a][0] += fx; fa[a][1] += fy; fa[a][2] += fz;
                wsite -= fx * rx + fy * ry + fz * rz;
                const float ce = 3.f * C * mbr * rinv5, cm = -C * (rinv3 - kd);
                const float ex = ce * rx + cm * muj[b][0], ey = ce * ry + cm * muj[b][1], ez = ce * rz + cm * muj[b][2];
                ea[a][0] += ex;
                ea[a][1] += ey;
                ea[a][2] += ez;
                if (HP) {
                    pw += fx * vs[a][0] + fy * vs[a][1] + fz * vs[a][2];
                    pw += ex * wmu[a][0] + ey * wmu[a][1] + ez * wmu[a][2];
                }
            }
            fa[a][0] = fmaf(g, rx, fa[a][0]); fa[a][1] = fmaf(g, ry, fa[a][1]); fa[a][2] = fmaf(g, rz, fa[a][2]);
            if (mlj || (mq && elec == ELEC_EWALD)) wsite += wv;
            if (HP) pw = fmaf(g, rx * vs[a][0] + ry * vs[a][1] + rz * vs[a][2], pw);
            if (MASS) {
                const float rd = rx * dx + ry * dy + rz * dz;
                wvv += fmaf(hh * rd, rd, g * (dd2 - 2.f * rd));
            }
        }
    }
    w += wsite;
    if (MASS) vv += wvv;
    if (MOLD && rfq) {
        erf_[0] += sm.tmd[jl];
        erf_[1] += sm.tmd[TJ + jl];
        erf_[2] += sm.tmd[2 * TJ + jl];
        if (HP) pw += 2.f * C * krf * (sm.tmd[jl] * wmd[0] + sm.tmd[TJ + jl] * wmd[1] + sm.tmd[2 * TJ + jl] * wmd[2]);
    }
    if (HP) {
        jh[0] = fmaf(dx, pw, jh[0]);
        jh[1] = fmaf(dy, pw, jh[1]);
        jh[2] = fmaf(dz, pw, jh[2]);
    }
    ++np;
    return cmask;
    }

    // Close-contact LJ site pair (owner site a, partner tile slot jl, site b) in
    // double-float: the centre difference exactly from the lattice, the site
    // offsets as stored, then r^2, r^-6, r^-12, the energy t12 - t6 and the
    // virial 12 t12 - 6 t6 with ~44-bit significands; the force on site a
    // (g r, g = -(12 t12 - 6 t6) / r^2) in FP32.
    __device__ __forceinline__ void close_pair(const Smem &sm, int TJ, int e) {
        using namespace dfl;
        const int jl = e & 0xFFFFFF, a = (e >> 24) & 15, b = (e >> 28) & 15;
        const uint4 pj = sm.tP[jl];
        const int dv[3] = {(int)(pj.x - Xi), (int)(pj.y - Yi), (int)(pj.z - Zi)};
        float sa[3] = {0.f, 0.f, 0.f}, c6h = 0.f, c6l = 0.f, c12h = 0.f, c12l = 0.f;
#pragma unroll
        for (int a2 = 0; a2 < NS; ++a2)
            if (a2 == a && ((LJM >> a2) & 1u)) {
#pragma unroll
                for (int k = 0; k < 3; ++k) sa[k] = si[a2][k];
            }
        if constexpr (MULTI) {
            const int spj = (int)pj.w, tb = sm.sljt[spj * MS2_MAXS + b];
            int ta = 0;
#pragma unroll
            for (int a2 = 0; a2 < NS; ++a2)
                if (a2 == a) ta = ljti[a2];
            const int idx = ta * MS2_MAXT + tb;
            c6h = sm.sc6[idx]; c6l = sm.sc6l[idx]; c12h = sm.sc12[idx]; c12l = sm.sc12l[idx];
        } else {
#pragma unroll
            for (int a2 = 0; a2 < NS; ++a2)
#pragma unroll
                for (int b2 = 0; b2 < NS; ++b2)
                    if (((LJM >> a2) & (LJM >> b2) & 1u) && a2 == a && b2 == b) {
                        c6h = hc6[a2][b2]; c6l = hc6l[a2][b2]; c12h = hc12[a2][b2]; c12l = hc12l[a2][b2];
                    }
        }
        // d = dv L / 2^32 exactly as hi + lo: dv = 256 hi + lo with both parts exact in FP32
        const float u256 = 256.f * l2l, u256l = 256.f * l2l_lo;
        df r[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int hi = dv[k] >> 8, lo = dv[k] & 255;
            const float fh = (float)hi, fl = (float)lo;
            df d = two_prod(fh, u256);
            d.l = __fmaf_rn(fh, u256l, d.l);
            d.l = __fmaf_rn(fl, l2l, d.l);
            d.l = __fmaf_rn(fl, l2l_lo, d.l);
            const float sb = sm.ts[(k * NS + b) * TJ + jl];
            r[k] = add(d, two_sum(sb, -sa[k]));
        }
        df r2 = add(add(sqr(r[0]), sqr(r[1])), sqr(r[2]));
        if (MULTI && r2.h < 1e-12f) r2 = df{1e-12f, 0.f};
        const df x = rcp(r2), x3 = mul(sqr(x), x);
        const df t6 = mul(df{c6h, c6l}, x3), t12 = mul(df{c12h, c12l}, sqr(x3));
        const df u = add(t12, neg(t6)), wv = add(mul_f(t12, 12.f), neg(mul_f(t6, 6.f)));
        ucl = add(ucl, u);
        wcl = add(wcl, wv);
        const float g = -__fmul_rn(__fadd_rn(wv.h, wv.l), x.h);
        if constexpr (MASS) {  // the g (d^2 - 2 r.d) part of the volume second derivative
            float dd = 0.f, rd = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float dk = __fsub_rn(r[k].h, __fsub_rn(sm.ts[(k * NS + b) * TJ + jl], sa[k]));
                dd = fmaf(dk, dk, dd);
                rd = fmaf(r[k].h, dk, rd);
            }
            vv = fmaf(g, dd - 2.f * rd, vv);
        }
#pragma unroll
        for (int a2 = 0; a2 < NS; ++a2)
            if (((LJM >> a2) & 1u) && a2 == a) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float f = __fmul_rn(g, r[k].h);
                    if constexpr (PKF) {
                        if (a2 == PA) { fp[k].x = __fsub_rn(fp[k].x, f); continue; }
                        if (a2 == PB) { fp[k].y = __fsub_rn(fp[k].y, f); continue; }
                    }
                    fa[a2][k] = __fadd_rn(fa[a2][k], f);
                }
            }
    }

    // the close LJ site pairs of one evaluated batch (cm from interact; lane
    // order, then site-pair order) into the ring cq; 32 at a time evaluated
    __device__ __forceinline__ void push_close(const Smem &sm, int TJ, unsigned long long cm, int jl, int lane, int *cq) {
        const unsigned below = (1u << lane) - 1u;
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
            for (int b = 0; b < NS; ++b) {
                if (!((LJM >> a) & (LJM >> b) & 1u)) continue;
                const bool c = (cm >> (a * NS + b)) & 1ull;
                const unsigned m = __ballot_sync(FULL, c);
                if (m == 0u) continue;
                if (c) cq[(cqh + cqn + __popc(m & below)) & (CQCAP - 1)] = jl | (a << 24) | (b << 28);
                cqn += __popc(m);
                __syncwarp();
                while (cqn >= 32) {
                    close_pair(sm, TJ, cq[(cqh + lane) & (CQCAP - 1)]);
                    __syncwarp();
                    cqh = (cqh + 32) & (CQCAP - 1);
                    cqn -= 32;
                }
            }
    }

    __device__ __forceinline__ void drain_close(const Smem &sm, int TJ, int lane, int *cq) {
        if (cqn > 0) {
            if (lane < cqn) close_pair(sm, TJ, cq[(cqh + lane) & (CQCAP - 1)]);
            __syncwarp();
            cqh = cqn = 0;
        }
    }

    // one full batch of 32 waiting partners at ring position head
    template <bool HP>
    __device__ __forceinline__ void run_batch(const Smem &sm, int TJ, const int *wq, int head, int lane) {
        const int jl = wq[(head + lane) & (QCAP - 1)];
        const unsigned long long cm = interact<HP>(sm, TJ, jl);
        __syncwarp();  // the batch is read before later passes overwrite its slots
        if constexpr (CLOSE && !HP) push_close(sm, TJ, cm, jl, lane, const_cast<int *>(wq) + QCAP);
    }

    // the last qn < 32 waiting partners, then the remaining close pairs
    template <bool HP>
    __device__ __forceinline__ void run_tail(const Smem &sm, int TJ, const int *wq, int head, int qn, int lane) {
        int jl = 0;
        unsigned long long cm = 0ull;
        if (lane < qn) {
            jl = wq[(head + lane) & (QCAP - 1)];
            cm = interact<HP>(sm, TJ, jl);
        }
        __syncwarp();
        if constexpr (CLOSE && !HP) {
            int *cq = const_cast<int *>(wq) + QCAP;
            push_close(sm, TJ, cm, jl, lane, cq);
            drain_close(sm, TJ, lane, cq);
        }
    }

    // scan tile slots [0, tn) (global index of slot 0: t0), partners in batches of 32.
    // Two groups of 32 candidates are tested per pass (independent chains); the
    // partners enter the ring queue wq in ascending slot order, so the batches are
    // those of a scan 32 at a time.
    template <bool HP = false>
    __device__ __forceinline__ void scan(const Smem &sm, int TJ, int t0, int tn, int *wq, int lane) {
        const unsigned below = (1u << lane) - 1u;
        const int il = i - t0;  // the owner's own slot (may lie outside the range)
        // branch-free test: a slot past the range reads the last one and is masked
        auto partner = [&](int jl) {
            const int js = min(jl, tn - 1);
            const uint4 p = sm.tP[js];
            const int dx = (int)(p.x - Xi), dy = (int)(p.y - Yi), dz = (int)(p.z - Zi);
            return (jl < tn) & (jl != il) & (lattice_d2(dx, dy, dz) < rc2);
        };
        int head = 0, qn = 0;  // first waiting partner in the ring, number waiting
        for (int base = 0; base < tn; base += 64) {
            const int j0 = base + lane, j1 = base + 32 + lane;
            const bool p0 = partner(j0), p1 = partner(j1);
            const unsigned m0 = __ballot_sync(FULL, p0), m1 = __ballot_sync(FULL, p1);
            const int n0 = __popc(m0);
            if (p0) wq[(head + qn + __popc(m0 & below)) & (QCAP - 1)] = j0;
            if (p1) wq[(head + qn + n0 + __popc(m1 & below)) & (QCAP - 1)] = j1;
            qn += n0 + __popc(m1);
            __syncwarp();
            while (qn >= 32) {
                run_batch<HP>(sm, TJ, wq, head, lane);
                head = (head + 32) & (QCAP - 1);
                qn -= 32;
            }
        }
        run_tail<HP>(sm, TJ, wq, head, qn, lane);
    }

    // The full scan of a whole-system tile (slots [0, tn)) that also lists, in
    // ascending slot order, the candidates within the list radius (lattice
    // rs2 >= rc2) into nl[0, lcap); returns how many there are (> lcap: the list
    // is incomplete).  The partners and their batches are those of scan().
    __device__ __forceinline__ int scan_build(const Smem &sm, int TJ, int tn, int *wq, int lane, uint16_t *nl,
                                              int lcap, unsigned long long rs2) {
        const unsigned below = (1u << lane) - 1u;
        auto test = [&](int jl, bool &listed) {
            const int js = min(jl, tn - 1);
            const uint4 p = sm.tP[js];
            const int dx = (int)(p.x - Xi), dy = (int)(p.y - Yi), dz = (int)(p.z - Zi);
            const unsigned long long d2 = lattice_d2(dx, dy, dz);
            const bool in = (jl < tn) & (jl != i);
            listed = in & (d2 < rs2);
            return in & (d2 < rc2);
        };
        int head = 0, qn = 0, nc = 0;
        for (int base = 0; base < tn; base += 64) {
            const int j0 = base + lane, j1 = base + 32 + lane;
            bool l0, l1;
            const bool p0 = test(j0, l0), p1 = test(j1, l1);
            const unsigned a0 = __ballot_sync(FULL, l0), a1 = __ballot_sync(FULL, l1);
            const int c0 = nc + __popc(a0 & below), c1 = nc + __popc(a0) + __popc(a1 & below);
            if (l0 && c0 < lcap) nl[c0] = (uint16_t)j0;
            if (l1 && c1 < lcap) nl[c1] = (uint16_t)j1;
            nc += __popc(a0) + __popc(a1);
            const unsigned m0 = __ballot_sync(FULL, p0), m1 = __ballot_sync(FULL, p1);
            const int n0 = __popc(m0);
            if (p0) wq[(head + qn + __popc(m0 & below)) & (QCAP - 1)] = j0;
            if (p1) wq[(head + qn + n0 + __popc(m1 & below)) & (QCAP - 1)] = j1;
            qn += n0 + __popc(m1);
            __syncwarp();
            while (qn >= 32) {
                run_batch<false>(sm, TJ, wq, head, lane);
                head = (head + 32) & (QCAP - 1);
                qn -= 32;
            }
        }
        run_tail<false>(sm, TJ, wq, head, qn, lane);
        return nc;
    }

    // The scan of a complete candidate list nl[0, cnt) (ascending slots of a
    // whole-system tile, the owner excluded): the exact centre test on each, the
    // partners in the order and batches of scan().
    __device__ __forceinline__ void scan_list(const Smem &sm, int TJ, const uint16_t *nl, int cnt, int *wq, int lane) {
        const unsigned below = (1u << lane) - 1u;
        auto test = [&](int k, int jl) {
            const uint4 p = sm.tP[jl];
            const int dx = (int)(p.x - Xi), dy = (int)(p.y - Yi), dz = (int)(p.z - Zi);
            return (k < cnt) & (lattice_d2(dx, dy, dz) < rc2);
        };
        // the list entries of the next pass are loaded while this pass runs
        const int last = cnt - 1;
        int n0 = cnt > 0 ? __ldcg(nl + min(lane, last)) : 0, n1 = cnt > 0 ? __ldcg(nl + min(lane + 32, last)) : 0;
        int head = 0, qn = 0;
        for (int base = 0; base < cnt; base += 64) {
            const int j0 = n0, j1 = n1;
            if (base + 64 < cnt) {
                n0 = __ldcg(nl + min(base + 64 + lane, last));
                n1 = __ldcg(nl + min(base + 96 + lane, last));
            }
            const bool p0 = test(base + lane, j0), p1 = test(base + 32 + lane, j1);
            const unsigned m0 = __ballot_sync(FULL, p0), m1 = __ballot_sync(FULL, p1);
            const int n0 = __popc(m0);
            if (p0) wq[(head + qn + __popc(m0 & below)) & (QCAP - 1)] = j0;
            if (p1) wq[(head + qn + n0 + __popc(m1 & below)) & (QCAP - 1)] = j1;
            qn += n0 + __popc(m1);
            __syncwarp();
            while (qn >= 32) {
                run_batch<false>(sm, TJ, wq, head, lane);
                head = (head + 32) & (QCAP - 1);
                qn -= 32;
            }
        }
        run_tail<false>(sm, TJ, wq, head, qn, lane);
    }

    // heat pass: the warp's sum_l d_kl P_kl (fixed tree, every lane)
    __device__ __forceinline__ void finish_heat(float out[3]) {
#pragma unroll
        for (int k = 0; k < 3; ++k) out[k] = warp_sum(jh[k]);
    }

    // fixed-tree warp reduction; the result is valid in lane 0
    __device__ __forceinline__ PairOut finish(int lane) {
        if constexpr (PKF) {  // the packed rows' negated sums
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                fa[PA][k] = 0.f - fp[k].x;
                fa[PB][k] = 0.f - fp[k].y;
            }
        }
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
        PairOut o;
        o.ulj = warp_sum(ulj);
        o.uqq = warp_sum(uqq);
        o.udd = warp_sum(udd);
        o.w = warp_sum(w);
        if constexpr (CLOSE) {  // the double-float close-contact sums (fixed xor tree), one rounding each
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) {
                ucl = dfl::add(ucl, dfl::df{__shfl_xor_sync(FULL, ucl.h, s), __shfl_xor_sync(FULL, ucl.l, s)});
                wcl = dfl::add(wcl, dfl::df{__shfl_xor_sync(FULL, wcl.h, s), __shfl_xor_sync(FULL, wcl.l, s)});
            }
            o.ulj = dfl::add(dfl::df{o.ulj, 0.f}, ucl).h;
            o.w = dfl::add(dfl::df{o.w, 0.f}, wcl).h;
        }
        if (elec == ELEC_RF) o.w += o.uqq;  // the bare-Coulomb site virials (before the molecular RF term)
        o.vv = MASS ? warp_sum(vv) : 0.f;
        o.np = warp_sum(np);
        o.F[0] = o.F[1] = o.F[2] = o.T[0] = o.T[1] = o.T[2] = 0.f;
        if (lane == 0) {
            // intramolecular part of the owner virial share: -2 sum_a s_ia.F_ia
            // (linear in the site forces, so j-range partials add up)
            float sf = 0.f;
#pragma unroll
            for (int a = 0; a < NS; ++a) sf += si[a][0] * fa[a][0] + si[a][1] * fa[a][1] + si[a][2] * fa[a][2];
            o.w -= 2.f * sf;
#pragma unroll
            for (int a = 0; a < NS; ++a) {
                o.F[0] += fa[a][0]; o.F[1] += fa[a][1]; o.F[2] += fa[a][2];
                o.T[0] += si[a][1] * fa[a][2] - si[a][2] * fa[a][1];
                o.T[1] += si[a][2] * fa[a][0] - si[a][0] * fa[a][2];
                o.T[2] += si[a][0] * fa[a][1] - si[a][1] * fa[a][0];
                if (DMU && ((DM >> a) & 1)) {
                    o.T[0] += mui[a][1] * ea[a][2] - mui[a][2] * ea[a][1];
                    o.T[1] += mui[a][2] * ea[a][0] - mui[a][0] * ea[a][2];
                    o.T[2] += mui[a][0] * ea[a][1] - mui[a][1] * ea[a][0];
                }
            }
            if (MOLD && rfq) {  // -2 C k_RF mu_i.mu_j and its torque 2 C k_RF mu_i x mu_j
                const float c2 = 2.f * C * krf;
                o.uqq -= c2 * (mdi[0] * erf_[0] + mdi[1] * erf_[1] + mdi[2] * erf_[2]);
                o.T[0] += c2 * (mdi[1] * erf_[2] - mdi[2] * erf_[1]);
                o.T[1] += c2 * (mdi[2] * erf_[0] - mdi[0] * erf_[2]);
                o.T[2] += c2 * (mdi[0] * erf_[1] - mdi[1] * erf_[0]);
            }
        }
        return o;
    }
};

}  // namespace pair_engine
