// Ewald reciprocal space (paper, Sec. "Algorithmic Developments", paragraph
// "Ewald summation": the long-range part is computed in Fourier space) as
// block-level tasks shared by the per-phase kernels (k_ewald.cu) and the fused
// step (k_step.cu):
//
//   S(k)  = sum_s q_s exp(i k.r_s),  k = 2 pi (nx, ny, nz) / L, |n_c| <= kmax_c
//   U_rec = (4 pi C / V) sum_{half space} A(k) |S(k)|^2,  A = exp(-k^2/4a^2)/k^2
//   W_at  = (4 pi C / V) sum_{half space} A |S|^2 (1 - k^2/(2 a^2))
//   F_s   = (8 pi C q_s / V) sum_{half space} A(k) k Im(S(k)* exp(i k.r_s))
//
// k is indexed (col, nx), col = (ny + ky)(2 kz + 1) + nz + kz, nx = 0..kx.
// Sites carry 32-bit lattice coordinates (centre lattice coordinate + rounded
// FP32 offset), so n X mod 2^32 is an exact phase and exp(i n theta) needs no
// range reduction: sincospif of the phase read as a signed fraction of pi.
// Every task's result depends only on its index, never on the number of threads
// that run it, and every sum has a fixed order: both paths give the same bits.
#pragma once
#include "ms2_internal.cuh"

namespace ewald {

constexpr int SKC_MIN = 16;  // sites per structure-factor task at least (S.sk_sites: per system)
constexpr int NXC = 9;       // nx values per structure-factor work item (the grouping of k into work items
                             // does not change any partial: each is one thread's sum over the task's sites)
constexpr int KB = 32;     // k vectors per sum task
constexpr int SLOTS = 32;  // fixed partial-sum slots of a sum task

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conjf2(float2 a, bool c) { return make_float2(a.x, c ? -a.y : a.y); }

// compensated (Kahan) FP32 accumulation: the value is sum - comp
__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x) {
    const float y = __fsub_rn(x, comp), t = __fadd_rn(sum, y);
    comp = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

__host__ __device__ inline int n_k(int kx, int ky, int kz) { return (2 * ky + 1) * (2 * kz + 1) * (kx + 1); }
// sites per structure-factor task for M sites and a fused grid of G blocks: all
// tasks in one round of the fused step (a function of the system and the device)
__host__ __device__ inline int sk_sites(int M, int G) { return max(SKC_MIN, (M + G - 1) / max(G, 1)); }
__host__ __device__ inline int n_site_tasks(int M, int skc) { return (M + skc - 1) / skc; }
__host__ __device__ inline int n_sum_tasks(int K) { return (K + KB - 1) / KB; }
__host__ __device__ inline size_t sk_smem(int kx, int ky, int kz, int skc) {
    return sizeof(float2) * skc * (size_t)(kx + ky + kz + 3) + sizeof(float) * skc;
}
__host__ __device__ inline size_t sum_smem() { return sizeof(float4) * SLOTS * KB; }
__host__ __device__ inline size_t force_smem(int kx, int kz, int ny_per_chunk, int sites) {
    return sizeof(float2) * ((size_t)ny_per_chunk * (2 * kz + 1) * (kx + 1) + (size_t)(kx + kz + 2) * sites);
}

// Structure-factor task sb: the sites [skc sb, skc (sb + 1)), skc = S.sk_sites.  Their charges and
// phase tables e^{i n theta_c}, n = 0..kmax_c, go to shared memory and to global
// memory (for the force tasks); then each work item (one (ny, nz) column, a run
// of NXC nx values) sums q_s e^{i k.r_s} over the task's sites in site order
// (FP32) and writes one partial per k to skpart[sb][k].  All threads of the
// block call it (tid = threadIdx.x, nt = blockDim.x).
__device__ __forceinline__ void sk_task(const SysParams *__restrict__ P, const DevSys &S, int sb, unsigned char *smem,
                                        int tid, int nt) {
    const int M = S.nsite_q, kx = S.kx, ky = S.ky, kz = S.kz, kstride = max(kx, max(ky, kz)) + 1;
    const int SKC = S.sk_sites, s0 = sb * SKC, nk = kx + ky + kz + 3;
    float2 *tab = (float2 *)smem;                     // [SKC][nk]: ex[0..kx], ey[0..ky], ez[0..kz]
    float *sq = (float *)(tab + (size_t)SKC * nk);    // [SKC]
    const int N = S.N, NS = S.ns;
    for (int t = tid; t < SKC * nk; t += nt) {
        const int ls = t % SKC, r = t / SKC, s = s0 + ls;
        const int c = r <= kx ? 0 : (r <= kx + ky + 1 ? 1 : 2);
        const int n = c == 0 ? r : (c == 1 ? r - kx - 1 : r - kx - ky - 2);
        float2 v = make_float2(0.f, 0.f);
        if (s < M) {
            const int a = s / N, i = s - a * N;
            const uint32_t Xc = __ldcg(S.X + c * N + i) +
                                (uint32_t)__float2int_rn(__ldcg(S.s + (c * NS + a) * N + i) * P->len_to_lat);
            const int ph = (int)((uint32_t)n * Xc);
            float sn, cs;
            sincospif((float)ph * 4.656612873077393e-10f, &sn, &cs);  // ph / 2^31
            v = make_float2(cs, sn);
            S.eik[((size_t)c * kstride + n) * M + s] = v;
        }
        tab[(size_t)ls * nk + r] = v;
    }
    for (int t = tid; t < SKC; t += nt) {
        const int s = s0 + t;
        float q = 0.f;
        if (s < M) {
            const int a = s / N, sp = S.species[s - a * N];
            q = (a < P->n_sites[sp]) ? P->q[sp][a] : 0.f;  // FP32 terms of S(k)
            S.qs[s] = q;
        }
        sq[t] = q;
    }
    __syncthreads();
    const int ncols = (2 * ky + 1) * (2 * kz + 1), nxch = (kx + NXC) / NXC;
    for (int w = tid; w < ncols * nxch; w += nt) {
        const int col = w / nxch, nx0 = (w % nxch) * NXC;
        const int ny = col / (2 * kz + 1) - ky, nz = col % (2 * kz + 1) - kz;
        const int ay = kx + 1 + abs(ny), az = kx + ky + 2 + abs(nz);
        float ar[NXC], ai[NXC];
#pragma unroll
        for (int k = 0; k < NXC; ++k) ar[k] = ai[k] = 0.f;
        for (int ls = 0; ls < SKC; ++ls) {
            const float2 *e = tab + (size_t)ls * nk;
            const float2 ey = conjf2(e[ay], ny < 0), ez = conjf2(e[az], nz < 0);
            const float q = sq[ls];
            const float2 eyz = cmul(make_float2(q * ey.x, q * ey.y), ez);
#pragma unroll
            for (int k = 0; k < NXC; ++k) {
                const int nx = min(nx0 + k, kx);  // beyond kx: computed, not written
                const float2 v = cmul(e[nx], eyz);
                ar[k] += v.x;
                ai[k] += v.y;
            }
        }
        float2 *out = S.skpart + ((size_t)sb * ncols + col) * (kx + 1);
#pragma unroll
        for (int k = 0; k < NXC; ++k)
            if (nx0 + k <= kx) out[nx0 + k] = make_float2(ar[k], ai[k]);
    }
    __syncthreads();  // the scratch is free for the next task
}

// Sum task kc: the KB consecutive k = KB kc + j.  Slot sl (0..SLOTS-1) sums the
// partials of the site tasks sl, sl + SLOTS, ... in order (compensated FP32, rows
// of consecutive k: coalesced); the slots are added in slot order; then lane j
// of warp 0 forms A S(k_j) (FP32, for the force tasks) and the energy and
// virial terms from the host tables A(k) (zero outside the half space) and
// A(k)(1 - k^2/2a^2), summed by a fixed warp tree into kblk[kc].  All threads of
// the block call it.
__device__ __forceinline__ void sum_task(const DevSys &S, float2 *AS, int kc, int nsb, unsigned char *smem, int tid,
                                         int nt) {
    const int K = n_k(S.kx, S.ky, S.kz);
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5, k = kc * KB + lane;
    float4 *wacc = (float4 *)smem;  // [SLOTS][KB]: (sum re, compensation re, sum im, compensation im)
    for (int sl = warp; sl < SLOTS; sl += nw) {
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < K) {
            int b = sl;
            for (; b + 7 * SLOTS < nsb; b += 8 * SLOTS) {  // 8 loads in flight, then the adds in order
                float2 p[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) p[u] = __ldcg(S.skpart + (size_t)(b + u * SLOTS) * K + k);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    kahan_add(a.x, a.y, p[u].x);
                    kahan_add(a.z, a.w, p[u].y);
                }
            }
            for (; b < nsb; b += SLOTS) {
                const float2 p = __ldcg(S.skpart + (size_t)b * K + k);
                kahan_add(a.x, a.y, p.x);
                kahan_add(a.z, a.w, p.y);
            }
        }
        wacc[sl * KB + lane] = a;
    }
    __syncthreads();
    if (warp == 0) {
        double e = 0.0, w = 0.0;
        if (k < K) {
            float hr = 0.f, cr = 0.f, hi = 0.f, ci = 0.f;
            for (int sl = 0; sl < SLOTS; ++sl) {
                const float4 a = wacc[sl * KB + lane];
                kahan_add(hr, cr, a.x);
                kahan_add(hr, cr, -a.y);
                kahan_add(hi, ci, a.z);
                kahan_add(hi, ci, -a.w);
            }
            const double sr = (double)hr - (double)cr, si = (double)hi - (double)ci;
            const double A = S.Ak[k], s2 = sr * sr + si * si;
            AS[k] = make_float2((float)(A * sr), (float)(A * si));
            e = A * s2;
            w = S.Bk[k] * s2;
        }
        e = warp_sum(e);
        w = warp_sum(w);
        if (lane == 0) {
            S.kblk[2 * kc] = e;
            S.kblk[2 * kc + 1] = w;
        }
    }
    __syncthreads();  // the scratch is free for the next task
}

// U_rec and W_rec from the nkc sum tasks' pairs, in task order (one warp)
__device__ __forceinline__ void sum_finish(const SysParams *__restrict__ P, const DevSys &S, int nkc, int lane) {
    double te = 0.0, tw = 0.0;
    for (int b = lane; b < nkc; b += 32) {
        te += __ldcg(S.kblk + 2 * b);
        tw += __ldcg(S.kblk + 2 * b + 1);
    }
    te = warp_sum(te);
    tw = warp_sum(tw);
    if (lane == 0) {
        const double pre = 4.0 * 3.141592653589793 * ((double)P->coulomb + (double)P->coulomb_lo) / P->V;
        S.scal[SC_UREC] = pre * te;
        S.scal[SC_WREC_AT] = pre * tw;
    }
}

// Force task: the sites [s0, s0 + nt) (thread tid owns site s0 + tid) and the k
// chunk ch (ny = -ky + ch ny_per_chunk ..): the chunk's A S(k) and the sites'
// e^{i nx theta_x} and e^{i nz theta_z} are staged in shared memory; each thread sums its site's
// force over the chunk (FP32, fixed k order) into frec[ch][3][site].  KXT: kx + 1
// at compile time (nx loop unrolled, the site's x phases in registers) or 0.  All
// threads of the block call it.
template <int KXT>
__device__ __forceinline__ void force_task(const SysParams *__restrict__ P, const DevSys &S, const float2 *AS, int s0,
                                           int ch, int ny_per_chunk, unsigned char *smem, int tid, int nt) {
    const int M = S.nsite_q, s = s0 + tid;
    const int kx = KXT > 0 ? KXT - 1 : S.kx, ky = S.ky, kz = S.kz, kstride = max(kx, max(ky, kz)) + 1;
    const int nyb = -ky + ch * ny_per_chunk, nye = min(ky, nyb + ny_per_chunk - 1);
    const int ncz = 2 * kz + 1, nchunk = (nye - nyb + 1) * ncz * (kx + 1);
    float2 *as_s = (float2 *)smem;                                  // the chunk's A S(k), k order
    float2 *ex_s = as_s + (size_t)ny_per_chunk * ncz * (kx + 1);   // [kx + 1][nt]
    float2 *ez_s = ex_s + (size_t)(kx + 1) * nt;                    // [kz + 1][nt]
    const float2 *asg = AS + (size_t)(nyb + ky) * ncz * (kx + 1);
    for (int t = tid; t < nchunk; t += nt) as_s[t] = __ldcg(asg + t);
    const int ss = s < M ? s : 0;
    for (int nx = 0; nx <= kx; ++nx) ex_s[nx * nt + tid] = __ldcg(S.eik + (size_t)nx * M + ss);
    for (int n = 0; n <= kz; ++n) ez_s[n * nt + tid] = __ldcg(S.eik + ((size_t)2 * kstride + n) * M + ss);
    __syncthreads();
    // the column sums enter compensated sums (their FP32 roundings would reach
    // the molecular virial through the site levers, sum_s F_s.s_s)
    float fx = 0.f, fy = 0.f, fz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    const float q = __ldcg(S.qs + ss);
    float2 exr[KXT > 0 ? KXT : 1];
    const float2 *ey = S.eik + (size_t)kstride * M + ss;
    if constexpr (KXT > 0) {
#pragma unroll
        for (int nx = 0; nx < KXT; ++nx) exr[nx] = ex_s[nx * nt + tid];
    }
    if (s < M && q != 0.f) {
        for (int ny = nyb; ny <= nye; ++ny) {
            const float2 eyv = conjf2(__ldcg(ey + (size_t)abs(ny) * M), ny < 0);
            for (int nz = -kz; nz <= kz; ++nz) {
                const float2 eyz = cmul(eyv, conjf2(ez_s[abs(nz) * nt + tid], nz < 0));
                const float2 *as = as_s + ((size_t)(ny - nyb) * ncz + nz + kz) * (kx + 1);
                float sx = 0.f, syz = 0.f;
                if constexpr (KXT > 0) {
#pragma unroll
                    for (int nx = 0; nx < KXT; ++nx) {
                        const float2 e = cmul(exr[nx], eyz);
                        const float2 a = as[nx];
                        const float im = a.x * e.y - a.y * e.x;  // Im(A S* e)
                        sx += (float)nx * im;
                        syz += im;
                    }
                } else {
                    for (int nx = 0; nx <= kx; ++nx) {
                        const float2 e = cmul(ex_s[nx * nt + tid], eyz);
                        const float2 a = as[nx];
                        const float im = a.x * e.y - a.y * e.x;  // Im(A S* e)
                        sx += (float)nx * im;
                        syz += im;
                    }
                }
                kahan_add(fx, cx, sx);
                kahan_add(fy, cy, (float)ny * syz);
                kahan_add(fz, cz, (float)nz * syz);
            }
        }
        // the prefactor (8 pi C / V) (2 pi / L) q_s as hi + lo: the host's FP64
        // constant and the site's charge, each carried as two floats (one FP32
        // rounding of either would scale every site force of its kind the same
        // way and bias the lever sum sum_s F_s.s_s of the molecular virial)
        const int a = ss / S.N, sp = S.species[ss - a * S.N];
        const float ql = a < P->n_sites[sp] ? P->qlo[sp][a] : 0.f;
        const float ph = S.ew_fpre * q;
        const float pl = fmaf(S.ew_fpre, q, -ph) + fmaf(S.ew_fpre, ql, S.ew_fpre_lo * q);
        fx -= cx; fy -= cy; fz -= cz;
        fx = fmaf(fx, ph, fx * pl); fy = fmaf(fy, ph, fy * pl); fz = fmaf(fz, ph, fz * pl);
    }
    if (s < M) {
        float *o = S.frec + (size_t)ch * 3 * M + s;
        o[0] = fx;
        o[M] = fy;
        o[2 * M] = fz;
    }
    __syncthreads();  // the scratch is free for the next task
}

}  // namespace ewald
