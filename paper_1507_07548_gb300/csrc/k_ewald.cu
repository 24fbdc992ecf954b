// K3/K4: Ewald reciprocal space (paper, Sec. "Algorithmic Developments",
// paragraph "Ewald summation": the long-range part is computed in Fourier space).
//
//   S(k)  = sum_s q_s exp(i k.r_s),  k = 2 pi (nx, ny, nz) / L, |n_c| <= kmax_c
//   U_rec = (4 pi C / V) sum_{half space} A(k) |S(k)|^2,  A = exp(-k^2/4a^2)/k^2
//   W_at  = (4 pi C / V) sum_{half space} A |S|^2 (1 - k^2/(2 a^2))
//   F_s   = (8 pi C q_s / V) sum_{half space} A(k) k Im(S(k)* exp(i k.r_s))
// Sites carry 32-bit lattice coordinates (centre lattice coordinate + rounded
// FP32 offset), so n * X mod 2^32 is an exact phase and exp(i n theta) needs no
// range reduction: sincospif of the phase read as a signed fraction of pi.
//
// Per step: k_ewald_skp (phase tables and partial S(k) of site blocks),
// k_ewald_sksum (S(k) in fixed order, A S(k), U_rec and W_rec),
// k_ewald_force (site forces of k chunks) and k_ewald_fsum (the chunks summed
// per site).  Every sum has a fixed order, so results are bitwise reproducible.
#include "ms2_internal.cuh"

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

// S(k) in two passes.  Pass 1 (k_ewald_skp): block b takes the EW_SKC sites
// [EW_SKC b, EW_SKC (b+1)), forms their charges and phase tables
// e^{i n theta_c}, n = 0..kmax_c (theta_c from the site's lattice coordinate c:
// centre lattice coordinate + rounded FP32 offset, so n X mod 2^32 is an exact
// phase and sincospif of it read as a signed fraction of pi needs no range
// reduction), keeps them in shared memory and stores them for the force kernel;
// then every thread owns one (ny, nz) column and a run of EW_NXC nx
// values of the k lattice: it sums q_s e^{i k.r_s} over the block's sites into
// registers (FP32, site order) and writes one partial per k.  Each site's table
// is read once from L2; the (ny, nz) phase product is formed once per site and
// column.  Pass 2 (k_ewald_sksum): a thread per k sums the block partials in
// block order (FP64), forms A(k) S(k) for the force kernel and the energy and
// virial terms of the half space, reduced over the grid in a fixed tree (last
// block: U_rec, W_rec).
constexpr int EW_SKC = 16;  // sites per block of pass 1
constexpr int EW_NXC = 9;   // nx values per work item of pass 1

size_t ms2_ewald_skp_smem(int kx, int ky, int kz) {
    return sizeof(float2) * EW_SKC * (size_t)(kx + ky + kz + 3) + sizeof(float) * EW_SKC;
}
int ms2_ewald_skp_blocks(int M) { return (M + EW_SKC - 1) / EW_SKC; }

__global__ void __launch_bounds__(320) k_ewald_skp(const SysParams *__restrict__ P, DevSys S) {
    extern __shared__ __align__(16) unsigned char ew_smem[];
    const int M = S.nsite_q, kx = S.kx, ky = S.ky, kz = S.kz, kstride = max(kx, max(ky, kz)) + 1;
    const int s0 = blockIdx.x * EW_SKC, nk = kx + ky + kz + 3;
    float2 *tab = (float2 *)ew_smem;                     // [EW_SKC][nk]: ex[0..kx], ey[0..ky], ez[0..kz]
    float *sq = (float *)(tab + (size_t)EW_SKC * nk);    // [EW_SKC]
    const int N = S.N, NS = S.ns;
    for (int t = threadIdx.x; t < EW_SKC * nk; t += blockDim.x) {
        const int ls = t % EW_SKC, r = t / EW_SKC, s = s0 + ls;
        const int c = r <= kx ? 0 : (r <= kx + ky + 1 ? 1 : 2);
        const int n = c == 0 ? r : (c == 1 ? r - kx - 1 : r - kx - ky - 2);
        float2 v = make_float2(0.f, 0.f);
        if (s < M) {
            const int a = s / N, i = s - a * N;
            const uint32_t Xc = S.X[c * N + i] + (uint32_t)__float2int_rn(S.s[(c * NS + a) * N + i] * P->len_to_lat);
            const int ph = (int)((uint32_t)n * Xc);
            float sn, cs;
            sincospif((float)ph * 4.656612873077393e-10f, &sn, &cs);  // ph / 2^31
            v = make_float2(cs, sn);
            S.eik[((size_t)c * kstride + n) * M + s] = v;
        }
        tab[(size_t)ls * nk + r] = v;
    }
    for (int t = threadIdx.x; t < EW_SKC; t += blockDim.x) {
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
    const int ncols = (2 * ky + 1) * (2 * kz + 1), nxch = (kx + EW_NXC) / EW_NXC;
    for (int w = threadIdx.x; w < ncols * nxch; w += blockDim.x) {
        const int col = w / nxch, nx0 = (w % nxch) * EW_NXC;
        const int ny = col / (2 * kz + 1) - ky, nz = col % (2 * kz + 1) - kz;
        const int ay = kx + 1 + abs(ny), az = kx + ky + 2 + abs(nz);
        float ar[EW_NXC], ai[EW_NXC];
#pragma unroll
        for (int k = 0; k < EW_NXC; ++k) ar[k] = ai[k] = 0.f;
        for (int ls = 0; ls < EW_SKC; ++ls) {
            const float2 *e = tab + (size_t)ls * nk;
            const float2 ey = conjf2(e[ay], ny < 0), ez = conjf2(e[az], nz < 0);
            const float q = sq[ls];
            const float2 eyz = cmul(make_float2(q * ey.x, q * ey.y), ez);
#pragma unroll
            for (int k = 0; k < EW_NXC; ++k) {
                const int nx = min(nx0 + k, kx);  // beyond kx: computed, not written
                const float2 v = cmul(e[nx], eyz);
                ar[k] += v.x;
                ai[k] += v.y;
            }
        }
        float2 *out = S.skpart + ((size_t)blockIdx.x * ncols + col) * (kx + 1);
#pragma unroll
        for (int k = 0; k < EW_NXC; ++k)
            if (nx0 + k <= kx) out[nx0 + k] = make_float2(ar[k], ai[k]);
    }
}

// Pass 2: a block of 32 warps per 32 consecutive k = (col, nx).  Warp w reads
// the rows b = w, w + 32, ... of the partials (32 consecutive k: coalesced) and
// lane j sums k_j over them in order; the 32 warp sums of each k are added in
// warp order through shared memory.  The sums are compensated FP32 sums (Kahan:
// about FP64 accuracy for these few hundred terms, where FP64 adds and
// conversions would occupy the small FP64 unit); then lane j of warp 0 forms A S(k_j) and the
// energy and virial terms of k_j from the host-made tables A(k) (zero outside the
// half space) and A(k) (1 - k^2 / 2 alpha^2), reduced in a fixed tree into one
// (energy, virial) pair per block; the last block sums those in block order.
constexpr int EW_KB = 32;  // k vectors per block of pass 2
int ms2_ewald_sksum_blocks(int K) { return (K + EW_KB - 1) / EW_KB; }

__global__ void __launch_bounds__(1024) k_ewald_sksum(const SysParams *__restrict__ P, DevSys S, float2 *AS, int nblk) {
    const int kx = S.kx, ky = S.ky, kz = S.kz;
    const int ncols = (2 * ky + 1) * (2 * kz + 1), K = ncols * (kx + 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int k0 = blockIdx.x * EW_KB;
    __shared__ float4 wacc[32][EW_KB];  // per warp and k: (sum re, compensation re, sum im, compensation im)
    {
        const int k = k0 + lane;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < K)
            for (int b = warp; b < nblk; b += nw) {
                const float2 p = __ldcg(S.skpart + (size_t)b * K + k);
                kahan_add(a.x, a.y, p.x);
                kahan_add(a.z, a.w, p.y);
            }
        wacc[warp][lane] = a;
    }
    __syncthreads();
    __shared__ bool last;
    if (warp == 0) {
        const int k = k0 + lane;
        double e = 0.0, w = 0.0;
        if (k < K) {
            float hr = 0.f, cr = 0.f, hi = 0.f, ci = 0.f;
            for (int q = 0; q < nw; ++q) {
                const float4 a = wacc[q][lane];
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
            S.kblk[2 * blockIdx.x] = e;
            S.kblk[2 * blockIdx.x + 1] = w;
            __threadfence();
            last = atomicAdd(S.counter + 4, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < 32) {
        double te = 0.0, tw2 = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) {
            te += __ldcg(S.kblk + 2 * b);
            tw2 += __ldcg(S.kblk + 2 * b + 1);
        }
        te = warp_sum(te);
        tw2 = warp_sum(tw2);
        if (threadIdx.x == 0) {
            const double pre = 4.0 * 3.141592653589793 * (double)P->coulomb / P->V;
            S.scal[SC_UREC] = pre * te;
            S.scal[SC_WREC_AT] = pre * tw2;
            S.counter[4] = 0u;
        }
    }
}

// grid: x = block of EW_FB sites, y = chunk of ny values.  Each thread owns one
// site and sums its chunk of k vectors; the block stages the chunk's A S(k) and
// its sites' e^{i nx theta_x} in shared memory, so the k loop reads no global
// memory.  Partial forces go to frec[chunk][3][site].
constexpr int EW_FB = 128;
size_t ms2_ewald_force_smem(int kx, int kz, int ny_per_chunk) {
    return sizeof(float2) * ((size_t)ny_per_chunk * (2 * kz + 1) * (kx + 1) + (size_t)(kx + 1) * EW_FB);
}

// KXT: kx + 1 at compile time (the nx loop unrolled, the site's e^{i nx theta_x}
// in registers), or 0 for any kx
template <int KXT>
__global__ void __launch_bounds__(EW_FB) k_ewald_force(const SysParams *__restrict__ P, DevSys S, const float2 *AS,
                                                      int ny_per_chunk) {
    extern __shared__ __align__(16) unsigned char ew_smem[];
    const int M = S.nsite_q, s = blockIdx.x * blockDim.x + threadIdx.x;
    const int kx = KXT > 0 ? KXT - 1 : S.kx, ky = S.ky, kz = S.kz, kstride = max(kx, max(ky, kz)) + 1;
    const int nyb = -ky + blockIdx.y * ny_per_chunk, nye = min(ky, nyb + ny_per_chunk - 1);
    const int ncz = 2 * kz + 1, nchunk = (nye - nyb + 1) * ncz * (kx + 1);
    float2 *as_s = (float2 *)ew_smem;                                   // the chunk's A S(k), k order
    float2 *ex_s = as_s + (size_t)ny_per_chunk * ncz * (kx + 1);        // [kx + 1][EW_FB]
    const float2 *asg = AS + (size_t)(nyb + ky) * ncz * (kx + 1);
    for (int t = threadIdx.x; t < nchunk; t += blockDim.x) as_s[t] = asg[t];
    const int ss = s < M ? s : 0;
    for (int nx = 0; nx <= kx; ++nx) ex_s[nx * EW_FB + threadIdx.x] = S.eik[(size_t)nx * M + ss];
    __syncthreads();
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const float q = S.qs[ss];
    float2 exr[KXT > 0 ? KXT : 1];
    if constexpr (KXT > 0) {
#pragma unroll
        for (int nx = 0; nx < KXT; ++nx) exr[nx] = ex_s[nx * EW_FB + threadIdx.x];
    }
    if (s < M && q != 0.f) {
        const float2 *ey = S.eik + (size_t)kstride * M + ss, *ez = S.eik + (size_t)2 * kstride * M + ss;
        for (int ny = nyb; ny <= nye; ++ny) {
            const float2 eyv = conjf2(ey[(size_t)abs(ny) * M], ny < 0);
            for (int nz = -kz; nz <= kz; ++nz) {
                const float2 eyz = cmul(eyv, conjf2(ez[(size_t)abs(nz) * M], nz < 0));
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
                        const float2 e = cmul(ex_s[nx * EW_FB + threadIdx.x], eyz);
                        const float2 a = as[nx];
                        const float im = a.x * e.y - a.y * e.x;  // Im(A S* e)
                        sx += (float)nx * im;
                        syz += im;
                    }
                }
                fx += sx;
                fy += (float)ny * syz;
                fz += (float)nz * syz;
            }
        }
        const float pre = (float)(8.0 * 3.141592653589793 * (double)P->coulomb / P->V * 2.0 * 3.141592653589793 / P->L) * q;
        fx *= pre; fy *= pre; fz *= pre;
    }
    if (s < M) {
        float *o = S.frec + (size_t)blockIdx.y * 3 * M + s;
        o[0] = fx;
        o[M] = fy;
        o[2 * M] = fz;
    }
}

// Thread per (component c, site s): the kchunks partial site forces summed in
// chunk order (FP32, independent loads), in place into chunk 0 of frec.
__global__ void __launch_bounds__(128) k_ewald_fsum(const SysParams *__restrict__ P, DevSys S) {
    const int M = S.nsite_q, t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * M) return;
    const int c = t / M, s = t - c * M;
    float f = 0.f;
    int ch = 0;
    for (; ch + 8 <= S.kchunks; ch += 8) {
        float p[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) p[u] = __ldcg(S.frec + ((size_t)(ch + u) * 3 + c) * M + s);
#pragma unroll
        for (int u = 0; u < 8; ++u) f += p[u];
    }
    for (; ch < S.kchunks; ++ch) f += __ldcg(S.frec + ((size_t)ch * 3 + c) * M + s);
    S.frec[(size_t)c * M + s] = f;
}

// the force kernel for kx = 8 (the default |n| <= 8), or any kx
void *ms2_ewald_force_kernel(int kx) {
    return kx == 8 ? (void *)&k_ewald_force<9> : (void *)&k_ewald_force<0>;
}
