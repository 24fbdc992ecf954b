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
#include "ms2_internal.cuh"

// per site (slot-major index s = a*N + i): lattice coordinates, charge and
// exp(i n theta_c) for n = 0..kmax_c, c = x, y, z
__global__ void k_ewald_prep(const SysParams *__restrict__ P, DevSys S) {
    const int M = S.nsite_q, s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const int N = S.N, NS = S.ns, a = s / N, i = s - a * N;
    const int sp = S.species[i];
    const float l2 = P->len_to_lat;
    const int km[3] = {S.kx, S.ky, S.kz};
    const int kstride = max(S.kx, max(S.ky, S.kz)) + 1;
    for (int c = 0; c < 3; ++c) {
        const uint32_t Xc = S.X[c * N + i] + (uint32_t)__float2int_rn(S.s[(c * NS + a) * N + i] * l2);
        S.Xs[c * M + s] = Xc;
        for (int n = 0; n <= km[c]; ++n) {
            const int ph = (int)((uint32_t)n * Xc);
            float sn, cs;
            sincospif((float)ph * 4.656612873077393e-10f, &sn, &cs);  // ph / 2^31
            S.eik[((size_t)c * kstride + n) * M + s] = make_float2(cs, sn);
        }
    }
    S.qs[s] = (a < P->n_sites[sp]) ? P->q[sp][a] : 0.f;  // FP32 terms of S(k)
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conjf2(float2 a, bool c) { return make_float2(a.x, c ? -a.y : a.y); }

// grid: x = (ny, nz) column in [-ky,ky] x [-kz,kz], y = chunk of 8 nx values.
// Writes AS[k] = A(k) S(k) (FP32, for the force kernel) for half-space k
// (zero elsewhere) and one energy/virial partial per block.
constexpr int SK_NX = 8;
__global__ void __launch_bounds__(256) k_ewald_sk(const SysParams *__restrict__ P, DevSys S, float2 *AS) {
    const int M = S.nsite_q;
    const int kx = S.kx, ky = S.ky, kz = S.kz, kstride = max(kx, max(ky, kz)) + 1;
    const int col = blockIdx.x, ny = col / (2 * kz + 1) - ky, nz = col % (2 * kz + 1) - kz;
    const int nx0 = blockIdx.y * SK_NX;
    const int nxlo = (ny > 0 || (ny == 0 && nz > 0)) ? 0 : 1;  // half space
    float ar[SK_NX], ai[SK_NX];
#pragma unroll
    for (int k = 0; k < SK_NX; ++k) ar[k] = ai[k] = 0.f;
    const float2 *ex = S.eik, *ey = S.eik + (size_t)kstride * M + (size_t)abs(ny) * M,
                 *ez = S.eik + (size_t)2 * kstride * M + (size_t)abs(nz) * M;
    for (int s = threadIdx.x; s < M; s += blockDim.x) {
        const float q = S.qs[s];
        const float2 eyz = cmul(conjf2(ey[s], ny < 0), conjf2(ez[s], nz < 0));
#pragma unroll
        for (int k = 0; k < SK_NX; ++k) {
            const int nx = nx0 + k;
            if (nx <= kx) {
                const float2 e = cmul(ex[(size_t)nx * M + s], eyz);
                ar[k] += q * e.x;
                ai[k] += q * e.y;
            }
        }
    }
    __shared__ double red[8][SK_NX][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < SK_NX; ++k) {
        const float r = warp_sum(ar[k]), im = warp_sum(ai[k]);
        if (lane == 0) { red[warp][k][0] = r; red[warp][k][1] = im; }
    }
    __syncthreads();
    if (threadIdx.x < SK_NX) {
        const int k = threadIdx.x, nx = nx0 + k;
        double sr = 0, si = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sr += red[w][k][0]; si += red[w][k][1]; }
        const double tw = 2.0 * 3.141592653589793 / P->L;
        const double kk = tw * tw * ((double)nx * nx + (double)ny * ny + (double)nz * nz);
        const bool on = nx <= kx && nx >= nxlo;
        const double A = on ? exp(-kk / (4.0 * (double)P->alpha * P->alpha)) / kk : 0.0;
        const double e = A * (sr * sr + si * si);
        red[0][k][0] = e;
        red[0][k][1] = e * (1.0 - kk / (2.0 * (double)P->alpha * P->alpha));
        if (nx <= kx) AS[((size_t)col) * (kx + 1) + nx] = make_float2((float)(A * sr), (float)(A * si));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 0, w = 0;
        for (int k = 0; k < SK_NX; ++k) { e += red[0][k][0]; w += red[0][k][1]; }
        const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        S.kblk[2 * b] = e;
        S.kblk[2 * b + 1] = w;
    }
}

// fixed-order sum of the S(k) block partials -> U_rec, W_rec (atomic part)
__global__ void k_ewald_energy(const SysParams *__restrict__ P, DevSys S, int nblk) {
    __shared__ double part[2][256];
    double e = 0, w = 0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) { e += S.kblk[2 * b]; w += S.kblk[2 * b + 1]; }
    part[0][threadIdx.x] = e;
    part[1][threadIdx.x] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
        double te = 0, tw = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) { te += part[0][t]; tw += part[1][t]; }
        const double pre = 4.0 * 3.141592653589793 * (double)P->coulomb / P->V;
        S.scal[SC_UREC] = pre * te;
        S.scal[SC_WREC_AT] = pre * tw;
    }
}

// grid: x = block of sites, y = chunk of ny values.  Each thread owns one site
// and sums its chunk of k vectors; partial forces go to frec[chunk][3][site].
__global__ void __launch_bounds__(128) k_ewald_force(const SysParams *__restrict__ P, DevSys S, const float2 *AS,
                                                    int ny_per_chunk) {
    const int M = S.nsite_q, s = blockIdx.x * blockDim.x + threadIdx.x;
    const int kx = S.kx, ky = S.ky, kz = S.kz, kstride = max(kx, max(ky, kz)) + 1;
    const int nyb = -ky + blockIdx.y * ny_per_chunk, nye = min(ky, nyb + ny_per_chunk - 1);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const int ss = s < M ? s : 0;
    const float q = S.qs[ss];
    if (s < M && q != 0.f) {
        const float2 *ex = S.eik + ss, *ey = S.eik + (size_t)kstride * M + ss, *ez = S.eik + (size_t)2 * kstride * M + ss;
        for (int ny = nyb; ny <= nye; ++ny) {
            const float2 eyv = conjf2(ey[(size_t)abs(ny) * M], ny < 0);
            for (int nz = -kz; nz <= kz; ++nz) {
                const float2 eyz = cmul(eyv, conjf2(ez[(size_t)abs(nz) * M], nz < 0));
                const float2 *as = AS + ((size_t)((ny + ky) * (2 * kz + 1) + nz + kz)) * (kx + 1);
                float sx = 0.f, syz = 0.f;
                for (int nx = 0; nx <= kx; ++nx) {
                    const float2 e = cmul(ex[(size_t)nx * M], eyz);
                    const float2 a = as[nx];
                    const float im = a.x * e.y - a.y * e.x;  // Im(A S* e)
                    sx += (float)nx * im;
                    syz += im;
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
