// K7: radial distribution function between LJ sites (paper, Sec. "Property
// Calculations", Eq. 2: g(r) from the number of sites in spherical shells; "The
// RDF is sampled between all LJ sites").
//
// Integer histogram of intermolecular LJ-site pairs at SITE minimum image: each
// site gets a 32-bit lattice coordinate (centre lattice coordinate + rounded FP32
// offset), so the minimum image is an exact 32-bit wrap-around difference.
// Counts are integers, so shared-memory and global integer atomics give the
// same totals in any order.
#include "ms2_internal.cuh"

// grid-stride over molecules i; each thread pairs one j > i at a time.
__global__ void __launch_bounds__(256) k_rdf(const SysParams *__restrict__ P, DevSys S) {
    extern __shared__ unsigned int hist[];  // [rows][bins]
    const int N = S.N, NS = S.ns, nb = S.rdf_bins, rows = S.rdf_rows;
    for (int k = threadIdx.x; k < rows * nb; k += blockDim.x) hist[k] = 0u;
    __syncthreads();
    const float l2l = P->lat_to_len, l2 = P->len_to_lat;
    const float rmax2 = S.rdf_rmax2, inv_dr = S.rdf_inv_dr;
    const int T = P->n_ljt;
    for (int i = blockIdx.x; i < N; i += gridDim.x) {
        const int spi = S.species[i];
        for (int a = 0; a < NS; ++a) {
            const int ta = S.rdf_kind[spi * MS2_MAXS + a];
            if (ta < 0) continue;
            uint32_t Xa[3];
            for (int c = 0; c < 3; ++c)
                Xa[c] = S.X[c * N + i] + (uint32_t)__float2int_rn(S.s[(c * NS + a) * N + i] * l2);
            for (int j = i + 1 + threadIdx.x; j < N; j += blockDim.x) {
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
