// K3/K4: Ewald reciprocal space as per-phase kernels over the tasks of
// ewald_dev.cuh (the fused step runs the same tasks): k_ewald_skp (phase tables
// and partial S(k) of 16-site blocks), k_ewald_sksum (S(k) in fixed order,
// A S(k), and in the last block U_rec and W_rec), k_ewald_force (site forces of
// k chunks; the reduction sums the chunks per site).
#include "ewald_dev.cuh"

using namespace ewald;

size_t ms2_ewald_skp_smem(int kx, int ky, int kz, int skc) { return sk_smem(kx, ky, kz, skc); }
int ms2_ewald_sk_sites(int M, int G) { return sk_sites(M, G); }
int ms2_ewald_skp_blocks(int M, int skc) { return n_site_tasks(M, skc); }
int ms2_ewald_sksum_blocks(int K) { return n_sum_tasks(K); }
size_t ms2_ewald_force_smem(int kx, int kz, int ny_per_chunk) { return force_smem(kx, kz, ny_per_chunk, 128); }

__global__ void __launch_bounds__(320) k_ewald_skp(const SysParams *__restrict__ P, DevSys S) {
    extern __shared__ __align__(16) unsigned char ew_smem[];
    sk_task(P, S, blockIdx.x, ew_smem, threadIdx.x, blockDim.x);
}

__global__ void __launch_bounds__(1024) k_ewald_sksum(const SysParams *__restrict__ P, DevSys S, float2 *AS, int nblk) {
    __shared__ __align__(16) unsigned char sm[sizeof(float4) * SLOTS * KB];
    sum_task(S, AS, blockIdx.x, nblk, sm, threadIdx.x, blockDim.x);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(S.counter + 4, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < 32) sum_finish(P, S, gridDim.x, threadIdx.x);
    if (threadIdx.x == 0) S.counter[4] = 0u;
}

template <int KXT>
__global__ void __launch_bounds__(128) k_ewald_force(const SysParams *__restrict__ P, DevSys S, const float2 *AS,
                                                    int ny_per_chunk) {
    extern __shared__ __align__(16) unsigned char ew_smem[];
    force_task<KXT>(P, S, AS, blockIdx.x * blockDim.x, blockIdx.y, ny_per_chunk, ew_smem, threadIdx.x, blockDim.x);
}

// the force kernel for kx = 8 (the default |n| <= 8), or any kx
void *ms2_ewald_force_kernel(int kx, int kz) {
    (void)kz;
    return kx == 8 ? (void *)&k_ewald_force<9> : (void *)&k_ewald_force<0>;
}
