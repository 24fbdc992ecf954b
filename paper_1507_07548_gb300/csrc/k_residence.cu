// Residence time and solvation number (paper, Sec. "Algorithmic Developments",
// residence time, Eq. 7, with the tolerance of Impey et al.).
//
// Every extended time step the shell membership of the solvent molecules (a
// species) around each centre molecule (another species) is taken from the
// integer centre lattice -- the same exact minimum-image test as the cut-off --
// and pushed through a ring of the last n_lags time origins.  For every open
// origin and centre, each member carries an alive bit and the length of its
// current excursion; an excursion longer than t_star samples ends the member's
// residence for that origin.  k_res_update (one block per centre) counts, per
// origin, the members alive and inside now, with integer shared-memory
// atomics (order-free, exact); k_res_accum (one block) adds the fractions
// count / n_i(origin) to their lag in a fixed centre order, so the result is
// bitwise reproducible.  The sample counter lives on the device, so the steps
// can be replayed as CUDA graphs.
#include "ms2_internal.cuh"

// sampling state (RES_* doubles at the head of the state block)
enum { RES_SAMPLES = 0, RES_NSUM, RES_NCOUNT, RES_HEAD };

// one block per centre i (A0 + blockIdx.x); threads over 32-molecule words of
// the solvent range [B0, B0 + NB)
__global__ void __launch_bounds__(256) k_res_update(const SysParams *__restrict__ P, DevSys S, ResArgs a) {
    extern __shared__ unsigned res_smem[];
    unsigned *inside = res_smem;          // [WB] membership words now
    int *count = (int *)(inside + a.WB);  // [M] members alive and inside, per origin slot
    const int ci = blockIdx.x, i = a.A0 + ci, M = a.M, N = S.N;
    const long long s = (long long)__ldcg(a.state + RES_SAMPLES);  // index of this sample
    for (int o = threadIdx.x; o < M; o += blockDim.x) count[o] = 0;
    const uint32_t Xi = __ldcg(S.X + i), Yi = __ldcg(S.X + N + i), Zi = __ldcg(S.X + 2 * N + i);
    for (int w = threadIdx.x; w < a.WB; w += blockDim.x) {
        unsigned bits = 0u;
        for (int l = 0; l < 32; ++l) {
            const int k = a.B0 + 32 * w + l;
            if (k >= a.B0 + a.NB || k == i) continue;
            const int dx = (int)(__ldcg(S.X + k) - Xi), dy = (int)(__ldcg(S.X + N + k) - Yi),
                      dz = (int)(__ldcg(S.X + 2 * N + k) - Zi);
            if (lattice_d2(dx, dy, dz) < a.r2) bits |= 1u << l;
        }
        inside[w] = bits;
    }
    __syncthreads();
    const int slot_new = (int)(s % M);
    // open origins: samples s-1 .. s-M+1 (those that exist), lags 1 .. M-1
    const int nopen = (int)(s < M - 1 ? s : M - 1);
    for (int w = threadIdx.x; w < a.WB; w += blockDim.x) {
        const unsigned in = inside[w];
        for (int lag = 1; lag <= nopen; ++lag) {
            const int o = (int)((s - lag) % M);
            const size_t base = ((size_t)o * a.NA + ci);
            unsigned al = a.alive[base * a.WB + w];
            if (al == 0u) continue;
            unsigned char *out = a.out + base * a.NB + 32 * (size_t)w;
            for (int l = 0; l < 32; ++l) {
                if (!((al >> l) & 1u)) continue;
                if ((in >> l) & 1u) {
                    out[l] = 0;
                } else if (++out[l] > a.t_star) {
                    al &= ~(1u << l);
                }
            }
            a.alive[base * a.WB + w] = al;
            const int c = __popc(al & in);
            if (c) atomicAdd(&count[o], c);
        }
    }
    // the new origin of this sample replaces the one that reached lag M
    int n0 = 0;
    for (int w = threadIdx.x; w < a.WB; w += blockDim.x) {
        const size_t base = ((size_t)slot_new * a.NA + ci);
        a.alive[base * a.WB + w] = inside[w];
        unsigned char *out = a.out + base * a.NB + 32 * (size_t)w;
        for (int l = 0; l < 32 && 32 * w + l < a.NB; ++l) out[l] = 0;
        n0 += __popc(inside[w]);
    }
    __syncthreads();
    if (threadIdx.x == 0) count[slot_new] = 0;
    __syncthreads();
    if (n0) atomicAdd(&count[slot_new], n0);
    __syncthreads();
    for (int o = threadIdx.x; o < M; o += blockDim.x) a.counts[(size_t)ci * M + o] = count[o];
    if (threadIdx.x == 0) a.n0[(size_t)slot_new * a.NA + ci] = count[slot_new];
}

// one block: per open origin (a thread each) the fractions of the NA centres in
// centre order, added to their lag; then the solvation sums and the counter
__global__ void __launch_bounds__(256) k_res_accum(ResArgs a) {
    const int M = a.M;
    const long long s = (long long)__ldcg(a.state + RES_SAMPLES);
    const int nopen = (int)(s < M - 1 ? s : M - 1);
    double *num = a.state + RES_HEAD, *cnt = num + M;
    for (int lag = threadIdx.x; lag <= nopen; lag += blockDim.x) {
        const int o = (int)((s - lag) % M);
        double f = 0.0, c = 0.0;
        for (int ci = 0; ci < a.NA; ++ci) {
            const int n0 = a.n0[(size_t)o * a.NA + ci];
            if (n0 == 0) continue;
            f += (double)a.counts[(size_t)ci * M + o] / (double)n0;
            c += 1.0;
        }
        num[lag] += f;
        cnt[lag] += c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int o = (int)(s % M);
        double ns = 0.0;
        for (int ci = 0; ci < a.NA; ++ci) ns += (double)a.n0[(size_t)o * a.NA + ci];
        a.state[RES_NSUM] += ns;
        a.state[RES_NCOUNT] += (double)a.NA;
        a.state[RES_SAMPLES] = (double)(s + 1);
    }
}

void ms2_launch_residence(cudaStream_t st, const SysParams *P, const DevSys &S, const ResArgs &a) {
    const size_t smem = sizeof(unsigned) * (size_t)a.WB + sizeof(int) * (size_t)a.M;
    k_res_update<<<a.NA, 256, smem, st>>>(P, S, a);
    k_res_accum<<<1, 256, 0, st>>>(a);
}

size_t ms2_residence_state_doubles(int M) { return RES_HEAD + 2 * (size_t)M; }
