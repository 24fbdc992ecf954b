// K1 site build, K5 integration (velocity Verlet; leapfrog + quaternion implicit
// midpoint + isokinetic scaling) and K6 thermo reduction.
//
// FP64 holds the state and every accumulation (R, v, q, L, F, tau, energy and
// virial sums).  On GB300 one warp sees ~1/4 of an SM's small FP64 unit: a
// dependent FP64 instruction costs ~70 cycles whatever the number of active
// lanes.  So each molecule is handled by a quad of lanes (lanes 0-2: the x, y, z
// components; lane 3: the rotation), no FP64 divide or square root runs per
// step (host-side reciprocals, Newton rsqrt from an FP32 seed), the rotation
// increment of the implicit-midpoint sweeps is evaluated in FP32 and added to
// the FP64 quaternion, and a step reduces only the five scalars it needs; the
// energy breakdown is summed on demand.  All system-wide sums are fixed-order
// "last block" reductions (no float atomics: bitwise reproducible).
#include "ms2_internal.cuh"

#include "integrate_dev.cuh"

using namespace integ;

// one quad per molecule: 4 lanes, lanes 0-2 build rows 0-2
__global__ void k_build(const SysParams *__restrict__ P, DevSys S) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x, i = t >> 2, c = t & 3;
    if (i >= S.N || c == 3) return;
    const int N = S.N;
    const double q[4] = {S.q[i], S.q[N + i], S.q[2 * N + i], S.q[3 * N + i]};
    build_row(P, S, i, c, q, S.R[c * N + i], S.species[i]);
}

// Sums the pair partials (and Ewald site forces) into F, tau and per-molecule
// energies; the kinetic energy of the stored velocities.  Leapfrog
// (RED_LAMBDA): also the kinetic energy the velocities will have after the kick
// with these forces, hence the thermostat factor the next drift applies.
// Verlet (RED_HALFKICK): applies the second half kick.  One warp per reduction
// unit (a contiguous molecule range, a quad per molecule), 4 units per block;
// the last block sums the units in fixed order and finishes the step.
__global__ void __launch_bounds__(128) k_reduce(const SysParams *__restrict__ P, DevSys S, int mode) {
    const int lane = threadIdx.x & 31, u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (u < S.nunits) reduce_unit<false>(P, S, global_io(S), mode, u, S.nunits, lane);
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(S.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double tot[MS2_NRED];
    reduce_totals(S, S.nunits, tot, (mode & RED_GK) ? Q_N + 3 : Q_N);
    __syncthreads();
    if (threadIdx.x < 32) finish_step_warp(P, S, mode, tot, threadIdx.x, S.acc, global_consts(S));
    if (threadIdx.x == 0) *S.counter = 0u;
    if ((mode & RED_GK) && threadIdx.x < 32) gk_update(S, tot, threadIdx.x);
}

// Heat flux of a sampled step (after k_reduce and the power pass k_heat): one
// warp per reduction unit (integ::heat_unit); the last block records the sample.
__global__ void __launch_bounds__(128) k_heat_reduce(const SysParams *__restrict__ P, DevSys S) {
    const int lane = threadIdx.x & 31, u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (u < S.nunits) heat_unit<false>(P, S, S.hpart, S.N, global_view(S), S.Ui, S.N, 0, u, S.nunits, lane);
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(S.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < 32) heat_record(S, S.nunits, threadIdx.x);
    __syncthreads();
    if (threadIdx.x == 0) *S.counter = 0u;
}

// On-demand breakdown of the current configuration (single block, fixed order):
// out[0..5] = sums of U_lj, U_qq, U_dd, W_pair (owner-doubled), partner counts,
// and the reciprocal molecular-virial correction sum_s F_s.s_s.
__global__ void k_terms(const SysParams *__restrict__ P, DevSys S, double *out) {
    __shared__ double sh[256][6];
    const int N = S.N;
    double a[6] = {0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        for (int k = 0; k < 3; ++k) a[k] += S.Ui[k * N + i];
        a[4] += S.npart[i];
        if (S.wcorr) a[5] += S.wcorr[i];
    }
    for (int k = 0; k < 6; ++k) sh[threadIdx.x][k] = a[k];
    __syncthreads();
    if (threadIdx.x < 6) {
        double x = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) x += sh[t][threadIdx.x];
        out[threadIdx.x] = x;
    }
}

// ------------------------------------------------------------------ drift
// One quad per molecule (drift_quad): kick with the forces of the last
// reduction and the thermostat factor it left in SC_LAMBDA, drift, rotation,
// then the site build for the new configuration.
__global__ void __launch_bounds__(128) k_drift(const SysParams *__restrict__ P, DevSys S, int verlet) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x, i = t >> 2;
    const double lam = verlet ? 1.0 : S.scal[SC_LAMBDA];
    drift_quad<false>(P, S, global_view(S), i, i, i < S.N, t & 3, verlet != 0, lam);
}
