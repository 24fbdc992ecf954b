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
    build_row(P, S, i, c, q);
}

// Sums the pair partials (and Ewald site forces) into F, tau and per-molecule
// energies; the kinetic energy of the stored velocities.  Leapfrog
// (RED_LAMBDA): also the kinetic energy the velocities will have after the kick
// with these forces, hence the thermostat factor the next drift applies.
// Verlet (RED_HALFKICK): applies the second half kick.  One quad per molecule,
// 32 molecules per block.
__global__ void __launch_bounds__(128) k_reduce(const SysParams *__restrict__ P, DevSys S, int mode) {
    __shared__ double sh_f[32][3 * MS2_MAXS];   // Ewald site forces of the block's molecules
    __shared__ double sh_t[32][3];               // torques (for the kicked rotational energy)
    const int N = S.N, tq = threadIdx.x >> 2, c = threadIdx.x & 3;
    const int i = blockIdx.x * (blockDim.x >> 2) + tq;
    const bool on = i < N;
    const int ii = on ? i : 0;
    double r[Q_N] = {0, 0, 0, 0, 0, 0};
    const int sp = S.species[ii];
    double Fc = 0, Tc = 0;
    if (mode & RED_SUM) {
        // force / torque component c on lanes 0-2; energies and virial on lane 3
        if (c < 3) {
            for (int p = 0; p < S.jsplit; ++p) {
                if (mode & RED_FP64PART) {
                    const double *o = S.part64 + (size_t)p * MS2_NPV * N + ii;
                    Fc += o[(PV_FX + c) * N];
                    Tc += o[(PV_TX + c) * N];
                } else {
                    const float *o = S.part + (size_t)p * MS2_NPV * N + ii;
                    Fc += (double)o[(PV_FX + c) * N];
                    Tc += (double)o[(PV_TX + c) * N];
                }
            }
        } else {
            double u[4] = {0, 0, 0, 0}, np = 0;
            for (int p = 0; p < S.jsplit; ++p) {
                if (mode & RED_FP64PART) {
                    const double *o = S.part64 + (size_t)p * MS2_NPV * N + ii;
                    u[0] += o[PV_ULJ * N]; u[1] += o[PV_UQQ * N]; u[2] += o[PV_UDD * N]; u[3] += o[PV_W * N];
                    np += o[PV_NP * N];
                } else {
                    const float *o = S.part + (size_t)p * MS2_NPV * N + ii;
                    u[0] += (double)o[PV_ULJ * N]; u[1] += (double)o[PV_UQQ * N]; u[2] += (double)o[PV_UDD * N];
                    u[3] += (double)o[PV_W * N];
                    np += (double)o[PV_NP * N];
                }
            }
            r[Q_U] = u[0] + u[1] + u[2];
            r[Q_W] = u[3];
            if (on) {
                for (int k = 0; k < 4; ++k) S.Ui[k * N + i] = u[k];
                S.npart[i] = (int)np;
            }
        }
        if (mode & RED_EWALD) {  // reciprocal-space site forces, summed over k chunks
            const int NS = S.ns, M = S.nsite_q;
            if (c < 3)
                for (int a = 0; a < NS; ++a) {
                    double f = 0;
                    for (int ch = 0; ch < S.kchunks; ++ch) f += (double)S.frec[((size_t)ch * 3 + c) * M + a * N + ii];
                    sh_f[tq][3 * a + c] = f;
                    Fc += f;
                }
            __syncwarp();
            double wc = 0;
            if (c < 3) {  // torque component c and the molecular-virial correction -F_s.s_s
                const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
                for (int a = 0; a < NS; ++a) {
                    const double o1 = S.s[(c1 * NS + a) * N + ii], o2 = S.s[(c2 * NS + a) * N + ii];
                    const double oc = S.s[(c * NS + a) * N + ii];
                    Tc += o1 * sh_f[tq][3 * a + c2] - o2 * sh_f[tq][3 * a + c1];
                    wc += oc * sh_f[tq][3 * a + c];
                }
                r[Q_W] = -2.0 * wc;  // pair virial sums are halved at the end
            }
            // per-molecule reciprocal virial correction for the on-demand breakdown
            const double w0 = __shfl_sync(0xffffffffu, wc, (threadIdx.x & 28) | 0);
            const double w1 = __shfl_sync(0xffffffffu, wc, (threadIdx.x & 28) | 1);
            const double w2 = __shfl_sync(0xffffffffu, wc, (threadIdx.x & 28) | 2);
            if (c == 3 && on) S.wcorr[i] = w0 + w1 + w2;
        }
        if (c < 3 && on) {
            S.F[c * N + i] = Fc;
            S.tau[c * N + i] = Tc;
        }
        r[Q_BAD] = (c < 3 && !(fabs(Fc) < 1e30)) ? 1.0 : 0.0;  // NaN fails the comparison too
    } else if (c < 3) {
        Fc = S.F[c * N + ii];
        Tc = S.tau[c * N + ii];
    }
    if (c < 3) sh_t[tq][c] = Tc;
    __syncwarp();
    // kinetic energies: lane c takes component c of v and body component c of L
    if (c < 3) {
        const double M = P->mass[sp], Ii = P->Iinv[sp][c];
        const double q[4] = {S.q[ii], S.q[N + ii], S.q[2 * N + ii], S.q[3 * N + ii]};
        double col[3], L[3];
        rot_column(q, c, col);
        for (int k = 0; k < 3; ++k) L[k] = S.Lm[k * N + ii];
        double v = S.v[c * N + ii];
        const double lb = col[0] * L[0] + col[1] * L[1] + col[2] * L[2];
        r[Q_KTR] = 0.5 * M * v * v;
        r[Q_KROT] = 0.5 * Ii * lb * lb;
        if (mode & (RED_LAMBDA | RED_HALFKICK)) {
            const double h = (mode & RED_HALFKICK) ? 0.5 * P->dt : P->dt;
            const double ct = h * P->kconv;
            v += ct * P->inv_mass[sp] * Fc;
            const double lb1 = lb + ct * (col[0] * sh_t[tq][0] + col[1] * sh_t[tq][1] + col[2] * sh_t[tq][2]);
            r[Q_K1] = 0.5 * M * v * v + 0.5 * Ii * lb1 * lb1;
            if (mode & RED_HALFKICK) {  // Verlet: velocities at t + dt, recorded
                if (on) S.v[c * N + i] = v;
                r[Q_KTR] = 0.5 * M * v * v;
            }
        }
    }
    if (!on)
        for (int k = 0; k < Q_N; ++k) r[k] = 0.0;
    // block reduction (fixed shuffle tree), then the last block over blocks
    __shared__ double sred[4][Q_N];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int k = 0; k < Q_N; ++k) {
        const double x = warp_sum(r[k]);
        if (lane == 0) sred[warp][k] = x;
    }
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x < Q_N) {
        double x = 0;
        for (int w = 0; w < nw; ++w) x += sred[w][threadIdx.x];
        S.blk[(size_t)blockIdx.x * MS2_NRED + threadIdx.x] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(S.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double tot[MS2_NRED];
    if (warp == 0) {
        for (int k = 0; k < Q_N; ++k) {
            double x = 0;
            for (int b = lane; b < (int)gridDim.x; b += 32) x += __ldcg(S.blk + (size_t)b * MS2_NRED + k);
            x = warp_sum(x);
            if (lane == 0) tot[k] = x;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        finish_step(P, S, mode, tot);
        *S.counter = 0u;
    }
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
// One quad per molecule.  Lanes 0-2, component c:
//   leapfrog: v_c <- lambda (v_c + dt F_c/M) (kick + isokinetic scaling with the
//             factor from the last reduction), R_c += dt v_c;
//   Verlet  : v_c += dt/2 F_c/M, R_c += dt v_c;
// lane 3 (leapfrog): L <- lambda (L + dt tau), q <- rotate(q, L).  Then lanes 0-2
// rebuild lattice coordinate c and row c of the site offsets.
__global__ void __launch_bounds__(128) k_drift(const SysParams *__restrict__ P, DevSys S, int verlet) {
    const int N = S.N, t = blockIdx.x * blockDim.x + threadIdx.x, i = t >> 2, c = t & 3;
    const bool on = i < N;
    const int ii = on ? i : 0;
    const int sp = S.species[ii];
    const double dt = P->dt;
    double q[4] = {S.q[ii], S.q[N + ii], S.q[2 * N + ii], S.q[3 * N + ii]};
    if (verlet) {
        if (c < 3 && on) {
            const double v = S.v[c * N + i] + 0.5 * dt * P->kconv * P->inv_mass[sp] * S.F[c * N + i];
            S.v[c * N + i] = v;
            S.R[c * N + i] += dt * v;
        }
    } else {
        const double lam = S.scal[SC_LAMBDA];
        if (c < 3) {
            if (on) {
                const double v = lam * (S.v[c * N + i] + dt * P->kconv * P->inv_mass[sp] * S.F[c * N + i]);
                S.v[c * N + i] = v;
                S.R[c * N + i] += dt * v;
            }
        } else {
            const double ct = dt * P->kconv;
            double L[3];
            for (int k = 0; k < 3; ++k) {
                L[k] = lam * (S.Lm[k * N + ii] + ct * S.tau[k * N + ii]);
                if (on) S.Lm[k * N + i] = L[k];
            }
            const double *Ii = P->Iinv[sp];
            if (Ii[0] != 0.0 || Ii[1] != 0.0 || Ii[2] != 0.0) {
                double q1[4];
                rotate_q(Ii, q, L, dt, P->quat_iters, q1);
                for (int k = 0; k < 4; ++k) {
                    q[k] = q1[k];
                    if (on) S.q[k * N + i] = q1[k];
                }
            }
        }
        for (int k = 0; k < 4; ++k) q[k] = __shfl_sync(0xffffffffu, q[k], (threadIdx.x & 28) | 3);
    }
    if (c < 3 && on) build_row(P, S, i, c, q);
}
