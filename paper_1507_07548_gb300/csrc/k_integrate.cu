// K1 site build, K5 integration (velocity Verlet; leapfrog + quaternion implicit
// midpoint + isokinetic scaling) and K6 thermo reduction.
//
// FP64 is used for the state and the integrator.  GB300's FP64 rate is ~1/57 of
// its FP32 rate (~1.2 vs ~67 TFLOP/s measured), so these kernels are launched with
// small blocks that spread the per-molecule FP64 work over all SMs, and every
// system-wide sum is a fixed-order "last block" reduction (no float atomics, so
// results are bitwise reproducible).
#include "ms2_internal.cuh"

// ------------------------------------------------------------ site build
// lattice centre coordinates; space-frame FP32 site offsets and dipoles
__device__ __forceinline__ void build_one(const SysParams *__restrict__ P, const DevSys &S, int i) {
    const int N = S.N, NS = S.ns;
    const double lat = P->lat_scale;
    const double R0 = S.R[i], R1 = S.R[N + i], R2 = S.R[2 * N + i];
    S.X[i] = lattice_coord(R0, lat);
    S.X[N + i] = lattice_coord(R1, lat);
    S.X[2 * N + i] = lattice_coord(R2, lat);
    double A[9];
    rotmat(S.q[i], S.q[N + i], S.q[2 * N + i], S.q[3 * N + i], A);
    const int sp = S.species[i];
    const int nsp = P->n_sites[sp];
    double md[3] = {0, 0, 0};
    for (int a = 0; a < NS; ++a) {
        double o[3] = {0, 0, 0}, m[3] = {0, 0, 0};
        if (a < nsp) {
            const double *b = P->bpos[sp][a];
            const double *u = P->bdip[sp][a];
            for (int r = 0; r < 3; ++r) {
                o[r] = A[3 * r] * b[0] + A[3 * r + 1] * b[1] + A[3 * r + 2] * b[2];
                m[r] = A[3 * r] * u[0] + A[3 * r + 1] * u[1] + A[3 * r + 2] * u[2];
            }
        }
        for (int k = 0; k < 3; ++k) {
            S.s[(k * NS + a) * N + i] = (float)o[k];
            if (S.mu) S.mu[(k * NS + a) * N + i] = (float)m[k];
            if (a < nsp) md[k] += P->qd[sp][a] * o[k];
        }
    }
    if (S.mum)
        for (int k = 0; k < 3; ++k) S.mum[k * N + i] = (float)md[k];
}

__global__ void k_build(const SysParams *__restrict__ P, DevSys S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S.N) build_one(P, S, i);
}

// ------------------------------------------------------- rigid rotation
// q1 from q0 with space-frame angular momentum Lsp held at its half-step value:
// implicit midpoint rule q1 = q0 + dt/2 * qm (x) (0, w_b), qm = (q0+q1)/2,
// w_b = I^-1 A(qm/|qm|)^T L, solved by `iters` fixed-point sweeps from q1 = q0,
// then normalised.
__device__ void rotate_q(const double Iinv[3], const double q0[4], const double Lsp[3], double dt, int iters,
                         double q1[4]) {
    for (int k = 0; k < 4; ++k) q1[k] = q0[k];
    for (int it = 0; it < iters; ++it) {
        double qm[4];
        for (int k = 0; k < 4; ++k) qm[k] = 0.5 * (q0[k] + q1[k]);
        const double inv = 1.0 / sqrt(qm[0] * qm[0] + qm[1] * qm[1] + qm[2] * qm[2] + qm[3] * qm[3]);
        double A[9];
        rotmat(qm[0] * inv, qm[1] * inv, qm[2] * inv, qm[3] * inv, A);
        double w[3];
        for (int c = 0; c < 3; ++c) w[c] = Iinv[c] * (A[c] * Lsp[0] + A[3 + c] * Lsp[1] + A[6 + c] * Lsp[2]);
        // qm (x) (0, w)
        const double d0 = -qm[1] * w[0] - qm[2] * w[1] - qm[3] * w[2];
        const double d1 = qm[0] * w[0] + qm[2] * w[2] - qm[3] * w[1];
        const double d2 = qm[0] * w[1] - qm[1] * w[2] + qm[3] * w[0];
        const double d3 = qm[0] * w[2] + qm[1] * w[1] - qm[2] * w[0];
        const double h = 0.5 * dt;
        q1[0] = q0[0] + h * d0;
        q1[1] = q0[1] + h * d1;
        q1[2] = q0[2] + h * d2;
        q1[3] = q0[3] + h * d3;
    }
    const double inv = 1.0 / sqrt(q1[0] * q1[0] + q1[1] * q1[1] + q1[2] * q1[2] + q1[3] * q1[3]);
    for (int k = 0; k < 4; ++k) q1[k] *= inv;
}

// kinetic energies (mass units; divided by kconv in the final reduction)
__device__ __forceinline__ double ke_rot(const SysParams *__restrict__ P, int sp, const double A[9], double L0,
                                         double L1, double L2) {
    double e = 0;
    for (int c = 0; c < 3; ++c) {
        const double lb = A[c] * L0 + A[3 + c] * L1 + A[6 + c] * L2;
        e += P->Iinv[sp][c] * lb * lb;
    }
    return 0.5 * e;
}

// ------------------------------------------------------------- reduction
// reduction slots of the per-block partial sums
enum { R_ULJ = 0, R_UQQ, R_UDD, R_W, R_NP, R_KETR, R_KEROT, R_KETR1, R_KEROT1, R_WCORR, R_BAD, R_NRED_USED };

enum { RED_SUM = 1, RED_RECORD = 2, RED_KICK = 4, RED_HALFKICK = 8, RED_FP64PART = 16, RED_EWALD = 32 };

// final fixed-order sum of the block partials and the system scalars; run by
// the last block to finish
__device__ void finish_reduction(const SysParams *__restrict__ P, const DevSys &S, int mode, double *tot) {
    double *sc = S.scal;
    const double kc = P->kconv;
    if (mode & RED_SUM) {
        sc[SC_ULJ] = 0.5 * tot[R_ULJ];
        sc[SC_UQQ] = 0.5 * tot[R_UQQ];
        sc[SC_UDD] = 0.5 * tot[R_UDD];
        sc[SC_WPAIR] = 0.5 * tot[R_W];
        sc[SC_NPAIRS] = 0.5 * tot[R_NP];
        sc[SC_WREC_CORR] = (mode & RED_EWALD) ? tot[R_WCORR] : 0.0;
        sc[SC_UNSTABLE] = tot[R_BAD];
        const double U = sc[SC_ULJ] + sc[SC_UQQ] + sc[SC_UDD] + ((mode & RED_EWALD) ? sc[SC_UREC] : 0.0) +
                         sc[SC_UCONST] + sc[SC_ULRC];
        const double W = sc[SC_WPAIR] + ((mode & RED_EWALD) ? sc[SC_WREC_AT] - sc[SC_WREC_CORR] : 0.0) + sc[SC_WBG];
        sc[SC_UTOT] = U;
        sc[SC_WTOT] = W;
    }
    const double ketr = tot[R_KETR] / kc, kerot = tot[R_KEROT] / kc;
    sc[SC_KETR_NOW] = ketr;
    sc[SC_KEROT_NOW] = kerot;
    sc[SC_T] = 2.0 * (ketr + kerot) / P->ndof;
    sc[SC_P] = (2.0 * ketr / 3.0 + sc[SC_WTOT] / 3.0) / P->V + sc[SC_PLRC];
    if (mode & RED_RECORD) {
        double *ac = S.acc;
        ac[AC_N] += 1.0;
        ac[AC_U] += sc[SC_UTOT];
        ac[AC_P] += sc[SC_P];
        ac[AC_T] += sc[SC_T];
        ac[AC_BN] += 1.0;
        ac[AC_BU] += sc[SC_UTOT];
        ac[AC_BP] += sc[SC_P];
        if (ac[AC_BN] >= 100.0) {  // close a block of 100 steps
            const double bu = ac[AC_BU] / ac[AC_BN], bp = ac[AC_BP] / ac[AC_BN];
            ac[AC_NB] += 1.0;
            ac[AC_SBU] += bu;
            ac[AC_SBU2] += bu * bu;
            ac[AC_SBP] += bp;
            ac[AC_SBP2] += bp * bp;
            ac[AC_BN] = ac[AC_BU] = ac[AC_BP] = 0.0;
        }
    }
    if (mode & RED_KICK) {
        const double k1 = tot[R_KETR1] / kc, r1 = tot[R_KEROT1] / kc;
        const double Tp = 2.0 * (k1 + r1) / P->ndof;
        sc[SC_LAMBDA] = (P->thermostat && Tp > 0) ? sqrt(P->T0 / Tp) : 1.0;
    }
}

// Sums the pair partials (and Ewald site forces) into F, tau and per-molecule
// energies; records the kinetic energy of the stored velocities; optionally
// kicks the velocities with the new forces (leapfrog: full step, then the
// thermostat factor from the kicked kinetic energy; Verlet: half step).
__global__ void k_reduce(const SysParams *__restrict__ P, DevSys S, int mode) {
    const int N = S.N, i = blockIdx.x * blockDim.x + threadIdx.x;
    double r[R_NRED_USED];
    for (int k = 0; k < R_NRED_USED; ++k) r[k] = 0.0;
    if (i < N) {
        const int sp = S.species[i];
        double F[3], T[3];
        if (mode & RED_SUM) {
            double u[4] = {0, 0, 0, 0}, np = 0;
            for (int k = 0; k < 3; ++k) F[k] = T[k] = 0.0;
            for (int p = 0; p < S.jsplit; ++p) {
                if (mode & RED_FP64PART) {
                    const double *o = S.part64 + (size_t)p * MS2_NPV * N + i;
                    for (int k = 0; k < 3; ++k) { F[k] += o[(PV_FX + k) * N]; T[k] += o[(PV_TX + k) * N]; }
                    u[0] += o[PV_ULJ * N]; u[1] += o[PV_UQQ * N]; u[2] += o[PV_UDD * N]; u[3] += o[PV_W * N];
                    np += o[PV_NP * N];
                } else {
                    const float *o = S.part + (size_t)p * MS2_NPV * N + i;
                    for (int k = 0; k < 3; ++k) { F[k] += (double)o[(PV_FX + k) * N]; T[k] += (double)o[(PV_TX + k) * N]; }
                    u[0] += (double)o[PV_ULJ * N]; u[1] += (double)o[PV_UQQ * N]; u[2] += (double)o[PV_UDD * N];
                    u[3] += (double)o[PV_W * N];
                    np += (double)o[PV_NP * N];
                }
            }
            if (mode & RED_EWALD) {  // reciprocal-space site forces, summed over k chunks
                const int NS = S.ns, M = S.nsite_q;
                double wc = 0;
                for (int a = 0; a < NS; ++a) {
                    const int s = a * N + i;
                    double f[3] = {0, 0, 0};
                    for (int c = 0; c < S.kchunks; ++c)
                        for (int k = 0; k < 3; ++k) f[k] += (double)S.frec[((size_t)c * 3 + k) * M + s];
                    const double o0 = S.s[(0 * NS + a) * N + i], o1 = S.s[(1 * NS + a) * N + i],
                                 o2 = S.s[(2 * NS + a) * N + i];
                    F[0] += f[0]; F[1] += f[1]; F[2] += f[2];
                    T[0] += o1 * f[2] - o2 * f[1];
                    T[1] += o2 * f[0] - o0 * f[2];
                    T[2] += o0 * f[1] - o1 * f[0];
                    wc += f[0] * o0 + f[1] * o1 + f[2] * o2;
                }
                r[R_WCORR] = wc;
            }
            for (int k = 0; k < 3; ++k) { S.F[k * N + i] = F[k]; S.tau[k * N + i] = T[k]; }
            for (int k = 0; k < 4; ++k) S.Ui[k * N + i] = u[k];
            S.npart[i] = (int)np;
            r[R_ULJ] = u[0]; r[R_UQQ] = u[1]; r[R_UDD] = u[2]; r[R_W] = u[3]; r[R_NP] = np;
            const double fm = fmax(fabs(F[0]), fmax(fabs(F[1]), fabs(F[2])));
            r[R_BAD] = (fm < 1e30) ? 0.0 : 1.0;  // NaN fails the comparison too
        } else {
            for (int k = 0; k < 3; ++k) { F[k] = S.F[k * N + i]; T[k] = S.tau[k * N + i]; }
        }
        // kinetic energy of the stored velocities
        const double M = P->mass[sp];
        double v[3], L[3], A[9];
        for (int k = 0; k < 3; ++k) { v[k] = S.v[k * N + i]; L[k] = S.Lm[k * N + i]; }
        rotmat(S.q[i], S.q[N + i], S.q[2 * N + i], S.q[3 * N + i], A);
        r[R_KETR] = 0.5 * M * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        r[R_KEROT] = ke_rot(P, sp, A, L[0], L[1], L[2]);
        if (mode & (RED_KICK | RED_HALFKICK)) {
            const double h = (mode & RED_HALFKICK) ? 0.5 * P->dt : P->dt;
            const double cf = h * P->kconv / M, ct = h * P->kconv;
            for (int k = 0; k < 3; ++k) {
                v[k] += cf * F[k];
                L[k] += ct * T[k];
                S.v[k * N + i] = v[k];
                S.Lm[k * N + i] = L[k];
            }
            r[R_KETR1] = 0.5 * M * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            r[R_KEROT1] = ke_rot(P, sp, A, L[0], L[1], L[2]);
            if (mode & RED_HALFKICK) {  // Verlet: the recorded kinetic energy is the one at t + dt
                r[R_KETR] = r[R_KETR1];
                r[R_KEROT] = r[R_KEROT1];
            }
        }
    }
    // block reduction in fixed order: warp shuffles, then warp 0 over warps
    __shared__ double sred[32][R_NRED_USED];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int k = 0; k < R_NRED_USED; ++k) {
        double x = warp_sum(r[k]);
        if (k == R_BAD) x = x > 0 ? 1.0 : 0.0;
        if (lane == 0) sred[warp][k] = x;
    }
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) {
        double *blk = S.blk + (size_t)blockIdx.x * MS2_NRED;
        for (int k = 0; k < R_NRED_USED; ++k) {
            double x = 0;
            for (int w = 0; w < nw; ++w) x += sred[w][k];
            blk[k] = x;
        }
        __threadfence();
        const unsigned prev = atomicAdd(S.counter, 1u);
        last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double tot[MS2_NRED];
    if (threadIdx.x < R_NRED_USED) {
        double x = 0;
        for (int b = 0; b < (int)gridDim.x; ++b) x += ((volatile double *)S.blk)[(size_t)b * MS2_NRED + threadIdx.x];
        tot[threadIdx.x] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        finish_reduction(P, S, mode, tot);
        *S.counter = 0u;
    }
}

// ------------------------------------------------------------------ drift
// leapfrog: v, L *= lambda (thermostat); R += dt v; q <- rotate(q, L); rebuild
// Verlet  : v += dt/2 F/M; R += dt v; rebuild
__global__ void k_drift(const SysParams *__restrict__ P, DevSys S, int verlet) {
    const int N = S.N, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int sp = S.species[i];
    const double dt = P->dt;
    double v[3];
    if (verlet) {
        const double cf = 0.5 * dt * P->kconv / P->mass[sp];
        for (int k = 0; k < 3; ++k) {
            v[k] = S.v[k * N + i] + cf * S.F[k * N + i];
            S.v[k * N + i] = v[k];
        }
    } else {
        const double lam = S.scal[SC_LAMBDA];
        double L[3];
        for (int k = 0; k < 3; ++k) {
            v[k] = lam * S.v[k * N + i];
            L[k] = lam * S.Lm[k * N + i];
            S.v[k * N + i] = v[k];
            S.Lm[k * N + i] = L[k];
        }
        const double *Ii = P->Iinv[sp];
        if (Ii[0] != 0.0 || Ii[1] != 0.0 || Ii[2] != 0.0) {
            double q0[4] = {S.q[i], S.q[N + i], S.q[2 * N + i], S.q[3 * N + i]}, q1[4];
            rotate_q(Ii, q0, L, dt, P->quat_iters, q1);
            for (int k = 0; k < 4; ++k) S.q[k * N + i] = q1[k];
        }
    }
    for (int k = 0; k < 3; ++k) S.R[k * N + i] += dt * v[k];
    build_one(P, S, i);
}
