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

__device__ __forceinline__ double rsqrt_fp64(double x) {  // FP32 seed + two Newton steps (~1 ulp)
    double y = (double)rsqrtf((float)x);
    y = y * fma(-0.5 * x * y, y, 1.5);
    return y * fma(-0.5 * x * y, y, 1.5);
}

// ------------------------------------------------------------ site build
// lattice centre coordinate of component c; row c of the space-frame site
// offsets, dipoles and molecular charge dipole (lane c of a quad)
__device__ __forceinline__ void build_row(const SysParams *__restrict__ P, const DevSys &S, int i, int c,
                                          const double q[4]) {
    const int N = S.N, NS = S.ns;
    S.X[c * N + i] = lattice_coord(S.R[c * N + i], P->lat_scale);
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    double a0, a1, a2;  // row c of A(q)
    if (c == 0) { a0 = 1.0 - 2.0 * (y * y + z * z); a1 = 2.0 * (x * y - w * z); a2 = 2.0 * (x * z + w * y); }
    else if (c == 1) { a0 = 2.0 * (x * y + w * z); a1 = 1.0 - 2.0 * (x * x + z * z); a2 = 2.0 * (y * z - w * x); }
    else { a0 = 2.0 * (x * z - w * y); a1 = 2.0 * (y * z + w * x); a2 = 1.0 - 2.0 * (x * x + y * y); }
    const int sp = S.species[i], nsp = P->n_sites[sp];
    double md = 0.0;
    for (int a = 0; a < NS; ++a) {
        double o = 0.0, m = 0.0;
        if (a < nsp) {
            const double *b = P->bpos[sp][a], *u = P->bdip[sp][a];
            o = a0 * b[0] + a1 * b[1] + a2 * b[2];
            if (S.mu) m = a0 * u[0] + a1 * u[1] + a2 * u[2];
            md += P->qd[sp][a] * o;
        }
        S.s[(c * NS + a) * N + i] = (float)o;
        if (S.mu) S.mu[(c * NS + a) * N + i] = (float)m;
    }
    if (S.mum) S.mum[c * N + i] = (float)md;
}

// one quad per molecule: 4 lanes, lanes 0-2 build rows 0-2
__global__ void k_build(const SysParams *__restrict__ P, DevSys S) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x, i = t >> 2, c = t & 3;
    if (i >= S.N || c == 3) return;
    const int N = S.N;
    const double q[4] = {S.q[i], S.q[N + i], S.q[2 * N + i], S.q[3 * N + i]};
    build_row(P, S, i, c, q);
}

// ------------------------------------------------------- rigid rotation
// q1 from q0 with space-frame angular momentum L held at its half-step value:
// implicit midpoint rule q1 = q0 + dt/2 * qm (x) (0, w_b), qm = (q0+q1)/2,
// w_b = I^-1 A(qm/|qm|)^T L, solved by `iters` fixed-point sweeps from q1 = q0,
// then normalised.  A(qm/|qm|) is taken in its homogeneous form
// A_h(qm) / |qm|^2 (the same matrix).  The sweeps evaluate the increment in
// FP32 (a ~1e-2 correction: ~1e-9 absolute error); it is added to the FP64
// quaternion, which is renormalised in FP64.
__device__ void rotate_q(const double Iinv[3], const double q0[4], const double Lsp[3], double dt, int iters,
                         double q1[4]) {
    const float a0 = (float)q0[0], a1 = (float)q0[1], a2 = (float)q0[2], a3 = (float)q0[3];
    const float L0 = (float)Lsp[0], L1 = (float)Lsp[1], L2 = (float)Lsp[2];
    const float I0 = (float)Iinv[0], I1 = (float)Iinv[1], I2 = (float)Iinv[2], h = (float)(0.5 * dt);
    float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;  // increment q1 - q0
    for (int it = 0; it < iters; ++it) {
        const float w = a0 + 0.5f * d0, x = a1 + 0.5f * d1, y = a2 + 0.5f * d2, z = a3 + 0.5f * d3;
        const float ww = w * w, xx = x * x, yy = y * y, zz = z * z;
        const float inv = 1.0f / (ww + xx + yy + zz);
        const float xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y, wz = w * z;
        const float lb0 = (ww + xx - yy - zz) * L0 + 2.f * (xy + wz) * L1 + 2.f * (xz - wy) * L2;
        const float lb1 = 2.f * (xy - wz) * L0 + (ww - xx + yy - zz) * L1 + 2.f * (yz + wx) * L2;
        const float lb2 = 2.f * (xz + wy) * L0 + 2.f * (yz - wx) * L1 + (ww - xx - yy + zz) * L2;
        const float o0 = I0 * lb0 * inv, o1 = I1 * lb1 * inv, o2 = I2 * lb2 * inv;
        d0 = h * (-x * o0 - y * o1 - z * o2);
        d1 = h * (w * o0 + y * o2 - z * o1);
        d2 = h * (w * o1 - x * o2 + z * o0);
        d3 = h * (w * o2 + x * o1 - y * o0);
    }
    q1[0] = q0[0] + (double)d0;
    q1[1] = q0[1] + (double)d1;
    q1[2] = q0[2] + (double)d2;
    q1[3] = q0[3] + (double)d3;
    const double inv = rsqrt_fp64(q1[0] * q1[0] + q1[1] * q1[1] + q1[2] * q1[2] + q1[3] * q1[3]);
    for (int k = 0; k < 4; ++k) q1[k] *= inv;
}

// column c of A(q): the body component c of a space vector v is column_c . v
__device__ __forceinline__ void rot_column(const double q[4], int c, double col[3]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    if (c == 0) { col[0] = 1.0 - 2.0 * (y * y + z * z); col[1] = 2.0 * (x * y + w * z); col[2] = 2.0 * (x * z - w * y); }
    else if (c == 1) { col[0] = 2.0 * (x * y - w * z); col[1] = 1.0 - 2.0 * (x * x + z * z); col[2] = 2.0 * (y * z + w * x); }
    else { col[0] = 2.0 * (x * z + w * y); col[1] = 2.0 * (y * z - w * x); col[2] = 1.0 - 2.0 * (x * x + y * y); }
}

// ------------------------------------------------------------- reduction
enum { RED_SUM = 1, RED_RECORD = 2, RED_LAMBDA = 4, RED_HALFKICK = 8, RED_FP64PART = 16, RED_EWALD = 32 };
// per-step scalars: potential energy (pair part), virial (pair + reciprocal
// molecular correction), kinetic energy of the stored velocities (translation,
// rotation), kinetic energy after the kick, non-finite force flag
enum { Q_U = 0, Q_W, Q_KTR, Q_KROT, Q_K1, Q_BAD, Q_N };

// final fixed-order scalars of a step; run by the last block
__device__ void finish_step(const SysParams *__restrict__ P, const DevSys &S, int mode, const double *tot) {
    double *sc = S.scal;
    const double ikc = P->inv_kconv;
    if (mode & RED_SUM) {
        const double U = 0.5 * tot[Q_U] + ((mode & RED_EWALD) ? sc[SC_UREC] : 0.0) + sc[SC_UCONST] + sc[SC_ULRC];
        const double W = 0.5 * tot[Q_W] + ((mode & RED_EWALD) ? sc[SC_WREC_AT] : 0.0) + sc[SC_WBG];
        sc[SC_UTOT] = U;
        sc[SC_WTOT] = W;
        sc[SC_UNSTABLE] = tot[Q_BAD] > 0 ? 1.0 : 0.0;
    }
    const double ketr = tot[Q_KTR] * ikc, kerot = tot[Q_KROT] * ikc;
    sc[SC_KETR_NOW] = ketr;
    sc[SC_KEROT_NOW] = kerot;
    sc[SC_T] = 2.0 * (ketr + kerot) * P->inv_ndof;
    sc[SC_P] = (2.0 * ketr + sc[SC_WTOT]) * (1.0 / 3.0) * P->inv_V + sc[SC_PLRC];
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
            const double bu = ac[AC_BU] * 0.01, bp = ac[AC_BP] * 0.01;
            ac[AC_NB] += 1.0;
            ac[AC_SBU] += bu;
            ac[AC_SBU2] += bu * bu;
            ac[AC_SBP] += bp;
            ac[AC_SBP2] += bp * bp;
            ac[AC_BN] = ac[AC_BU] = ac[AC_BP] = 0.0;
        }
    }
    if (mode & RED_LAMBDA) {  // isokinetic factor sqrt(T0 / T') for the next drift
        const double x = 2.0 * tot[Q_K1] * ikc * P->inv_ndof * P->inv_T0;
        sc[SC_LAMBDA] = (P->thermostat && x > 0) ? rsqrt_fp64(x) : 1.0;
    }
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
