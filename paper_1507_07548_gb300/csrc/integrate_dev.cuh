// Device helpers of the integrator shared by the single-system kernels
// (k_integrate.cu) and the batched per-system kernel (batch.cu).
#pragma once
#include "ms2_internal.cuh"

namespace integ {

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

// ------------------------------------------------------- rigid rotation
// q1 from q0 with space-frame angular momentum L held at its half-step value:
// implicit midpoint rule q1 = q0 + dt/2 * qm (x) (0, w_b), qm = (q0+q1)/2,
// w_b = I^-1 A(qm/|qm|)^T L, solved by `iters` fixed-point sweeps from q1 = q0,
// then normalised.  A(qm/|qm|) is taken in its homogeneous form
// A_h(qm) / |qm|^2 (the same matrix).  The sweeps evaluate the increment in
// FP32 (a ~1e-2 correction: ~1e-9 absolute error); it is added to the FP64
// quaternion, which is renormalised in FP64.
__device__ __forceinline__ void rotate_q(const double Iinv[3], const double q0[4], const double Lsp[3], double dt, int iters,
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
__device__ __forceinline__ void finish_step(const SysParams *__restrict__ P, const DevSys &S, int mode, const double *tot) {
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


}  // namespace integ
