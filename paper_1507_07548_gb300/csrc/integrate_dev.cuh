// Device helpers of the integrator shared by the single-system kernels
// (k_integrate.cu) and the batched per-system kernel (batch.cu).
#pragma once
#include "ms2_internal.cuh"
#include "ewald_dev.cuh"

namespace integ {

__device__ __forceinline__ double rsqrt_fp64(double x) {  // FP32 seed + two Newton steps (~1 ulp)
    double y = f2d(rsqrtf(d2f(x)));
    y = y * fma(-0.5 * x * y, y, 1.5);
    return y * fma(-0.5 * x * y, y, 1.5);
}

// ------------------------------------------------------------ site build
// row c of A(q) for the cyclic order (c, c1, c2), with v = (x, y, z):
//   A[c][c] = 1 - 2 (v_c1^2 + v_c2^2), A[c][c1] = 2 (v_c v_c1 - w v_c2),
//   A[c][c2] = 2 (v_c v_c2 + w v_c1)
// (one instruction stream for the three lanes: no branch on c)
__device__ __forceinline__ void rot_row(const double q[4], int c, double &acc, double &ac1, double &ac2) {
    const double w = q[0];
    const double vc = c == 0 ? q[1] : (c == 1 ? q[2] : q[3]);
    const double v1 = c == 0 ? q[2] : (c == 1 ? q[3] : q[1]);
    const double v2 = c == 0 ? q[3] : (c == 1 ? q[1] : q[2]);
    acc = 1.0 - 2.0 * (v1 * v1 + v2 * v2);
    ac1 = 2.0 * (vc * v1 - w * v2);
    ac2 = 2.0 * (vc * v2 + w * v1);
}

// component c of the space-frame offset o and dipole m of site a of species sp
// (0 where a is not one of its sites), from row c of A(q)
__device__ __forceinline__ void site_row(const SysParams *__restrict__ P, int sp, int a, int c, double acc, double ac1,
                                         double ac2, bool dip, double &o, double &m) {
    const int c1 = c == 2 ? 0 : c + 1, c2 = c == 0 ? 2 : c - 1;
    o = 0.0;
    m = 0.0;
    if (a < P->n_sites[sp]) {
        const double *b = P->bpos[sp][a], *u = P->bdip[sp][a];
        o = acc * b[c] + ac1 * b[c1] + ac2 * b[c2];
        if (dip) m = acc * u[c] + ac1 * u[c1] + ac2 * u[c2];
    }
}

// lattice centre coordinate of component c; row c of the space-frame site
// offsets, dipoles and molecular charge dipole (lane c of a quad)
__device__ __forceinline__ void build_row(const SysParams *__restrict__ P, const DevSys &S, int i, int c,
                                          const double q[4], double Rc, int sp) {
    const int N = S.N, NS = S.ns;
    S.X[c * N + i] = lattice_coord(Rc, P->lat_scale);
    double acc, ac1, ac2;
    rot_row(q, c, acc, ac1, ac2);
    const int nsp = P->n_sites[sp];
    if (P->point[sp]) {  // sites and dipoles at the centre: the offsets are zero in every orientation
        for (int a = 0; a < NS; ++a) {
            S.s[(c * NS + a) * N + i] = 0.f;
            if (S.mu) S.mu[(c * NS + a) * N + i] = 0.f;
        }
        if (S.mum) S.mum[c * N + i] = 0.f;
        return;
    }
    double md = 0.0;
    for (int a = 0; a < NS; ++a) {
        double o, m;
        site_row(P, sp, a, c, acc, ac1, ac2, S.mu != nullptr, o, m);
        if (a < nsp) md += P->qd[sp][a] * o;
        S.s[(c * NS + a) * N + i] = d2f(o);
        if (S.mu) S.mu[(c * NS + a) * N + i] = d2f(m);
    }
    if (S.mum) S.mum[c * N + i] = d2f(md);
}

// build_row split by site, for a warp per site: site a's offset and dipole rows
// (returns the offset for build_md); the lattice coordinate is left to the caller
__device__ __forceinline__ double build_site(const SysParams *__restrict__ P, const DevSys &S, int i, int c,
                                             const double q[4], int sp, int a) {
    const int N = S.N, NS = S.ns;
    double o = 0.0, m = 0.0;
    if (!P->point[sp]) {
        double acc, ac1, ac2;
        rot_row(q, c, acc, ac1, ac2);
        site_row(P, sp, a, c, acc, ac1, ac2, S.mu != nullptr, o, m);
    }
    S.s[(c * NS + a) * N + i] = d2f(o);
    if (S.mu) S.mu[(c * NS + a) * N + i] = d2f(m);
    return o;
}

// the molecular charge dipole of build_row from the site offsets od[a] of build_site
__device__ __forceinline__ void build_md(const SysParams *__restrict__ P, const DevSys &S, int i, int c, int sp,
                                         const double *od, int ostride) {
    if (!S.mum) return;
    const int N = S.N, NS = S.ns, nsp = P->n_sites[sp];
    double md = 0.0;
    if (!P->point[sp])
        for (int a = 0; a < NS; ++a)
            if (a < nsp) md += P->qd[sp][a] * od[a * ostride];
    S.mum[c * N + i] = d2f(md);
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
    const float a0 = d2f(q0[0]), a1 = d2f(q0[1]), a2 = d2f(q0[2]), a3 = d2f(q0[3]);
    const float L0 = d2f(Lsp[0]), L1 = d2f(Lsp[1]), L2 = d2f(Lsp[2]);
    const float I0 = d2f(Iinv[0]), I1 = d2f(Iinv[1]), I2 = d2f(Iinv[2]), h = d2f(0.5 * dt);
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
    q1[0] = q0[0] + f2d(d0);
    q1[1] = q0[1] + f2d(d1);
    q1[2] = q0[2] + f2d(d2);
    q1[3] = q0[3] + f2d(d3);
    const double inv = rsqrt_fp64(q1[0] * q1[0] + q1[1] * q1[1] + q1[2] * q1[2] + q1[3] * q1[3]);
    for (int k = 0; k < 4; ++k) q1[k] *= inv;
}

// rotate_q for the 4 lanes of a quad (lane c = component c): the FP32 sweeps run
// in every lane (identical), the FP64 update and normalisation one component
// per lane (the norm by a quad shuffle tree whose result is the same in all 4
// lanes); returns q1[c].  The normalisation 1/|q1| = (1 + e)^-1/2,
// e = |q1|^2 - 1, takes the series 1 - e/2 + 3e^2/8 - 5e^3/16 + 35e^4/128
// (error below 63/256 e^5, under 1e-20 for |e| < 1e-4) and rsqrt_fp64 beyond.
__device__ __forceinline__ double rotate_q_quad(const double Iinv[3], const double q0[4], const double Lsp[3],
                                                double dt, int iters, int c) {
    const float a0 = d2f(q0[0]), a1 = d2f(q0[1]), a2 = d2f(q0[2]), a3 = d2f(q0[3]);
    const float L0 = d2f(Lsp[0]), L1 = d2f(Lsp[1]), L2 = d2f(Lsp[2]);
    const float I0 = d2f(Iinv[0]), I1 = d2f(Iinv[1]), I2 = d2f(Iinv[2]), h = d2f(0.5 * dt);
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
    const float dc = c == 0 ? d0 : (c == 1 ? d1 : (c == 2 ? d2 : d3));
    const double qc = (c == 0 ? q0[0] : (c == 1 ? q0[1] : (c == 2 ? q0[2] : q0[3]))) + f2d(dc);
    double n2 = qc * qc;
    n2 += __shfl_xor_sync(0xffffffffu, n2, 1);
    n2 += __shfl_xor_sync(0xffffffffu, n2, 2);
    const double e = n2 - 1.0;
    double inv;
    if (fabs(e) < 1e-4)
        inv = fma(e, fma(e, fma(e, fma(e, 35.0 / 128.0, -5.0 / 16.0), 3.0 / 8.0), -0.5), 1.0);
    else
        inv = rsqrt_fp64(n2);
    return qc * inv;
}

// column c of A(q): the body component c of a space vector u is column_c . u.
// For the cyclic order (c, c1, c2): A[c][c] = 1 - 2 (v_c1^2 + v_c2^2),
// A[c1][c] = 2 (v_c1 v_c + w v_c2), A[c2][c] = 2 (v_c2 v_c - w v_c1); the
// entries come back in space order (no branch on c).
__device__ __forceinline__ void rot_column(const double q[4], int c, double col[3]) {
    const double w = q[0];
    const double vc = c == 0 ? q[1] : (c == 1 ? q[2] : q[3]);
    const double v1 = c == 0 ? q[2] : (c == 1 ? q[3] : q[1]);
    const double v2 = c == 0 ? q[3] : (c == 1 ? q[1] : q[2]);
    const double acc = 1.0 - 2.0 * (v1 * v1 + v2 * v2), a1c = 2.0 * (v1 * vc + w * v2), a2c = 2.0 * (v2 * vc - w * v1);
    col[0] = c == 0 ? acc : (c == 1 ? a2c : a1c);
    col[1] = c == 0 ? a1c : (c == 1 ? acc : a2c);
    col[2] = c == 0 ? a2c : (c == 1 ? a1c : acc);
}

// ------------------------------------------------------------- reduction
// reduction modes (RED_*) are in ms2_internal.cuh
// per-step scalars: potential energy (pair part), virial (pair + reciprocal
// molecular correction), kinetic energy of the stored velocities (translation,
// rotation), kinetic energy after the kick, non-finite force flag
enum { Q_U = 0, Q_W, Q_KTR, Q_KROT, Q_K1, Q_BAD, Q_VV, Q_N };  // Q_VV: d2U/dV2 owner sums

// Final fixed-order scalars of a step (potential energy, virial, T, P, the
// running averages, the next thermostat factor), by a whole warp: every lane
// calls it.  The scalars are formed on one instruction stream with
// lane-selected operands, so that independent values share FP64 instructions
// (an FP64 warp instruction costs an SMSP the same for one active lane or 32):
// lanes 0-3 form U, W and the kinetic energies, lanes 0-1 T and P, and lane
// k < AC_COUNT_ updates running sum k as acc_k + f_k g_k.  Every path calls
// this one function, so they agree to the bit.  acc holds the running sums and
// kc the launch constants (U_const, U_lrc, W_bg, P_lrc): S.acc and global_consts
// on the per-phase paths, a block's shared-memory copies in the fused step.
struct StepConsts {
    double uconst, ulrc, wbg, plrc;
};
__device__ __forceinline__ StepConsts global_consts(const DevSys &S) {
    return StepConsts{S.scal[SC_UCONST], S.scal[SC_ULRC], S.scal[SC_WBG], S.scal[SC_PLRC]};
}
__device__ __forceinline__ void finish_step_warp(const SysParams *__restrict__ P, const DevSys &S, int mode,
                                                 const double *tot, int lane, double *acc, const StepConsts &kc) {
    const unsigned FM = 0xffffffffu;
    double *sc = S.scal;
    const bool sum = mode & RED_SUM, ew = mode & RED_EWALD, ms = sum && P->massieu, rec = mode & RED_RECORD;
    const double plrc = kc.plrc;
    // U = 0.5 t_U + urec + uconst + ulrc,  W = 0.5 t_W + wrec + wbg,  K = t_K / kconv
    double m = 0.0, t = 0.0, p = 0.0, q = 0.0, r = 0.0;
    if (lane == 0) { m = 0.5; t = tot[Q_U]; p = ew ? sc[SC_UREC] : 0.0; q = kc.uconst; r = kc.ulrc; }
    if (lane == 1) { m = 0.5; t = tot[Q_W]; p = ew ? sc[SC_WREC_AT] : 0.0; q = kc.wbg; }
    if (lane == 2) { m = tot[Q_KTR]; t = P->inv_kconv; }
    if (lane == 3) { m = tot[Q_KROT]; t = P->inv_kconv; }
    double v = (fma(m, t, p) + q) + r;
    double U = __shfl_sync(FM, v, 0), W = __shfl_sync(FM, v, 1);
    const double ketr = __shfl_sync(FM, v, 2), kerot = __shfl_sync(FM, v, 3);
    if (!sum) {  // the stored configuration scalars
        U = sc[SC_UTOT];
        W = sc[SC_WTOT];
    }
    // T = (2 (K_tr + K_rot)) / ndof on lane 0, P = (2 K_tr + W) / (3 V) + P_lrc on lane 1
    const double c1 = lane == 1 ? 2.0 : 1.0, c2 = lane == 1 ? W : kerot;
    const double k1 = lane == 1 ? (1.0 / 3.0) : 2.0, k2 = lane == 1 ? P->inv_V : P->inv_ndof, k3 = lane == 1 ? plrc : 0.0;
    const double tp = fma(k1 * fma(c1, ketr, c2), k2, k3);
    const double T = __shfl_sync(FM, tp, 0), Pr = __shfl_sync(FM, tp, 1);
    double UV = 0.0, UVV = 0.0;
    if (ms) {  // volume derivatives of this configuration (Sec. 2, Eq. 1)
        UV = fma(-W * (1.0 / 3.0), P->inv_V, -plrc);
        UVV = fma(0.5 * tot[Q_VV] * (1.0 / 9.0) * P->inv_V, P->inv_V, 2.0 * plrc * P->inv_V);
    } else if (rec && P->massieu) {
        UV = sc[SC_UV];
        UVV = sc[SC_UVV];
    }
    double lam = 1.0;
    if (mode & RED_LAMBDA) {  // isokinetic factor sqrt(T0 / T') for the next drift (as lambda_of)
        const double x = P->lam_c * tot[Q_K1];
        lam = (P->thermostat && x > 0) ? rsqrt_fp64(x) : 1.0;
    }
    if (rec) {
        double a = lane < AC_COUNT_ ? acc[lane] : 0.0;
        double f = 0.0, g = 0.0;
        if (lane == AC_N || lane == AC_BN) { f = 1.0; g = 1.0; }
        if (lane == AC_U || lane == AC_BU) { f = 1.0; g = U; }
        if (lane == AC_P || lane == AC_BP) { f = 1.0; g = Pr; }
        if (lane == AC_T) { f = 1.0; g = T; }
        if (P->massieu) {  // Massieu-derivative moments, shifted by the first sample
            const double mn = __shfl_sync(FM, a, AC_MN);
            const double mu0 = mn == 0.0 ? U : __shfl_sync(FM, a, AC_MU0);
            const double mv0 = mn == 0.0 ? UV : __shfl_sync(FM, a, AC_MV0);
            if (lane == AC_MU0) a = mu0;
            if (lane == AC_MV0) a = mv0;
            const double x = U - mu0, y = UV - mv0, w = UVV, xx = x * x, xy = x * y;
            if (lane == AC_MN) { f = 1.0; g = 1.0; }
            if (lane == AC_MX) { f = 1.0; g = x; }
            if (lane == AC_MX2) { f = x; g = x; }
            if (lane == AC_MX3) { f = xx; g = x; }
            if (lane == AC_MY) { f = 1.0; g = y; }
            if (lane == AC_MY2) { f = y; g = y; }
            if (lane == AC_MXY) { f = x; g = y; }
            if (lane == AC_MX2Y) { f = xx; g = y; }
            if (lane == AC_MXY2) { f = xy; g = y; }
            if (lane == AC_MW) { f = 1.0; g = w; }
            if (lane == AC_MXW) { f = x; g = w; }
        }
        a = fma(f, g, a);
        if (__shfl_sync(FM, a, AC_BN) >= 100.0) {  // close a block of 100 steps
            const double bu = __shfl_sync(FM, a, AC_BU) * 0.01, bp = __shfl_sync(FM, a, AC_BP) * 0.01;
            double f2 = 0.0, g2 = 0.0;
            if (lane == AC_NB) { f2 = 1.0; g2 = 1.0; }
            if (lane == AC_SBU) { f2 = 1.0; g2 = bu; }
            if (lane == AC_SBU2) { f2 = bu; g2 = bu; }
            if (lane == AC_SBP) { f2 = 1.0; g2 = bp; }
            if (lane == AC_SBP2) { f2 = bp; g2 = bp; }
            a = fma(f2, g2, a);
            if (lane == AC_BN || lane == AC_BU || lane == AC_BP) a = 0.0;
        }
        if (lane < AC_COUNT_) acc[lane] = a;
    }
    if (lane == 0) {
        if (sum) {
            sc[SC_UTOT] = U;
            sc[SC_WTOT] = W;
            sc[SC_UNSTABLE] = tot[Q_BAD] > 0 ? 1.0 : 0.0;
        }
        if (ms) {
            sc[SC_UV] = UV;
            sc[SC_UVV] = UVV;
        }
        if (mode & RED_GK) {
            sc[SC_JX] = tot[Q_N];
            sc[SC_JY] = tot[Q_N + 1];
            sc[SC_JZ] = tot[Q_N + 2];
        }
        sc[SC_KETR_NOW] = ketr;
        sc[SC_KEROT_NOW] = kerot;
        sc[SC_T] = T;
        sc[SC_P] = Pr;
        if (mode & RED_LAMBDA) sc[SC_LAMBDA] = lam;
    }
}

// ------------------------------------------------------ one step, per quad
// Per-molecule state as seen by a kernel: component c of molecule m at
// [c * ld + m] (global arrays: ld = N, m = i; the fused step keeps a block's
// molecules in shared memory: ld = its capacity, m = i - first molecule).
struct StateView {
    double *R, *v, *q, *L, *F, *tau;
    const int *spc;  // species of each slot
    int ld;
};

// load from a view: SH = shared memory (plain load), else global memory through
// L2 (data another block may have written in a persistent kernel)
template <bool SH, typename T>
__device__ __forceinline__ T ldv(const T *p) {
    if constexpr (SH) return *p;
    else return __ldcg(p);
}

__device__ __forceinline__ StateView global_view(const DevSys &S) {
    return StateView{S.R, S.v, S.q, S.Lm, S.F, S.tau, S.species, S.N};
}

// Drift of molecule i (state slot m) by the 4 lanes of a quad (c = lane & 3),
// all lanes on one instruction stream (an FP64 instruction costs the warp the
// same whatever its active lanes, so divergent lane roles would add up):
//   leapfrog: lanes 0-2 kick, scale and drift component c of v and R and update
//             L_c <- lambda (L_c + dt tau_c); every lane then rotates the whole
//             quaternion (identical results in the 4 lanes) and lane c stores
//             component c;
//   Verlet  : v_c += dt/2 F_c/M, R_c += dt v_c (point molecules, no rotation).
// Lanes 0-2 then rebuild lattice coordinate c and row c of the site offsets.
// `on` is false for padding quads: they compute on slot/molecule 0 and store
// nothing.  F and tau come through L2 loads (another block may have written
// them in a persistent kernel).
template <bool SH, bool BUILD = true>
__device__ __forceinline__ void drift_quad(const SysParams *__restrict__ P, const DevSys &S, const StateView &sv, int m,
                                           int i, bool on, int c, bool verlet, double lam) {
    const int ld = sv.ld, mm = on ? m : 0, cc = c < 3 ? c : 2;
    const int sp = sv.spc[mm];
    const double dt = P->dt;
    const unsigned qb = threadIdx.x & 28u;  // first lane of the quad within the warp
    double q[4] = {sv.q[mm], sv.q[ld + mm], sv.q[2 * ld + mm], sv.q[3 * ld + mm]};
    double Rc = sv.R[cc * ld + mm];
    if (verlet) {
        if (c < 3 && on) {
            const double v = sv.v[c * ld + m] + 0.5 * dt * P->kconv * P->inv_mass[sp] * ldv<SH>(sv.F + c * ld + m);
            sv.v[c * ld + m] = v;
            Rc += dt * v;
            sv.R[c * ld + m] = Rc;
        }
    } else {
        const double v = lam * (sv.v[cc * ld + mm] + P->kick[sp] * ldv<SH>(sv.F + cc * ld + mm));
        const double Lc = lam * (sv.L[cc * ld + mm] + P->dtk * ldv<SH>(sv.tau + cc * ld + mm));
        Rc += dt * v;
        if (c < 3 && on) {
            sv.v[c * ld + m] = v;
            sv.R[c * ld + m] = Rc;
            sv.L[c * ld + m] = Lc;
        }
        const bool rot = P->rot[sp] != 0;
        // quads of one warp may differ in species: every lane takes the same
        // shuffles, a non-rotating quad just keeps its quaternion (a warp of
        // non-rotating quads skips the rotation)
        if (__any_sync(0xffffffffu, rot)) {
            double L[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) L[k] = __shfl_sync(0xffffffffu, Lc, qb | k);
            const double q1c = rotate_q_quad(P->Iinv[sp], q, L, dt, rot ? P->quat_iters : 0, c);
            double qn[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) qn[k] = __shfl_sync(0xffffffffu, q1c, qb | k);
            if (rot) {
#pragma unroll
                for (int k = 0; k < 4; ++k) q[k] = qn[k];
                if (on) sv.q[c * ld + m] = q1c;
            }
        }
    }
    if (BUILD && c < 3 && on) build_row(P, S, i, c, q, Rc, sp);
}

// Fixed-tree sum of 8 values over a warp: 9 FP64 adds instead of 8 x 5.  On
// return lane l holds the total of value (l >> 2) & 7.
__device__ __forceinline__ double warp_sum8(double x[8], int lane) {
    const unsigned F = 0xffffffffu;
    const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double send = u16 ? x[k] : x[k + 4], keep = u16 ? x[k + 4] : x[k];
        x[k] = keep + __shfl_xor_sync(F, send, 16);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const double send = u8 ? x[k] : x[k + 2], keep = u8 ? x[k + 2] : x[k];
        x[k] = keep + __shfl_xor_sync(F, send, 8);
    }
    {
        const double send = u4 ? x[0] : x[1], keep = u4 ? x[1] : x[0];
        x[0] = keep + __shfl_xor_sync(F, send, 4);
    }
    x[0] += __shfl_xor_sync(F, x[0], 2);
    x[0] += __shfl_xor_sync(F, x[0], 1);
    return x[0];
}

// Fixed-tree sum of 4 values over a warp (5 FP64 adds); on return lane l holds
// the total of value (l >> 3) & 3.
__device__ __forceinline__ double warp_sum4(double x[4], int lane) {
    const unsigned F = 0xffffffffu;
    const bool u16 = lane & 16, u8 = lane & 8;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const double send = u16 ? x[k] : x[k + 2], keep = u16 ? x[k + 2] : x[k];
        x[k] = keep + __shfl_xor_sync(F, send, 16);
    }
    {
        const double send = u8 ? x[0] : x[1], keep = u8 ? x[1] : x[0];
        x[0] = keep + __shfl_xor_sync(F, send, 8);
    }
    x[0] += __shfl_xor_sync(F, x[0], 4);
    x[0] += __shfl_xor_sync(F, x[0], 2);
    x[0] += __shfl_xor_sync(F, x[0], 1);
    return x[0];
}

// Where a reduction unit reads the pair partials and writes the per-molecule
// results: partial value v of j-range p for slot m at [(p * NPV + v) * pld + m];
// energies k at Ui[k * uld + m], partner counts at np[m]; state through sv.
// Slot m holds molecule i0 + m.
struct RedIO {
    const float *part;
    const double *part64;
    int pld;
    StateView sv;
    double *Ui;
    int *np;
    int uld;
    int i0;
};

__device__ __forceinline__ RedIO global_io(const DevSys &S) {
    return RedIO{S.part, S.part64, S.N, global_view(S), S.Ui, S.npart, S.N, 0};
}

// The kinetic terms of the stored state of the molecule in slot m, for lane c of
// its quad (they need no forces): column cc of A(q), the body component lb of L,
// and the translational and rotational kinetic energies of component c (0 in
// lane 3).  reduce_unit forms them inline, or takes what kin_pre formed earlier
// with the same arithmetic.
template <bool SH>
__device__ __forceinline__ void kin_terms(const SysParams *__restrict__ P, const StateView &sv, int m, int sp, int c,
                                          int cc, bool anyrot, double col[3], double &lb, double &ktr, double &krot) {
    const int ld = sv.ld;
    const double hM = P->half_mass[sp], hI = P->half_Iinv[sp][cc];
    col[0] = col[1] = col[2] = 0.0;
    lb = 0.0;
    if (anyrot) {
        const double q[4] = {ldv<SH>(sv.q + m), ldv<SH>(sv.q + ld + m), ldv<SH>(sv.q + 2 * ld + m),
                             ldv<SH>(sv.q + 3 * ld + m)};
        double L[3];
        rot_column(q, cc, col);
#pragma unroll
        for (int k = 0; k < 3; ++k) L[k] = ldv<SH>(sv.L + k * ld + m);
        lb = col[0] * L[0] + col[1] * L[1] + col[2] * L[2];
    }
    const double v = ldv<SH>(sv.v + cc * ld + m);
    ktr = c < 3 ? hM * v * v : 0.0;
    krot = (c < 3 && anyrot) ? hI * lb * lb : 0.0;
}

// Reduction unit u of U: molecules [N u / U, N (u+1) / U), one warp, a quad per
// molecule, passes of 8 molecules.  With RED_SUM the quad sums the pair partials
// over the j-ranges (lane c takes the partial values c, c+4, c+8 in j-range
// order) into F, tau, the per-molecule energies and the partner count; then
// lanes 0-2 form the kinetic energies of component c (and, for RED_LAMBDA /
// RED_HALFKICK, after the kick).  RED_EWALD folds the reciprocal-space site
// forces into F, tau and the molecular virial.  Each lane accumulates its passes
// in order; the warp's totals of the Q_N step scalars go to blk[u][*].
template <bool SH>
__device__ __forceinline__ void reduce_unit(const SysParams *__restrict__ P, const DevSys &S, const RedIO &io, int mode,
                                            int u, int U, int lane, const double *pre = nullptr) {
    const unsigned F = 0xffffffffu, qb = lane & 28;
    const int N = S.N, c = lane & 3, cc = c < 3 ? c : 2;
    const int i_lo = (int)((long long)N * u / U), i_hi = (int)((long long)N * (u + 1) / U);
    const StateView &sv = io.sv;
    const int ld = sv.ld;
    double r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double jr = 0.0;  // lane accumulator of the current flux, component c (RED_GK)
    for (int base = i_lo; base < i_hi; base += 8) {
        const int i = base + (lane >> 2);
        const bool on = i < i_hi;
        const int ii = on ? i : i_lo, m = ii - io.i0;
        const int sp = sv.spc[m];
        double x[Q_N] = {0, 0, 0, 0, 0, 0, 0};
        double Fc, Tc;
        if (mode & RED_SUM) {
            double a[3];  // partial values c, c + 4, c + 8, summed in j-range order
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const size_t o = (size_t)(c + 4 * k) * io.pld + m;
                a[k] = (mode & RED_FP64PART) ? ldv<SH>(io.part64 + o) : f2d(ldv<SH>(io.part + o));
            }
            for (int p = 1; p < S.jsplit; ++p)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const size_t o = ((size_t)p * MS2_NPV + c + 4 * k) * io.pld + m;
                    a[k] += (mode & RED_FP64PART) ? ldv<SH>(io.part64 + o) : f2d(ldv<SH>(io.part + o));
                }
            // value v sits in lane v % 4, slot v / 4
            auto val = [&](int v) { return __shfl_sync(F, a[v >> 2], qb | (v & 3)); };
            const double fx = val(PV_FX), fy = val(PV_FY), fz = val(PV_FZ);
            const double tx = val(PV_TX), ty = val(PV_TY), tz = val(PV_TZ);
            const double ulj = val(PV_ULJ), uqq = val(PV_UQQ), udd = val(PV_UDD), w = val(PV_W), np = val(PV_NP);
            const double vvm = val(PV_VV);
            Fc = c == 0 ? fx : (c == 1 ? fy : fz);
            Tc = c == 0 ? tx : (c == 1 ? ty : tz);
            x[Q_U] = c == 0 ? ulj + uqq + udd : 0.0;
            x[Q_W] = c == 0 ? w : 0.0;
            x[Q_VV] = c == 0 ? vvm : 0.0;
            if (mode & RED_EWALD) {  // reciprocal-space site forces: the k chunks summed in order (FP32)
                const int NS = S.ns, M = S.nsite_q, c1 = (cc + 1) % 3, c2 = (cc + 2) % 3;
                double wc = 0;  // -F_s.s_s molecular-virial correction, component c
                for (int a2 = 0; a2 < NS; ++a2) {
                    float fs = 0.f, fc = 0.f;  // compensated sum over the k chunks
                    const float *fr = S.frec + (size_t)cc * M + a2 * N + ii;
                    int ch = 0;
                    for (; ch + 8 <= S.kchunks; ch += 8) {  // 8 loads in flight, then the adds in order
                        float p[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) p[u] = __ldcg(fr + (size_t)(ch + u) * 3 * M);
#pragma unroll
                        for (int u = 0; u < 8; ++u) ewald::kahan_add(fs, fc, p[u]);
                    }
                    for (; ch < S.kchunks; ++ch) ewald::kahan_add(fs, fc, __ldcg(fr + (size_t)ch * 3 * M));
                    const double f = f2d(fs) - f2d(fc);
                    const double f1 = __shfl_sync(F, f, qb | c1), f2 = __shfl_sync(F, f, qb | c2);
                    const double o1 = f2d(__ldcg(S.s + (c1 * NS + a2) * N + ii)),
                                 o2 = f2d(__ldcg(S.s + (c2 * NS + a2) * N + ii));
                    const double oc = f2d(__ldcg(S.s + (cc * NS + a2) * N + ii));
                    Fc += f;
                    Tc += o1 * f2 - o2 * f1;
                    wc += oc * f;
                }
                if (c == 3) wc = 0.0;
                x[Q_W] += -2.0 * wc;  // pair virial sums are halved at the end
                const double w0 = __shfl_sync(F, wc, qb), w1 = __shfl_sync(F, wc, qb | 1), w2 = __shfl_sync(F, wc, qb | 2);
                if (c == 0 && on) S.wcorr[i] = w0 + w1 + w2;  // per molecule, for the on-demand breakdown
            }
            if (on) {
                if (c < 3) {
                    sv.F[c * ld + m] = Fc;
                    sv.tau[c * ld + m] = Tc;
                }
                const double uk = c == 0 ? ulj : (c == 1 ? uqq : (c == 2 ? udd : w));
                io.Ui[c * io.uld + m] = uk;
                if (c == 0) io.np[m] = (int)np;
            }
            const unsigned hiF = (unsigned)__double2hiint(Fc) & 0x7FF00000u;  // |F| >= 2^99, inf or nan
            x[Q_BAD] = (c < 3 && hiF >= ((1023u + 99u) << 20)) ? 1.0 : 0.0;
        } else {
            Fc = ldv<SH>(sv.F + cc * ld + m);
            Tc = ldv<SH>(sv.tau + cc * ld + m);
        }
        // kinetic energies: lane c takes component c of v and body component c of L.
        // The state may have been written by another block of a persistent kernel: L2 loads.
        // (a warp of non-rotating molecules has no rotational terms: hI = 0)
        {
            const double hM = P->half_mass[sp], hI = P->half_Iinv[sp][cc];
            const bool anyrot = __any_sync(F, P->rot[sp] != 0);
            double col[3], tq[3], lb, ktr, krot;
#pragma unroll
            for (int k = 0; k < 3; ++k) tq[k] = __shfl_sync(F, Tc, qb | k);
            if (pre) {  // formed earlier by kin_pre (one pass)
#pragma unroll
                for (int k = 0; k < 3; ++k) col[k] = pre[k * 32 + lane];
                lb = pre[3 * 32 + lane];
                ktr = pre[4 * 32 + lane];
                krot = pre[5 * 32 + lane];
            } else {
                kin_terms<SH>(P, sv, m, sp, c, cc, anyrot, col, lb, ktr, krot);
            }
            double v = ldv<SH>(sv.v + cc * ld + m);
            if (c < 3) {
                x[Q_KTR] = ktr;
                x[Q_KROT] = krot;
            }
            if (mode & RED_HALFKICK) {  // Verlet: velocities at t + dt, recorded
                v += 0.5 * P->kick[sp] * Fc;
                if (on && c < 3) sv.v[c * ld + m] = v;
                if (c < 3) x[Q_KTR] = x[Q_K1] = hM * v * v;
            } else if (mode & RED_LAMBDA) {  // the kinetic energy after the kick
                v += P->kick[sp] * Fc;
                if (anyrot) {
                    const double lb1 = lb + P->dtk * (col[0] * tq[0] + col[1] * tq[1] + col[2] * tq[2]);
                    if (c < 3) x[Q_K1] = hM * v * v + hI * lb1 * lb1;
                } else if (c < 3) {
                    x[Q_K1] = hM * v * v;
                }
            }
        }
        if (base == i_lo) {  // first pass: no add
#pragma unroll
            for (int k = 0; k < Q_N; ++k) r[k] = on ? x[k] : 0.0;
        } else if (on) {
#pragma unroll
            for (int k = 0; k < Q_N; ++k) r[k] += x[k];
        }
        if (mode & RED_GK) {  // electric current flux: q_k v_k, component c in lane c
            const double jc = (c < 3 && on) ? P->qmol[sp] * ldv<SH>(sv.v + cc * ld + m) : 0.0;
            jr = (base == i_lo) ? jc : jr + jc;
        }
    }
    const double t = warp_sum8(r, lane);
    const int k = (lane >> 2) & 7;
    if ((lane & 3) == 0 && k < Q_N) S.blk[(size_t)u * MS2_NRED + k] = t;
    if (mode & RED_GK) {  // the three flux components: a 4-value fixed tree
        double y[4] = {(lane & 3) == 0 ? jr : 0.0, (lane & 3) == 1 ? jr : 0.0, (lane & 3) == 2 ? jr : 0.0, 0.0};
        const double tj = warp_sum4(y, lane);
        const int kj = (lane >> 3) & 3;
        if ((lane & 7) == 0 && kj < 3) S.blk[(size_t)u * MS2_NRED + Q_N + kj] = tj;
    }
}

// The kinetic terms of reduction unit u of U (1 to 8 molecules: one pass of
// reduce_unit; the caller checks) into pre[6][32], as reduce_unit would form
// them: a warp with no other work forms them before the forces are known.
// Every lane calls it.
template <bool SH>
__device__ __forceinline__ void kin_pre(const SysParams *__restrict__ P, const DevSys &S, const RedIO &io, int u, int U,
                                        int lane, double *pre) {
    const int N = S.N, c = lane & 3, cc = c < 3 ? c : 2;
    const int i_lo = (int)((long long)N * u / U), i_hi = (int)((long long)N * (u + 1) / U);
    const int i = i_lo + (lane >> 2);
    const int ii = i < i_hi ? i : i_lo, m = ii - io.i0;
    const int sp = io.sv.spc[m];
    const bool anyrot = __any_sync(0xffffffffu, P->rot[sp] != 0);
    double col[3], lb, ktr, krot;
    kin_terms<SH>(P, io.sv, m, sp, c, cc, anyrot, col, lb, ktr, krot);
#pragma unroll
    for (int k = 0; k < 3; ++k) pre[k * 32 + lane] = col[k];
    pre[3 * 32 + lane] = lb;
    pre[4 * 32 + lane] = ktr;
    pre[5 * 32 + lane] = krot;
}

// total of per-unit scalar k over units [0, nvb) by one warp, in reduce_totals'
// order (lane l sums units l, l + 32, ... in order, then the fixed tree); every lane
__device__ __forceinline__ double unit_total(const DevSys &S, int nvb, int k, int lane) {
    // the lane's first 8 values are all loaded before the first add (one L2
    // round trip, not one per value), then added in unit order as the loop below
    double v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int b = lane + 32 * t;
        v[t] = b < nvb ? __ldcg(S.blk + (size_t)b * MS2_NRED + k) : 0.0;
    }
    double x = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t)
        if (lane + 32 * t < nvb) x += v[t];
    for (int b = lane + 256; b < nvb; b += 32) x += __ldcg(S.blk + (size_t)b * MS2_NRED + k);
    return warp_sum(x);
}

// Totals of the step scalars over the reduction units, fixed order: warp w
// takes scalars w, w + nwarps, ...; lane l sums units l, l + 32, ... in order,
// then a fixed shuffle tree.  Result in tot[0 .. Q_N) (shared memory).
__device__ __forceinline__ void reduce_totals(const DevSys &S, int nvb, double *tot, int nq = Q_N) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = warp; k < nq; k += nw) {
        const double x = unit_total(S, nvb, k, lane);
        if (lane == 0) tot[k] = x;
    }
}

// One flux sample j into a flux ring g (layout: [0] samples, [1..3] unused,
// ring [M][3], lag sums [M]) and its lag sums, by a whole warp:
// sums[m] += j(t).j(t - m) for m < min(samples, M), each sum in sample order
// (Sec. 4, Eqs. 3-5; the extended time step is the sampling interval).
__device__ __forceinline__ void acf_update(double *g, int M, double j0, double j1, double j2, int lane) {
    double *ring = g + 4, *sums = ring + 3 * (size_t)M;
    const long long n = (long long)g[0];
    const int slot = (int)(n % M);
    if (lane == 0) {
        ring[3 * slot] = j0;
        ring[3 * slot + 1] = j1;
        ring[3 * slot + 2] = j2;
    }
    __syncwarp();
    const int upto = (int)(n + 1 < M ? n + 1 : M);
    for (int m = lane; m < upto; m += 32) {
        const int sm = (slot - m + M) % M;
        sums[m] += j0 * ring[3 * sm] + j1 * ring[3 * sm + 1] + j2 * ring[3 * sm + 2];
    }
    __syncwarp();
    if (lane == 0) g[0] = (double)(n + 1);
}

// the electric current flux j = tot[Q_N .. Q_N+2] of one conductivity sample
__device__ __forceinline__ void gk_update(const DevSys &S, const double *tot, int lane) {
    acf_update(S.gk, S.gk_lags, tot[Q_N], tot[Q_N + 1], tot[Q_N + 2], lane);
}

// ------------------------------------------------------------- heat flux
// Velocity and angular velocity of molecule m (state view sv) at the integer
// time of the current forces, in FP32 for the heat-flux power pass, the same in
// every lane: v = v_{n-1/2} + dt/2 F/M, L = L_{n-1/2} + dt/2 tau (space frame,
// the mean of the two half steps of the leapfrog without the thermostat factor),
// w = A I^-1 A^T L.  Velocity Verlet (integrator 0, point molecules): its
// reduction already left v at the integer time.
__device__ __forceinline__ double half_kick(const SysParams *__restrict__ P, int sp) {
    return P->integrator == 0 ? 0.0 : 0.5 * P->kick[sp];
}

template <bool SH>
__device__ __forceinline__ void heat_velocities(const SysParams *__restrict__ P, const StateView &sv, int m, float v[3],
                                                float w[3]) {
    const int ld = sv.ld, sp = sv.spc[m];
    const double hk = half_kick(P, sp), hd = 0.5 * P->dtk;
    float L[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v[k] = d2f(fma(hk, ldv<SH>(sv.F + k * ld + m), ldv<SH>(sv.v + k * ld + m)));
        L[k] = d2f(fma(hd, ldv<SH>(sv.tau + k * ld + m), ldv<SH>(sv.L + k * ld + m)));
    }
    const float q0 = d2f(ldv<SH>(sv.q + m)), q1 = d2f(ldv<SH>(sv.q + ld + m)), q2 = d2f(ldv<SH>(sv.q + 2 * ld + m)),
                q3 = d2f(ldv<SH>(sv.q + 3 * ld + m));
    // A (body -> space) of the unit quaternion (w, x, y, z)
    const float A00 = 1.f - 2.f * (q2 * q2 + q3 * q3), A01 = 2.f * (q1 * q2 - q0 * q3), A02 = 2.f * (q1 * q3 + q0 * q2);
    const float A10 = 2.f * (q1 * q2 + q0 * q3), A11 = 1.f - 2.f * (q1 * q1 + q3 * q3), A12 = 2.f * (q2 * q3 - q0 * q1);
    const float A20 = 2.f * (q1 * q3 - q0 * q2), A21 = 2.f * (q2 * q3 + q0 * q1), A22 = 1.f - 2.f * (q1 * q1 + q2 * q2);
    const float b0 = d2f(P->Iinv[sp][0]) * (A00 * L[0] + A10 * L[1] + A20 * L[2]);
    const float b1 = d2f(P->Iinv[sp][1]) * (A01 * L[0] + A11 * L[1] + A21 * L[2]);
    const float b2 = d2f(P->Iinv[sp][2]) * (A02 * L[0] + A12 * L[1] + A22 * L[2]);
    w[0] = A00 * b0 + A01 * b1 + A02 * b2;
    w[1] = A10 * b0 + A11 * b1 + A12 * b2;
    w[2] = A20 * b0 + A21 * b1 + A22 * b2;
}

// Heat-flux reduction unit u of U (the molecules of reduce_unit's unit u, a
// quad per molecule): lane c forms component c of
//   E_k v_k - 1/2 sum_p hp[p][c][m],   E_k = K_k + 1/2 sum_l u_kl - h_k
// (Sec. 4, Eq. 6 with the pair partials sum_l d_kl P_kl, d_kl = R_l - R_k) at the
// velocities of heat_velocities in FP64; per-molecule energies from Ui.  The
// warp's three sums go to blk[u][Q_N + 3 ..].
template <bool SH>
__device__ __forceinline__ void heat_unit(const SysParams *__restrict__ P, const DevSys &S, const float *hp, int hld,
                                          const StateView &sv, const double *Ui, int uld, int i0, int u, int U,
                                          int lane) {
    const unsigned F = 0xffffffffu, qb = lane & 28;
    const int N = S.N, c = lane & 3, cc = c < 3 ? c : 2;
    const int i_lo = (int)((long long)N * u / U), i_hi = (int)((long long)N * (u + 1) / U);
    const int ld = sv.ld;
    double jr = 0.0;
    for (int base = i_lo; base < i_hi; base += 8) {
        const int i = base + (lane >> 2);
        const bool on = i < i_hi;
        const int m = (on ? i : i_lo) - i0;
        const int sp = sv.spc[m];
        double jc = 0.0;
        for (int p = 0; p < S.jsplit; ++p) jc += f2d(ldv<SH>(hp + ((size_t)p * 3 + cc) * hld + m));
        const double v = fma(half_kick(P, sp), ldv<SH>(sv.F + cc * ld + m), ldv<SH>(sv.v + cc * ld + m));
        const double Lc = fma(0.5 * P->dtk, ldv<SH>(sv.tau + cc * ld + m), ldv<SH>(sv.L + cc * ld + m));
        double L[3], col[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) L[k] = __shfl_sync(F, Lc, qb | k);
        const double q[4] = {ldv<SH>(sv.q + m), ldv<SH>(sv.q + ld + m), ldv<SH>(sv.q + 2 * ld + m),
                             ldv<SH>(sv.q + 3 * ld + m)};
        rot_column(q, cc, col);
        const double lb = col[0] * L[0] + col[1] * L[1] + col[2] * L[2];
        double ke = c < 3 ? P->half_mass[sp] * v * v + P->half_Iinv[sp][cc] * lb * lb : 0.0;
        ke += __shfl_xor_sync(F, ke, 1);
        ke += __shfl_xor_sync(F, ke, 2);
        const double uk = ldv<SH>(Ui + m) + ldv<SH>(Ui + uld + m) + ldv<SH>(Ui + 2 * uld + m);
        const double E = ke * P->inv_kconv + 0.5 * uk - P->henth[sp];
        const double x = (c < 3 && on) ? E * v - 0.5 * jc : 0.0;
        jr = (base == i_lo) ? x : jr + x;
    }
    double y[4] = {(lane & 3) == 0 ? jr : 0.0, (lane & 3) == 1 ? jr : 0.0, (lane & 3) == 2 ? jr : 0.0, 0.0};
    const double t = warp_sum4(y, lane);
    const int k = (lane >> 3) & 3;
    if ((lane & 7) == 0 && k < 3) S.blk[(size_t)u * MS2_NRED + Q_N + 3 + k] = t;
}

// one heat-flux sample from the heat units: SC_HX.. and the heat-flux ring
__device__ __forceinline__ void heat_record(const DevSys &S, int nvb, int lane) {
    const double j0 = unit_total(S, nvb, Q_N + 3, lane), j1 = unit_total(S, nvb, Q_N + 4, lane),
                 j2 = unit_total(S, nvb, Q_N + 5, lane);
    if (lane == 0) {
        S.scal[SC_HX] = j0;
        S.scal[SC_HY] = j1;
        S.scal[SC_HZ] = j2;
    }
    acf_update(S.hf, S.hf_lags, j0, j1, j2, lane);
}

// isokinetic factor sqrt(T0 / T') from the kicked kinetic energy (as finish_step_warp)
__device__ __forceinline__ double lambda_k1(const SysParams *__restrict__ P, double k1) {
    const double x = P->lam_c * k1;  // T' / T0
    return (P->thermostat && x > 0) ? rsqrt_fp64(x) : 1.0;
}

__device__ __forceinline__ double lambda_of(const SysParams *__restrict__ P, const double *tot) {
    return lambda_k1(P, tot[Q_K1]);
}

}  // namespace integ
