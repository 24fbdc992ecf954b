// Device helpers of the integrator shared by the single-system kernels
// (k_integrate.cu) and the batched per-system kernel (batch.cu).
#pragma once
#include "ms2_internal.cuh"

namespace integ {

__device__ __forceinline__ double rsqrt_fp64(double x) {  // FP32 seed + two Newton steps (~1 ulp)
    double y = f2d(rsqrtf(d2f(x)));
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
        S.s[(c * NS + a) * N + i] = d2f(o);
        if (S.mu) S.mu[(c * NS + a) * N + i] = d2f(m);
    }
    if (S.mum) S.mum[c * N + i] = d2f(md);
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
        sc[SC_LAMBDA] = (P->thermostat && x > 0) ? rsqrt_fp64(x) : 1.0;  // == lambda_of(P, tot)
    }
}

// ------------------------------------------------------ one step, per quad
// Drift of molecule i by the 4 lanes of a quad (c = lane & 3), all lanes on one
// instruction stream (an FP64 instruction costs the warp the same whatever its
// active lanes, so divergent lane roles would add up):
//   leapfrog: lanes 0-2 kick, scale and drift component c of v and R and update
//             L_c <- lambda (L_c + dt tau_c); every lane then rotates the whole
//             quaternion (identical results in the 4 lanes) and lane c stores
//             component c;
//   Verlet  : v_c += dt/2 F_c/M, R_c += dt v_c (point molecules, no rotation).
// Lanes 0-2 then rebuild lattice coordinate c and row c of the site offsets.
// `on` is false for padding quads: they compute on molecule 0 and store nothing.
// Cross-block data (F, tau) is read with __ldcg so that the persistent step
// kernel never sees a stale L1 line.
__device__ __forceinline__ void drift_quad(const SysParams *__restrict__ P, const DevSys &S, int i, bool on, int c,
                                           bool verlet, double lam) {
    const int N = S.N, ii = on ? i : 0, cc = c < 3 ? c : 2;
    const int sp = S.species[ii];
    const double dt = P->dt;
    const unsigned qb = threadIdx.x & 28u;  // first lane of the quad within the warp
    double q[4] = {S.q[ii], S.q[N + ii], S.q[2 * N + ii], S.q[3 * N + ii]};
    if (verlet) {
        if (c < 3 && on) {
            const double v = S.v[c * N + i] + 0.5 * dt * P->kconv * P->inv_mass[sp] * __ldcg(S.F + c * N + i);
            S.v[c * N + i] = v;
            S.R[c * N + i] += dt * v;
        }
    } else {
        const double v = lam * (S.v[cc * N + ii] + dt * P->kconv * P->inv_mass[sp] * __ldcg(S.F + cc * N + ii));
        const double Lc = lam * (S.Lm[cc * N + ii] + dt * P->kconv * __ldcg(S.tau + cc * N + ii));
        if (c < 3 && on) {
            S.v[c * N + i] = v;
            S.R[c * N + i] += dt * v;
            S.Lm[c * N + i] = Lc;
        }
        double L[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) L[k] = __shfl_sync(0xffffffffu, Lc, qb | k);
        const double *Ii = P->Iinv[sp];
        if (Ii[0] != 0.0 || Ii[1] != 0.0 || Ii[2] != 0.0) {
            double q1[4];
            rotate_q(Ii, q, L, dt, P->quat_iters, q1);
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = q1[k];
            if (on) S.q[c * N + i] = q1[c];
        }
    }
    if (c < 3 && on) build_row(P, S, i, c, q);
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

// Reduction unit `vb`: molecules 8 vb .. 8 vb + 7, one quad each, one warp.
// With RED_SUM the quad sums the pair partials over the j-ranges (lane c takes
// the partial values c, c+4, c+8 in j-range order) into F, tau, the
// per-molecule energies and the partner count; then lanes 0-2 form the kinetic
// energies of component c (and, for RED_LAMBDA / RED_HALFKICK, after the kick).
// RED_EWALD folds the reciprocal-space site forces into F, tau and the
// molecular virial.  The warp's totals of the Q_N step scalars go to blk[vb][*].
__device__ __forceinline__ void reduce_unit(const SysParams *__restrict__ P, const DevSys &S, int mode, int vb,
                                            int lane) {
    const unsigned F = 0xffffffffu, qb = lane & 28;
    const int N = S.N, c = lane & 3, i = vb * 8 + (lane >> 2);
    const bool on = i < N;
    const int ii = on ? i : 0, cc = c < 3 ? c : 2;
    const int sp = S.species[ii];
    double r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double Fc, Tc;
    if (mode & RED_SUM) {
        double a[3] = {0, 0, 0};  // partial values c, c + 4, c + 8
        for (int p = 0; p < S.jsplit; ++p)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const size_t o = ((size_t)p * MS2_NPV + c + 4 * k) * N + ii;
                a[k] += (mode & RED_FP64PART) ? __ldcg(S.part64 + o) : f2d(__ldcg(S.part + o));
            }
        // value v sits in lane v % 4, slot v / 4
        auto val = [&](int v) { return __shfl_sync(F, a[v >> 2], qb | (v & 3)); };
        const double fx = val(PV_FX), fy = val(PV_FY), fz = val(PV_FZ);
        const double tx = val(PV_TX), ty = val(PV_TY), tz = val(PV_TZ);
        const double ulj = val(PV_ULJ), uqq = val(PV_UQQ), udd = val(PV_UDD), w = val(PV_W), np = val(PV_NP);
        Fc = c == 0 ? fx : (c == 1 ? fy : fz);
        Tc = c == 0 ? tx : (c == 1 ? ty : tz);
        r[Q_U] = c == 0 ? ulj + uqq + udd : 0.0;
        r[Q_W] = c == 0 ? w : 0.0;
        if (mode & RED_EWALD) {  // reciprocal-space site forces, summed over k chunks
            const int NS = S.ns, M = S.nsite_q, c1 = (cc + 1) % 3, c2 = (cc + 2) % 3;
            double wc = 0;  // -F_s.s_s molecular-virial correction, component c
            for (int a = 0; a < NS; ++a) {
                double f = 0;
                for (int ch = 0; ch < S.kchunks; ++ch) f += f2d(__ldcg(S.frec + ((size_t)ch * 3 + cc) * M + a * N + ii));
                const double f1 = __shfl_sync(F, f, qb | c1), f2 = __shfl_sync(F, f, qb | c2);
                const double o1 = f2d(S.s[(c1 * NS + a) * N + ii]), o2 = f2d(S.s[(c2 * NS + a) * N + ii]);
                const double oc = f2d(S.s[(cc * NS + a) * N + ii]);
                Fc += f;
                Tc += o1 * f2 - o2 * f1;
                wc += oc * f;
            }
            if (c == 3) wc = 0.0;
            r[Q_W] += -2.0 * wc;  // pair virial sums are halved at the end
            const double w0 = __shfl_sync(F, wc, qb), w1 = __shfl_sync(F, wc, qb | 1), w2 = __shfl_sync(F, wc, qb | 2);
            if (c == 0 && on) S.wcorr[i] = w0 + w1 + w2;  // per molecule, for the on-demand breakdown
        }
        if (on) {
            if (c < 3) {
                S.F[c * N + i] = Fc;
                S.tau[c * N + i] = Tc;
            }
            const double uk = c == 0 ? ulj : (c == 1 ? uqq : (c == 2 ? udd : w));
            S.Ui[c * N + i] = uk;
            if (c == 0) S.npart[i] = (int)np;
        }
        const unsigned hiF = (unsigned)__double2hiint(Fc) & 0x7FF00000u;  // |F| >= 2^99, inf or nan
        r[Q_BAD] = (c < 3 && hiF >= ((1023u + 99u) << 20)) ? 1.0 : 0.0;
    } else {
        Fc = __ldcg(S.F + cc * N + ii);
        Tc = __ldcg(S.tau + cc * N + ii);
    }
    // kinetic energies: lane c takes component c of v and body component c of L
    {
        // state written by another block's drift in the persistent step kernel: L2 loads
        const double M = P->mass[sp], Ii = P->Iinv[sp][cc];
        const double q[4] = {__ldcg(S.q + ii), __ldcg(S.q + N + ii), __ldcg(S.q + 2 * N + ii), __ldcg(S.q + 3 * N + ii)};
        double col[3], L[3], tq[3];
        rot_column(q, cc, col);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            L[k] = __ldcg(S.Lm + k * N + ii);
            tq[k] = __shfl_sync(F, Tc, qb | k);
        }
        double v = __ldcg(S.v + cc * N + ii);
        const double lb = col[0] * L[0] + col[1] * L[1] + col[2] * L[2];
        if (c < 3) {
            r[Q_KTR] = 0.5 * M * v * v;
            r[Q_KROT] = 0.5 * Ii * lb * lb;
        }
        if (mode & (RED_LAMBDA | RED_HALFKICK)) {
            const double h = (mode & RED_HALFKICK) ? 0.5 * P->dt : P->dt;
            const double ct = h * P->kconv;
            v += ct * P->inv_mass[sp] * Fc;
            const double lb1 = lb + ct * (col[0] * tq[0] + col[1] * tq[1] + col[2] * tq[2]);
            if (c < 3) r[Q_K1] = 0.5 * M * v * v + 0.5 * Ii * lb1 * lb1;
            if (mode & RED_HALFKICK) {  // Verlet: velocities at t + dt, recorded
                if (on && c < 3) S.v[c * N + i] = v;
                if (c < 3) r[Q_KTR] = 0.5 * M * v * v;
            }
        }
    }
    if (!on)
#pragma unroll
        for (int k = 0; k < 8; ++k) r[k] = 0.0;
    const double t = warp_sum8(r, lane);
    const int k = (lane >> 2) & 7;
    if ((lane & 3) == 0 && k < Q_N) {
        S.blk[(size_t)vb * MS2_NRED + k] = t;
        __threadfence();
    }
}

// Totals of the step scalars over the reduction units, fixed order: warp w
// takes scalars w, w + nwarps, ...; lane l sums units l, l + 32, ... in order,
// then a fixed shuffle tree.  Result in tot[0 .. Q_N) (shared memory).
__device__ __forceinline__ void reduce_totals(const DevSys &S, int nvb, double *tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = warp; k < Q_N; k += nw) {
        double x = 0;
        for (int b = lane; b < nvb; b += 32) x += __ldcg(S.blk + (size_t)b * MS2_NRED + k);
        x = warp_sum(x);
        if (lane == 0) tot[k] = x;
    }
}

// isokinetic factor sqrt(T0 / T') from the kicked kinetic energy (as finish_step)
__device__ __forceinline__ double lambda_of(const SysParams *__restrict__ P, const double *tot) {
    const double x = 2.0 * tot[Q_K1] * P->inv_kconv * P->inv_ndof * P->inv_T0;
    return (P->thermostat && x > 0) ? rsqrt_fp64(x) : 1.0;
}

}  // namespace integ
