// Internal data layout and device helpers of libms2 (GB300, sm_103a).
//
// Layout in device memory (one system):
//   FP64 state, SoA by component:  R[3][N], v[3][N], q[4][N], Lm[3][N]
//   per step, written by the site build:
//     X[3][N]          uint32 centre coordinates on a 2^32-point lattice per edge
//     s[3][NS][N]      FP32 space-frame site offsets A(q_i) b_a (slot-major)
//     mu[3][NS][N]     FP32 space-frame dipoles (only when a slot carries one)
//     mum[3][N]        FP32 molecular charge dipoles (reaction field with charges)
//   pair-kernel output: part[JSPLIT][NPV][N] FP32 partial sums per j-range
//   reduced:           F[3][N], tau[3][N] FP64, per-molecule energy/virial
//   Ewald:             site lattice coordinates, e^{i n theta} tables, S(k)
// Everything a thread block reads for one molecule is contiguous per component,
// so consecutive lanes (molecules) make coalesced 4- or 8-byte accesses.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define MS2_MAXSP 4
#define MS2_MAXS 8
#define MS2_MAXT 16        // LJ site kinds (species x LJ slot)
#define MS2_NPV 12         // values per molecule in a pair-kernel partial
#define MS2_NRED 16        // per-block reduction scalars

// partial-slot meaning
enum { PV_FX = 0, PV_FY, PV_FZ, PV_TX, PV_TY, PV_TZ, PV_ULJ, PV_UQQ, PV_UDD, PV_W, PV_NP, PV_VV };  // PV_VV: d2U/dV2 sum

enum { ELEC_NONE = 0, ELEC_RF = 1, ELEC_EWALD = 2 };

// Per-system constants (models, mixing tables, electrostatics, integrator).
struct SysParams {
    int N, ns, n_species, n_ljt;
    int elec, integrator, thermostat, quat_iters;
    int has_dipole, multi, ndof, massieu;  // massieu: sample the Massieu-derivative moments
    double L, V, dt, kconv, T0;
    double inv_kconv, inv_ndof, inv_V, inv_T0;   // host-side reciprocals (no FP64 divide per step)
    double inv_mass[MS2_MAXSP];
    // per-step products, formed once on the host (an FP64 multiply costs a warp
    // ~68 cycles on GB300): dt kconv, the kick dt kconv / M, M/2, I^-1 / 2 and
    // the thermostat constant 2 / (kconv ndof T0)
    double dtk, kick[MS2_MAXSP], half_mass[MS2_MAXSP], half_Iinv[MS2_MAXSP][3], lam_c;
    double qmol[MS2_MAXSP];  // net molecular charge of each species (electric current flux)
    double henth[MS2_MAXSP]; // partial molar enthalpy of each species, energy units (heat flux)
    double lat_scale;          // 2^32 / L  (FP64, exact same value as the host computes)
    unsigned long long rc2;    // lattice cut-off threshold
    float lat_to_len;          // L / 2^32 (FP32 rounding of it)
    float lat_to_len_lo;       // L / 2^32 - lat_to_len (the rounding remainder)
    float len_to_lat;          // 2^32 / L
    float coulomb, krf, crf, alpha, two_alpha_sqrtpi;
    // LJ site pairs at close contact, r < 1.1 sigma_ab (t12 > close_k6 t6, with
    // close_k6 = 1.1^-6), are evaluated in double-float; +inf switches it off
    float close_k6;
    // Ewald: the FP32 rounding remainder of 2 alpha / sqrt(pi) (a rounded constant
    // would scale every real-space term of the molecular virial the same way;
    // alpha itself is taken as its FP32 value everywhere, so it is exact)
    float two_alpha_sqrtpi_lo;
    float pad_ew_[2];                      // keeps the struct a whole number of 16-byte words
    // species tables
    int n_sites[MS2_MAXSP];
    double bpos[MS2_MAXSP][MS2_MAXS][3];   // body-frame site positions
    double bdip[MS2_MAXSP][MS2_MAXS][3];   // body-frame dipoles
    float q[MS2_MAXSP][MS2_MAXS];          // charges (0: none), FP32 rounding
    float qlo[MS2_MAXSP][MS2_MAXS];        // q - (float)q
    float cq[MS2_MAXSP][MS2_MAXS];         // C q as hi + lo floats (C q computed in FP64)
    float cqlo[MS2_MAXSP][MS2_MAXS];
    double qd[MS2_MAXSP][MS2_MAXS];        // FP64 charges
    int ljt[MS2_MAXSP][MS2_MAXS];          // LJ kind or -1
    double mass[MS2_MAXSP];                // molecule mass
    double Iinv[MS2_MAXSP][3];             // inverse principal moments (0: free axis)
    int rot[MS2_MAXSP];                    // 1: some inverse moment is non-zero (the species rotates)
    int point[MS2_MAXSP];                  // 1: every site and dipole at the centre (no orientation)
    float c6[MS2_MAXT][MS2_MAXT];          // 4 eps sigma^6 (Lorentz-Berthelot), FP32 rounding
    float c12[MS2_MAXT][MS2_MAXT];         // 4 eps sigma^12, FP32 rounding
    float c6lo[MS2_MAXT][MS2_MAXT];        // remainders: c = hi + lo to ~48 bits, so that
    float c12lo[MS2_MAXT][MS2_MAXT];       // fmaf(hi, x, lo*x) is c*x correctly rounded
    float coulomb_lo;                      // coulomb - (float)coulomb
    double c6d[MS2_MAXT][MS2_MAXT], c12d[MS2_MAXT][MS2_MAXT];
};

// Device pointers of one system.
struct DevSys {
    int N, ns, jsplit, nunits;  // nunits: reduction units (contiguous molecule ranges)
    double *R, *v, *q, *Lm;           // FP64 state
    int *species;
    uint32_t *X;                       // [3][N]
    float *s, *mu;                     // [3][ns][N]
    float *mum;                        // [3][N] molecular dipole sum_a q_a s_ia (reaction field)
    double *gk;                        // conductivity: [0] samples, [1..3] -, ring [gk_lags][3], lag sums [gk_lags]
    int gk_lags;
    double *hf;                        // thermal conductivity: the same layout as gk (heat flux J_q)
    int hf_lags;
    float *hpart;                      // [jsplit][3][N] heat-flux pair partials sum_l d_kl P_kl
    float *part;                       // [jsplit][NPV][N]
    double *part64;                    // FP64 partials (FP64 pair path)
    double *F, *tau;                   // [3][N]
    double *Ui;                        // [4][N]: U_lj, U_qq, U_dd, W (owner sums over partners)
    double *wcorr;                     // [N] Ewald: sum_a F_rec,a . s_a (molecular-virial correction)
    double *terms;                     // [8] on-demand breakdown sums
    int *npart;                        // [N]
    double *blk;                       // [nblk][NRED] per-block partial sums
    unsigned int *counter;             // last-block counter
    double *scal;                      // system scalars (see SC_* below)
    double *acc;                       // running averages (see AC_* below)
    // Ewald
    int nk, kx, ky, kz, nsite_q, kchunks;
    int sk_sites;                      // sites per structure-factor task
    float ew_fpre, ew_fpre_lo;         // force prefactor 8 pi C / V * 2 pi / L (FP64 on the host) as hi + lo floats
    float *qs;                         // [nsite_q] site charges
    float2 *eik;                       // [3][kmax+1][nsite_q] e^{i n theta}
    double *Sk;                        // [nk][4]: A*Re S, A*Im S, |S|^2 A part, ... (scaled)
    float *frec;                       // [kchunks][3][nsite_q] partial site forces
    float2 *skpart;                    // [site blocks][k] partial structure factors
    double *Ak, *Bk;                   // [k] A(k) = exp(-k^2/4a^2)/k^2 on the half space (else 0), A (1 - k^2/2a^2)
    double *kblk;                      // per-block energy/virial partials of S(k)
    // RDF
    unsigned long long *rdf;           // [rows][nbins]
    int rdf_bins, rdf_rows;
    float rdf_inv_dr, rdf_rmax2;
    int *rdf_kind;                     // [MAXSP*MAXS] kind or -1
};

// system scalars written by the last block of a reduction
enum {
    SC_ULJ = 0, SC_UQQ, SC_UDD, SC_WPAIR, SC_NPAIRS, SC_KETR, SC_KEROT, SC_LAMBDA,
    SC_UREC, SC_WREC_AT, SC_WREC_CORR, SC_UCONST, SC_PLRC, SC_ULRC, SC_WBG, SC_UNSTABLE,
    SC_UTOT, SC_WTOT, SC_P, SC_T, SC_KETR_NOW, SC_KEROT_NOW, SC_STEP,
    SC_UV, SC_UVV,  // dU/dV and d2U/dV2 of the current configuration (with the Massieu option)
    SC_JX, SC_JY, SC_JZ,  // electric current flux of the last conductivity sample
    SC_TPAIR,  // fused step: pair-phase time of the last step of a chunk (ns)
    SC_TPH0, SC_TPH1, SC_TPH2, SC_TPH3, SC_TPH4, SC_TPH5, SC_TPH6, SC_TPH7, SC_TPH8,  // fused step: phase times (ns)
    SC_TPH9, SC_TPH10, SC_TPH11,  // fused Ewald step: the structure-factor, sum and force task phases (ns)
    SC_KERR,   // fused step: a grid-barrier wait timed out (sticky until read)
    SC_HX, SC_HY, SC_HZ,  // heat flux of the last thermal-conductivity sample
    SC_COUNT_
};
// running averages; AC_M*: Massieu-derivative moment sums of x = U - U0, y = U_V - V0, w = U_VV
enum { AC_N = 0, AC_U, AC_P, AC_T, AC_BN, AC_BU, AC_BP, AC_NB, AC_SBU, AC_SBU2, AC_SBP, AC_SBP2,
       AC_MN, AC_MX, AC_MX2, AC_MX3, AC_MY, AC_MY2, AC_MXY, AC_MX2Y, AC_MXY2, AC_MW, AC_MXW, AC_MU0, AC_MV0,
       AC_COUNT_ };

// modes of the reduction (k_reduce, the fused step): sum the pair partials,
// record the step, form the thermostat factor, Verlet second half kick, FP64
// partials, Ewald site forces, sample the electric current flux
enum { RED_SUM = 1, RED_RECORD = 2, RED_LAMBDA = 4, RED_HALFKICK = 8, RED_FP64PART = 16, RED_EWALD = 32,
       RED_GK = 64 };

// residence-time sampling state (k_residence.cu): centres [A0, A0 + NA), solvent
// molecules [B0, B0 + NB) (species are contiguous), WB = ceil(NB / 32) words,
// a ring of M origins
struct ResArgs {
    int A0, NA, B0, NB, WB, M, t_star;
    unsigned long long r2;   // shell threshold on the integer lattice
    unsigned *alive;         // [M][NA][WB] members still resident, per origin
    unsigned char *out;      // [M][NA][NB] current excursion length of each member
    int *n0;                 // [M][NA] shell count at each origin
    int *counts;             // [NA][M] members alive and inside at this sample
    double *state;           // samples, solvation sums, then [M] fraction sums and [M] term counts
};

// launch arguments of the fused step kernel (k_step.cu)
struct StepArgs {
    int nsteps;
    long long s0;          // step counter before the chunk (RDF sampling phase)
    int rdf_every;         // 0: no RDF sampling
    int gk_every;          // 0: no conductivity sampling, else the extended time step in steps
    int hf_every;          // 0: no heat-flux sampling, else its extended time step
    int TJ;                // j tile segmentation of the per-phase pair kernel
    int Np;                // stride of the staged system
    int mcap;              // molecules a block owns at most: ceil(N / gridDim.x)
    unsigned *bar;         // this launch's barrier counter (zero at entry)
    unsigned *bar_next;    // the next launch's counter, zeroed by this launch
    unsigned *err;         // sticky timeout flag
    int timing;            // record the phase times of the last step (SC_TPAIR, SC_TPH*, ns)
    int init;              // first evaluate the state as set (site build, forces, energies): after ms2_set_state
    float2 *AS;            // Ewald: A(k) S(k) of the step (the reciprocal-space force tasks read it)
    int ny_per_chunk;      // Ewald: ny values per force k chunk
    int ews;               // Ewald: bytes of the block's reciprocal-space task scratch
    unsigned long long *tmax;  // timing: [3] latest compute-end times over blocks (zero at entry, re-zeroed after use)
    unsigned long long wait_ns;  // limit of each grid-barrier wait
    unsigned bar_extra;          // arrivals the first barrier waits for beyond the grid (0; 1: a fault-path test)
};

// ------------------------------------------------------------ helpers
__device__ __forceinline__ void rotmat(const double q0, const double q1, const double q2, const double q3,
                                       double A[9]) {
    // body -> space rotation of the unit quaternion (w, x, y, z)
    A[0] = 1.0 - 2.0 * (q2 * q2 + q3 * q3);
    A[1] = 2.0 * (q1 * q2 - q0 * q3);
    A[2] = 2.0 * (q1 * q3 + q0 * q2);
    A[3] = 2.0 * (q1 * q2 + q0 * q3);
    A[4] = 1.0 - 2.0 * (q1 * q1 + q3 * q3);
    A[5] = 2.0 * (q2 * q3 - q0 * q1);
    A[6] = 2.0 * (q1 * q3 - q0 * q2);
    A[7] = 2.0 * (q2 * q3 + q0 * q1);
    A[8] = 1.0 - 2.0 * (q1 * q1 + q2 * q2);
}

// IEEE binary32 <-> binary64 conversions written on the integer pipe.  On GB300
// a conversion instruction occupies the SMSP's small FP64 unit for ~90-180
// cycles; these take a few integer operations and return exactly what the
// hardware conversion returns (round to nearest even), falling back to it
// outside the normal range.
__device__ __forceinline__ double f2d(float f) {
    const unsigned b = __float_as_uint(f), e = (b >> 23) & 0xFFu;
    const unsigned long long sgn = (unsigned long long)(b & 0x80000000u) << 32;
    if (e - 1u < 254u)  // normal
        return __longlong_as_double((long long)(sgn | ((unsigned long long)(e + 896u) << 52) |
                                                ((unsigned long long)(b & 0x7FFFFFu) << 29)));
    if ((b & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)sgn);  // signed zero
    return (double)f;  // subnormal, inf, nan
}

__device__ __forceinline__ float d2f(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), sgn = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu) - 896;  // binary32 biased exponent
    if (e >= 1 && e <= 254) {
        const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
        const unsigned rem = (unsigned)(m & 0x1FFFFFFFull), half = 0x10000000u;
        unsigned r = ((unsigned)e << 23) | (unsigned)(m >> 29);
        r += (rem > half || (rem == half && (r & 1u))) ? 1u : 0u;  // a carry into the exponent is correct
        return __uint_as_float(r | sgn);
    }
    if ((b & 0x7FFFFFFFFFFFFFFFull) == 0ull) return __uint_as_float(sgn);  // signed zero
    return (float)x;  // subnormal result, overflow, inf, nan
}

// lattice coordinate: floor(x * 2^32/L) mod 2^32, taken with one IEEE multiply
// (no contraction possible) so that host and device agree bit for bit.  For
// |t| < 2^51 the floor comes from one round-down add of 1.5 * 2^52 (the sum's
// unit in the last place is 1, and its low mantissa word is floor(t) mod 2^32);
// larger |t| takes floor and an integer conversion.
__device__ __forceinline__ uint32_t lattice_coord(double x, double scale) {
    const double t = __dmul_rn(x, scale);
    const unsigned ex = ((unsigned)__double2hiint(t) >> 20) & 0x7FFu;
    if (ex < 1023u + 51u) return (uint32_t)__double2loint(__dadd_rd(t, 6755399441055744.0));
    return (uint32_t)(unsigned long long)(long long)floor(t);
}

__device__ __forceinline__ unsigned long long lattice_d2(int dx, int dy, int dz) {
    return (unsigned long long)((long long)dx * dx) + (unsigned long long)((long long)dy * dy) +
           (unsigned long long)((long long)dz * dz);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// host-side launch accounting (one increment per kernel launch or graph node replay)
void ms2_count_launches(long long n);

#define MS2_CUDA_OK(call)                                                                     \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return ms2_fail_cuda(e_, #call, __FILE__, __LINE__);           \
    } while (0)
