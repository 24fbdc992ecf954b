/*
 * ms2 FP64 oracle — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU restatement of the molecular-dynamics hot
 * path of the ms2 2.0 release paper (Glass et al., arXiv 1507.07548):
 *   - interaction partner search with a molecule-centre cut-off near half the box
 *     edge (Sec. "Hybrid MPI & OpenMP Parallelization"),
 *   - energy, force and torque between rigid multi-site molecules built from
 *     Lennard-Jones 12-6 sites and point charges (Sec. "Massieu potential
 *     derivatives", which names LJ and Coulomb as the pair potentials), with the
 *     reaction-field treatment of electrostatics (same section) or Ewald summation
 *     (Sec. "Algorithmic Developments", paragraph "Ewald summation"),
 *   - point dipoles (needed by the Stockmayer-like workload; textbook form),
 *   - the analytic Lennard-Jones long-range correction (Sec. "Massieu ..."),
 *   - rigid-body integration (velocity Verlet; leapfrog + quaternion implicit
 *     midpoint) with isokinetic velocity scaling for NVT,
 *   - the radial distribution function between LJ sites (Sec. "Property
 *     Calculations", Eq. 2).
 * The paper states the ingredients and defers the formulas to Allen & Tildesley
 * and Frenkel & Smit; the formulas below are the textbook forms written out.
 *
 * Everything is FP64, loops over molecules i, partners j and site pairs (a, b)
 * in the order the definitions read.  OpenMP only splits the owner loop over i;
 * every sum over molecules is taken afterwards in index order, so results do not
 * depend on the thread count.
 *
 * Only tests/, the smoke check and the CPU-baseline leg of the benchmark use this
 * file.  The GPU library never links, includes or calls it.
 *
 * Readings where the paper is silent (documented with the design):
 *   - "molecule centre" = centre of mass; a pair (i, j) interacts iff the
 *     minimum-image centre distance is below rc; all site pairs of a partner
 *     pair interact with the molecule-centre image (no per-site minimum image);
 *   - the cut-off test is taken on centre coordinates rounded onto a lattice of
 *     2^32 points per box edge, in exact integer arithmetic (see or_lattice);
 *   - Lorentz-Berthelot mixing for unlike LJ sites;
 *   - reaction-field constants k_RF = (eps_RF-1)/((2 eps_RF+1) rc^3),
 *     c_RF = 1/rc + k_RF rc^2 with the molecule-centre rc;
 *   - Ewald with tin-foil boundary, a box of k vectors |n_x|,|n_y|,|n_z| <= kmax,
 *     real-space terms over the molecule-centre partner pairs;
 *   - isokinetic scaling of v(t+dt/2) and L(t+dt/2) by one factor, with the
 *     rotational kinetic energy evaluated at the orientation q(t).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* host threads of the OpenMP loops (timing only; the arithmetic does not depend on it) */
void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

#define OR_MAXSP 4
#define OR_MAXS 8
#define OR_NTERMS 16

typedef struct {
    /* species table: body frame = centre of mass at the origin, axes along the
     * principal axes of inertia (the caller's responsibility, checked in tests) */
    int n_species;
    int n_sites[OR_MAXSP];
    double pos[OR_MAXSP][OR_MAXS][3];
    double mass[OR_MAXSP][OR_MAXS];
    int lj[OR_MAXSP][OR_MAXS];
    double sigma[OR_MAXSP][OR_MAXS];
    double epsilon[OR_MAXSP][OR_MAXS];
    double charge[OR_MAXSP][OR_MAXS];
    double dipole[OR_MAXSP][OR_MAXS][3];
    /* system */
    int N;
    const int *species;  /* N entries */
    double L;            /* cubic box edge */
    double rc;           /* molecule-centre cut-off, rc < L/2 */
    int elec;            /* 0 none, 1 reaction field, 2 Ewald */
    double eps_rf;       /* reaction-field dielectric constant; <= 0 means conducting */
    double alpha;        /* Ewald splitting parameter */
    int kmax[3];         /* Ewald k box */
    double coulomb;      /* e^2/(4 pi eps0 kB) in the energy*length unit */
    double kconv;        /* energy unit expressed in mass*length^2/time^2 */
    int lrc;             /* 1: add the analytic LJ long-range correction */
    double crf_shift;    /* added to c_RF; 0 except in the shift-invariance check */
} or_system;

/* energy / virial breakdown (same order everywhere in this file) */
enum {
    T_ULJ = 0, T_UQQ, T_UDD, T_UREC, T_USELF, T_UINTRA, T_UBG, T_ULRC, T_UTOT,
    T_WPAIR, T_WREC, T_WBG, T_WTOT, T_PLRC, T_NPAIRS, T_SPARE
};

/* ------------------------------------------------------------------ vectors */
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
/* y = A x with A row-major 3x3 */
static void matvec(const double *A, const double *x, double *y) {
    for (int r = 0; r < 3; ++r) y[r] = A[3 * r] * x[0] + A[3 * r + 1] * x[1] + A[3 * r + 2] * x[2];
}
/* y = A^T x */
static void matTvec(const double *A, const double *x, double *y) {
    for (int c = 0; c < 3; ++c) y[c] = A[c] * x[0] + A[3 + c] * x[1] + A[6 + c] * x[2];
}

/* Rotation matrix (body -> space) of the unit quaternion q = (w, x, y, z):
 * v_space = q v_body q*.  Textbook form (Allen & Tildesley, rigid bodies). */
void or_rotation(const double *q, double *A) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    A[0] = 1 - 2 * (y * y + z * z); A[1] = 2 * (x * y - w * z);     A[2] = 2 * (x * z + w * y);
    A[3] = 2 * (x * y + w * z);     A[4] = 1 - 2 * (x * x + z * z); A[5] = 2 * (y * z - w * x);
    A[6] = 2 * (x * z - w * y);     A[7] = 2 * (y * z + w * x);     A[8] = 1 - 2 * (x * x + y * y);
}

/* ------------------------------------------------------------ model helpers */
static double mol_mass(const or_system *s, int sp) {
    double m = 0;
    for (int a = 0; a < s->n_sites[sp]; ++a) m += s->mass[sp][a];
    return m;
}
/* principal moments: diagonal of the body-frame inertia tensor */
static void mol_inertia(const or_system *s, int sp, double *I) {
    I[0] = I[1] = I[2] = 0;
    for (int a = 0; a < s->n_sites[sp]; ++a) {
        const double *p = s->pos[sp][a];
        double m = s->mass[sp][a];
        I[0] += m * (p[1] * p[1] + p[2] * p[2]);
        I[1] += m * (p[0] * p[0] + p[2] * p[2]);
        I[2] += m * (p[0] * p[0] + p[1] * p[1]);
    }
}
/* inverse moments; a moment below 1e-12 of the largest is a free axis of a
 * linear (or point) molecule and gets inverse 0, i.e. no rotation about it */
static void mol_inv_inertia(const or_system *s, int sp, double *Iinv) {
    double I[3];
    mol_inertia(s, sp, I);
    double mx = fmax(I[0], fmax(I[1], I[2]));
    for (int k = 0; k < 3; ++k) Iinv[k] = (mx > 0 && I[k] > 1e-12 * mx) ? 1.0 / I[k] : 0.0;
}
int or_rot_dof(const or_system *s, int sp) {
    double Iinv[3];
    mol_inv_inertia(s, sp, Iinv);
    return (Iinv[0] != 0) + (Iinv[1] != 0) + (Iinv[2] != 0);
}
int or_ndof(const or_system *s) {
    int n = 3 * s->N - 3;
    for (int i = 0; i < s->N; ++i) n += or_rot_dof(s, s->species[i]);
    return n;
}

/* absolute site positions r_ia = R_i + A(q_i) b_a, out[(i*OR_MAXS + a)*3 + k] */
void or_site_positions(const or_system *s, const double *R, const double *q, double *out) {
    for (int i = 0; i < s->N; ++i) {
        double A[9];
        or_rotation(q + 4 * i, A);
        int sp = s->species[i];
        for (int a = 0; a < s->n_sites[sp]; ++a) {
            double o[3];
            matvec(A, s->pos[sp][a], o);
            for (int k = 0; k < 3; ++k) out[(i * OR_MAXS + a) * 3 + k] = R[3 * i + k] + o[k];
        }
    }
}

/* ----------------------------------------------------- partner search (a2) */
/* Centre coordinate on the lattice of 2^32 points per box edge:
 * X = floor(x * (2^32 / L)) mod 2^32.  Differences of lattice coordinates taken
 * modulo 2^32 and read as signed 32-bit numbers are minimum-image differences. */
uint32_t or_lattice(double x, double scale /* = 4294967296.0 / L */) {
    double t = x * scale;
    double f = floor(t);
    int64_t k = (int64_t)f;
    return (uint32_t)(uint64_t)k;
}
/* Integer threshold: d2 < ceil((rc * 2^32 / L)^2)  <=>  |d| < rc on the lattice. */
uint64_t or_rc2_lattice(double rc, double L) {
    double sc = rc * 4294967296.0 / L;
    return (uint64_t)ceil(sc * sc);
}
static uint64_t lattice_d2(const uint32_t *Xi, const uint32_t *Xj) {
    uint64_t d2 = 0;
    for (int k = 0; k < 3; ++k) {
        int64_t d = (int32_t)(Xj[k] - Xi[k]);
        d2 += (uint64_t)(d * d);
    }
    return d2;
}
static void lattice_all(const or_system *s, const double *R, uint32_t *X) {
    double scale = 4294967296.0 / s->L;
    for (int i = 0; i < 3 * s->N; ++i) X[i] = or_lattice(R[i], scale);
}
/* number of partners j != i of each molecule i */
void or_partner_counts(const or_system *s, const double *R, int *counts) {
    uint32_t *X = (uint32_t *)malloc(sizeof(uint32_t) * 3 * s->N);
    lattice_all(s, R, X);
    uint64_t rc2 = or_rc2_lattice(s->rc, s->L);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < s->N; ++i) {
        int c = 0;
        for (int j = 0; j < s->N; ++j)
            if (j != i && lattice_d2(X + 3 * i, X + 3 * j) < rc2) ++c;
        counts[i] = c;
    }
    free(X);
}
/* FP64 minimum image of a centre difference (used for the interaction geometry;
 * for partners every axis component is below rc < L/2, so this image is the one
 * the lattice test used) */
static void min_image(const or_system *s, const double *Ri, const double *Rj, double *d) {
    for (int k = 0; k < 3; ++k) {
        double x = Rj[k] - Ri[k];
        d[k] = x - s->L * rint(x / s->L);
    }
}

/* ------------------------------------------------- electrostatic constants */
static double k_rf(const or_system *s) {
    double rc3 = s->rc * s->rc * s->rc;
    if (s->eps_rf <= 0) return 1.0 / (2.0 * rc3); /* conducting boundary */
    return (s->eps_rf - 1.0) / ((2.0 * s->eps_rf + 1.0) * rc3);
}
static double c_rf(const or_system *s) { return 1.0 / s->rc + k_rf(s) * s->rc * s->rc + s->crf_shift; }
static int has_dipole(const or_system *s, int sp, int a) {
    const double *m = s->dipole[sp][a];
    return m[0] != 0 || m[1] != 0 || m[2] != 0;
}

/* ------------------------------------------- site-pair interactions (a3) */
/* Interaction of owner molecule i with partner j.  d = centre minimum image
 * R_j - R_i.  Adds to the owner's force F, torque tau, energies u[3]
 * (LJ, charge-charge, dipole-dipole) and returns F_ij (force on i due to j). */
/* Site-pair sums of molecule pair (i, j), d = minimum-image R_j - R_i: force F and
 * torque tau on i, energies u[3] (LJ, charge-charge, dipole-dipole), the force
 * Fij on i from j, and wown += sum_ab (-r_ab.f_ab - 2 s_ia.f_ab): the owner share
 * of the molecular virial (summed over the partners j of i, and halved, the shares
 * add up to W = sum_{i<j} (R_i - R_j).F_ij, because the s_jb terms of the pair
 * virial move to molecule j's sum). */
static void pair_ij(const or_system *s, int i, int j, const double *Ai, const double *Aj, const double *d,
                    double *F, double *tau, double *u, double *Fij, double *wown) {
    int si = s->species[i], sj = s->species[j];
    double krf = (s->elec == 1) ? k_rf(s) : 0.0, crf = (s->elec == 1) ? c_rf(s) : 0.0;
    Fij[0] = Fij[1] = Fij[2] = 0;
    for (int a = 0; a < s->n_sites[si]; ++a) {
        double oa[3];
        matvec(Ai, s->pos[si][a], oa);
        for (int b = 0; b < s->n_sites[sj]; ++b) {
            double ob[3], r[3], f[3] = {0, 0, 0};
            matvec(Aj, s->pos[sj][b], ob);
            for (int k = 0; k < 3; ++k) r[k] = d[k] + ob[k] - oa[k]; /* from site a to site b */
            double r2 = dot3(r, r), rr = sqrt(r2);
            /* Lennard-Jones 12-6, Lorentz-Berthelot */
            if (s->lj[si][a] && s->lj[sj][b]) {
                double sig = 0.5 * (s->sigma[si][a] + s->sigma[sj][b]);
                double eps = sqrt(s->epsilon[si][a] * s->epsilon[sj][b]);
                double sr2 = sig * sig / r2, sr6 = sr2 * sr2 * sr2;
                u[0] += 4.0 * eps * (sr6 * sr6 - sr6);
                double g = -24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r2;
                for (int k = 0; k < 3; ++k) f[k] += g * r[k];
            }
            /* point charges: reaction field or Ewald real space */
            double qa = s->charge[si][a], qb = s->charge[sj][b];
            if (s->elec != 0 && qa != 0 && qb != 0) {
                double cqq = s->coulomb * qa * qb, g;
                if (s->elec == 1) {
                    u[1] += cqq * (1.0 / rr + krf * r2 - crf);
                    g = -cqq * (1.0 / (r2 * rr) - 2.0 * krf);
                } else {
                    double ar = s->alpha * rr;
                    u[1] += cqq * erfc(ar) / rr;
                    g = -cqq * (erfc(ar) / rr + 2.0 * s->alpha / sqrt(M_PI) * exp(-ar * ar)) / r2;
                }
                for (int k = 0; k < 3; ++k) f[k] += g * r[k];
            }
            /* point dipoles (reaction-field term with k_RF when elec == 1) */
            if (s->elec != 0 && has_dipole(s, si, a) && has_dipole(s, sj, b)) {
                double ma[3], mb[3];
                matvec(Ai, s->dipole[si][a], ma);
                matvec(Aj, s->dipole[sj][b], mb);
                double r5 = r2 * r2 * rr, r3 = r2 * rr, r7 = r5 * r2;
                double mab = dot3(ma, mb), mar = dot3(ma, r), mbr = dot3(mb, r), C = s->coulomb;
                u[2] += C * (mab / r3 - 3.0 * mar * mbr / r5 - 2.0 * krf * mab);
                for (int k = 0; k < 3; ++k)
                    f[k] += C * (-3.0 * mab * r[k] / r5 - 3.0 * mbr * ma[k] / r5 - 3.0 * mar * mb[k] / r5 +
                                 15.0 * mar * mbr * r[k] / r7);
                double E[3], t[3];
                for (int k = 0; k < 3; ++k) E[k] = -C * (mb[k] / r3 - 3.0 * mbr * r[k] / r5 - 2.0 * krf * mb[k]);
                cross3(ma, E, t);
                for (int k = 0; k < 3; ++k) tau[k] += t[k];
            }
            double t[3];
            cross3(oa, f, t);
            for (int k = 0; k < 3; ++k) {
                F[k] += f[k];
                Fij[k] += f[k];
                tau[k] += t[k];
            }
            *wown += -dot3(r, f) - 2.0 * dot3(oa, f);
        }
    }
}

/* ------------------------------------------------ Ewald reciprocal (a4) */
/* Direct k-space sum over the box of k = 2 pi n / L, 0 < |n_x|,|n_y|,|n_z| <= kmax
 * (tin-foil boundary):
 *   S(k)   = sum_s q_s exp(i k.r_s)
 *   U_rec  = (2 pi C / V) sum_k A(k) |S(k)|^2,       A(k) = exp(-k^2/(4 alpha^2)) / k^2
 *   F_s    = (4 pi C q_s / V) sum_k A(k) k Im(S(k)* exp(i k.r_s))
 *   W_at   = (2 pi C / V) sum_k A(k) |S(k)|^2 (1 - k^2/(2 alpha^2))  (= -dU/ds, all
 *            site coordinates and L scaled by s)
 * Site forces are returned per site slot, fsite[(i*OR_MAXS + a)*3 + k]. */
void or_ewald_reciprocal(const or_system *s, const double *R, const double *q, double *fsite, double *U_rec,
                         double *W_at) {
    int N = s->N;
    double *pos = (double *)malloc(sizeof(double) * 3 * OR_MAXS * N);
    or_site_positions(s, R, q, pos);
    int nx = s->kmax[0], ny = s->kmax[1], nz = s->kmax[2];
    int NK = (2 * nx + 1) * (2 * ny + 1) * (2 * nz + 1);
    double *Sre = (double *)calloc(NK, sizeof(double)), *Sim = (double *)calloc(NK, sizeof(double));
    double *Ak = (double *)calloc(NK, sizeof(double)), *kv = (double *)calloc(3 * NK, sizeof(double));
    double *uk = (double *)calloc(NK, sizeof(double)), *wk = (double *)calloc(NK, sizeof(double));
    double V = s->L * s->L * s->L, C = s->coulomb, tw = 2.0 * M_PI / s->L;
#pragma omp parallel for schedule(dynamic, 16)
    for (int m = 0; m < NK; ++m) {
        int ix = m / ((2 * ny + 1) * (2 * nz + 1)) - nx;
        int iy = (m / (2 * nz + 1)) % (2 * ny + 1) - ny;
        int iz = m % (2 * nz + 1) - nz;
        if (ix == 0 && iy == 0 && iz == 0) continue;
        double k[3] = {tw * ix, tw * iy, tw * iz}, k2 = dot3(k, k);
        double sr = 0, si = 0;
        for (int i = 0; i < N; ++i) {
            int sp = s->species[i];
            for (int a = 0; a < s->n_sites[sp]; ++a) {
                double qa = s->charge[sp][a];
                if (qa == 0) continue;
                double ph = dot3(k, pos + (i * OR_MAXS + a) * 3);
                sr += qa * cos(ph);
                si += qa * sin(ph);
            }
        }
        Sre[m] = sr; Sim[m] = si;
        Ak[m] = exp(-k2 / (4.0 * s->alpha * s->alpha)) / k2;
        for (int c = 0; c < 3; ++c) kv[3 * m + c] = k[c];
        double e = 2.0 * M_PI * C / V * Ak[m] * (sr * sr + si * si);
        uk[m] = e;
        wk[m] = e * (1.0 - k2 / (2.0 * s->alpha * s->alpha));
    }
    double U = 0, W = 0;
    for (int m = 0; m < NK; ++m) { U += uk[m]; W += wk[m]; }
    *U_rec = U; *W_at = W;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        int sp = s->species[i];
        for (int a = 0; a < OR_MAXS; ++a) {
            double *f = fsite + (i * OR_MAXS + a) * 3;
            f[0] = f[1] = f[2] = 0;
            if (a >= s->n_sites[sp] || s->charge[sp][a] == 0) continue;
            const double *p = pos + (i * OR_MAXS + a) * 3;
            double pre = 4.0 * M_PI * C * s->charge[sp][a] / V;
            for (int m = 0; m < NK; ++m) {
                if (Ak[m] == 0) continue;
                double ph = dot3(kv + 3 * m, p);
                double im = Sre[m] * sin(ph) - Sim[m] * cos(ph);
                for (int c = 0; c < 3; ++c) f[c] += pre * Ak[m] * kv[3 * m + c] * im;
            }
        }
    }
    free(pos); free(Sre); free(Sim); free(Ak); free(kv); free(uk); free(wk);
}

/* Ewald constants: self term, intramolecular (excluded) pairs, neutralising
 * background for a net charge Q. */
void or_ewald_constants(const or_system *s, double *U_self, double *U_intra, double *U_bg) {
    double C = s->coulomb, sq2 = 0, Q = 0, intra = 0;
    for (int i = 0; i < s->N; ++i) {
        int sp = s->species[i];
        for (int a = 0; a < s->n_sites[sp]; ++a) {
            sq2 += s->charge[sp][a] * s->charge[sp][a];
            Q += s->charge[sp][a];
            for (int b = a + 1; b < s->n_sites[sp]; ++b) {
                double qq = s->charge[sp][a] * s->charge[sp][b];
                if (qq == 0) continue;
                double r[3];
                for (int k = 0; k < 3; ++k) r[k] = s->pos[sp][b][k] - s->pos[sp][a][k];
                double rr = sqrt(dot3(r, r));
                intra += qq * erf(s->alpha * rr) / rr;
            }
        }
    }
    double V = s->L * s->L * s->L;
    *U_self = -C * s->alpha / sqrt(M_PI) * sq2;
    *U_intra = -C * intra;
    *U_bg = -M_PI * C * Q * Q / (2.0 * V * s->alpha * s->alpha);
}

/* ------------------------------------- LJ long-range correction (site-site) */
/* U_LRC = (2 pi / V) sum_{a,b} N_a N_b int_rc^inf r^2 u_ab(r) dr
 * P_LRC = -(2 pi / (3 V^2)) sum_{a,b} N_a N_b int_rc^inf r^3 u'_ab(r) dr
 * sums over ordered pairs of LJ site kinds (species, site), N_a = their counts. */
void or_lrc(const or_system *s, double *U, double *P) {
    int cnt[OR_MAXSP] = {0};
    for (int i = 0; i < s->N; ++i) cnt[s->species[i]]++;
    double V = s->L * s->L * s->L, rc = s->rc, u = 0, p = 0;
    for (int s1 = 0; s1 < s->n_species; ++s1)
        for (int a = 0; a < s->n_sites[s1]; ++a)
            for (int s2 = 0; s2 < s->n_species; ++s2)
                for (int b = 0; b < s->n_sites[s2]; ++b) {
                    if (!s->lj[s1][a] || !s->lj[s2][b]) continue;
                    double sig = 0.5 * (s->sigma[s1][a] + s->sigma[s2][b]);
                    double eps = sqrt(s->epsilon[s1][a] * s->epsilon[s2][b]);
                    double x3 = pow(sig / rc, 3), x9 = x3 * x3 * x3, s3 = sig * sig * sig;
                    double Iu = 4.0 * eps * s3 * (x9 / 9.0 - x3 / 3.0);
                    double Ip = 4.0 * eps * s3 * (-4.0 / 3.0 * x9 + 2.0 * x3);
                    double nn = (double)cnt[s1] * (double)cnt[s2];
                    u += nn * Iu;
                    p += nn * Ip;
                }
    *U = 2.0 * M_PI / V * u;
    *P = -2.0 * M_PI / (3.0 * V * V) * p;
}

/* --------------------------------------------------- total forces (a3+a4) */
/* Per-molecule force F (N x 3) and torque tau (N x 3) on the configuration
 * (R, q), plus the energy/virial breakdown terms[OR_NTERMS].
 * Molecular virial W = sum_{i<j} (R_i - R_j).F_ij over partner pairs (owner
 * computes: half of each owner's sum), plus reciprocal and background parts. */
void or_forces_mol(const or_system *s, const double *R, const double *q, double *F, double *tau, double *terms,
                   double *mol);
void or_forces(const or_system *s, const double *R, const double *q, double *F, double *tau, double *terms) {
    or_forces_mol(s, R, q, F, tau, terms, NULL);
}
/* as or_forces; mol (may be NULL) receives per molecule i the shares
 * 1/2 sum_j of the LJ, charge-charge and dipole-dipole pair energies and the
 * owner share of the molecular virial, 1/2 (sum_j sum_ab -r_ab.f_ab
 * - 2 sum_a s_ia.F_ia) with F_ia the total force on site a (N x 4).  The paper
 * defines W only as a system total; the shares add up to it (the pair form
 * sum_j (R_i - R_j).F_ij gives other shares with the same total). */
void or_forces_mol(const or_system *s, const double *R, const double *q, double *F, double *tau, double *terms,
                   double *mol) {
    int N = s->N;
    uint32_t *X = (uint32_t *)malloc(sizeof(uint32_t) * 3 * N);
    lattice_all(s, R, X);
    uint64_t rc2 = or_rc2_lattice(s->rc, s->L);
    double *A = (double *)malloc(sizeof(double) * 9 * N);
    for (int i = 0; i < N; ++i) or_rotation(q + 4 * i, A + 9 * i);
    double *Ui = (double *)calloc(3 * N, sizeof(double)), *Wi = (double *)calloc(N, sizeof(double));
    double *Wo = (double *)calloc(N, sizeof(double));
    int *np = (int *)calloc(N, sizeof(int));
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < N; ++i) {
        double f[3] = {0, 0, 0}, t[3] = {0, 0, 0}, u[3] = {0, 0, 0}, w = 0, wo = 0;
        for (int j = 0; j < N; ++j) {
            if (j == i || !(lattice_d2(X + 3 * i, X + 3 * j) < rc2)) continue;
            double d[3], Fij[3];
            min_image(s, R + 3 * i, R + 3 * j, d);
            pair_ij(s, i, j, A + 9 * i, A + 9 * j, d, f, t, u, Fij, &wo);
            w += -dot3(d, Fij);
            np[i]++;
        }
        for (int k = 0; k < 3; ++k) { F[3 * i + k] = f[k]; tau[3 * i + k] = t[k]; Ui[3 * i + k] = u[k]; }
        Wi[i] = w;
        Wo[i] = wo;
    }
    if (mol)
        for (int i = 0; i < N; ++i) {
            for (int k = 0; k < 3; ++k) mol[4 * i + k] = 0.5 * Ui[3 * i + k];
            mol[4 * i + 3] = 0.5 * Wo[i];
        }
    free(Wo);
    for (int k = 0; k < OR_NTERMS; ++k) terms[k] = 0;
    long long npairs = 0;
    for (int i = 0; i < N; ++i) {
        terms[T_ULJ] += 0.5 * Ui[3 * i];
        terms[T_UQQ] += 0.5 * Ui[3 * i + 1];
        terms[T_UDD] += 0.5 * Ui[3 * i + 2];
        terms[T_WPAIR] += 0.5 * Wi[i];
        npairs += np[i];
    }
    terms[T_NPAIRS] = (double)(npairs / 2);
    if (s->elec == 2) {
        double *fs = (double *)malloc(sizeof(double) * 3 * OR_MAXS * N), Ur, Wat, Wcorr = 0;
        or_ewald_reciprocal(s, R, q, fs, &Ur, &Wat);
        for (int i = 0; i < N; ++i) {
            int sp = s->species[i];
            for (int a = 0; a < s->n_sites[sp]; ++a) {
                double o[3], t[3];
                const double *fa = fs + (i * OR_MAXS + a) * 3;
                matvec(A + 9 * i, s->pos[sp][a], o);
                cross3(o, fa, t);
                for (int k = 0; k < 3; ++k) { F[3 * i + k] += fa[k]; tau[3 * i + k] += t[k]; }
                Wcorr += dot3(fa, o);
            }
        }
        terms[T_UREC] = Ur;
        terms[T_WREC] = Wat - Wcorr; /* molecular virial: W_mol = W_atomic - sum_s F_s . s_s */
        or_ewald_constants(s, &terms[T_USELF], &terms[T_UINTRA], &terms[T_UBG]);
        terms[T_WBG] = 3.0 * terms[T_UBG]; /* U_bg ~ 1/V */
        free(fs);
    }
    if (s->lrc) or_lrc(s, &terms[T_ULRC], &terms[T_PLRC]);
    terms[T_UTOT] = terms[T_ULJ] + terms[T_UQQ] + terms[T_UDD] + terms[T_UREC] + terms[T_USELF] + terms[T_UINTRA] +
                    terms[T_UBG] + terms[T_ULRC];
    terms[T_WTOT] = terms[T_WPAIR] + terms[T_WREC] + terms[T_WBG];
    free(X); free(A); free(Ui); free(Wi); free(np);
}

/* ---------------------------------------------------- kinetic energy (a6) */
/* ke[0] = translational, ke[1] = rotational kinetic energy in the energy unit.
 * v: centre velocities, Lang: space-frame angular momenta, rotational part
 * evaluated with the orientations q: KE_rot = 1/2 L_b . I^-1 L_b, L_b = A^T L. */
void or_kinetic(const or_system *s, const double *q, const double *v, const double *Lang, double *ke) {
    double kt = 0, kr = 0;
    for (int i = 0; i < s->N; ++i) {
        int sp = s->species[i];
        double M = mol_mass(s, sp);
        kt += 0.5 * M * dot3(v + 3 * i, v + 3 * i);
        double Iinv[3], A[9], Lb[3];
        mol_inv_inertia(s, sp, Iinv);
        or_rotation(q + 4 * i, A);
        matTvec(A, Lang + 3 * i, Lb);
        for (int k = 0; k < 3; ++k) kr += 0.5 * Lb[k] * Lb[k] * Iinv[k];
    }
    ke[0] = kt / s->kconv;
    ke[1] = kr / s->kconv;
}

/* pressure from the virial theorem: P = (2 KE_tr / 3 + W / 3) / V + P_LRC */
double or_pressure(const or_system *s, double ke_tr, const double *terms) {
    double V = s->L * s->L * s->L;
    return (2.0 * ke_tr / 3.0 + terms[T_WTOT] / 3.0) / V + terms[T_PLRC];
}

/* -------------------------------- Massieu potential derivatives (Sec. 2, Eq. 1) */
/* Volume derivatives of the potential energy at fixed scaled centres and fixed
 * orientations (the scaling that defines the molecular virial).  With
 * r_ab(lambda) = lambda d_ij + s_jb - s_ia and V' = lambda^3 V:
 *   dU/dV   = g'(1) / (3 V),   d2U/dV2 = (g''(1) - 2 g'(1)) / (9 V^2),
 *   g'  = sum_ab u'(r) (r.d) / r,
 *   g'' = sum_ab [u''(r) (r.d)^2 / r^2 + u'(r) / r (d^2 - (r.d)^2 / r^2)],
 * summed over partner pairs, plus the long-range parts -P_LRC and 2 P_LRC / V:
 * the mean-field tail pressure and its volume derivative (reading: the paper
 * leaves the LRC of these derivatives to its supplement; -P_LRC is what makes
 * -dU/dV the residual pressure).  LJ and point charges with the reaction field
 * (whose k_RF r^2 and c_RF terms drop out of neutral molecule pairs) or without
 * electrostatics; the paper does not combine these derivatives with Ewald, and
 * dipoles are not covered.  out[0] = dU/dV, out[1] = d2U/dV2. */
void or_volume_derivatives(const or_system *s, const double *R, const double *q, double *out) {
    int N = s->N;
    uint32_t *X = (uint32_t *)malloc(sizeof(uint32_t) * 3 * N);
    lattice_all(s, R, X);
    uint64_t rc2 = or_rc2_lattice(s->rc, s->L);
    double *A = (double *)malloc(sizeof(double) * 9 * N);
    for (int i = 0; i < N; ++i) or_rotation(q + 4 * i, A + 9 * i);
    double krf = (s->elec == 1) ? k_rf(s) : 0.0, g1 = 0, g2 = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : g1, g2)
    for (int i = 0; i < N; ++i) {
        int si = s->species[i];
        for (int j = 0; j < N; ++j) {
            if (j == i || !(lattice_d2(X + 3 * i, X + 3 * j) < rc2)) continue;
            int sj = s->species[j];
            double d[3];
            min_image(s, R + 3 * i, R + 3 * j, d);
            double d2 = dot3(d, d);
            for (int a = 0; a < s->n_sites[si]; ++a) {
                double oa[3];
                matvec(A + 9 * i, s->pos[si][a], oa);
                for (int b = 0; b < s->n_sites[sj]; ++b) {
                    double ob[3], r[3];
                    matvec(A + 9 * j, s->pos[sj][b], ob);
                    for (int k = 0; k < 3; ++k) r[k] = d[k] + ob[k] - oa[k];
                    double r2 = dot3(r, r), rr = sqrt(r2), rd = dot3(r, d), u1 = 0, u2 = 0;  /* u', u'' */
                    if (s->lj[si][a] && s->lj[sj][b]) {
                        double sig = 0.5 * (s->sigma[si][a] + s->sigma[sj][b]);
                        double eps = sqrt(s->epsilon[si][a] * s->epsilon[sj][b]);
                        double sr6 = pow(sig * sig / r2, 3), sr12 = sr6 * sr6;
                        u1 += 4.0 * eps * (-12.0 * sr12 + 6.0 * sr6) / rr;
                        u2 += 4.0 * eps * (156.0 * sr12 - 42.0 * sr6) / r2;
                    }
                    double qa = s->charge[si][a], qb = s->charge[sj][b];
                    if (s->elec == 1 && qa != 0 && qb != 0) {
                        double cqq = s->coulomb * qa * qb;   /* u = cqq (1/r + k_RF r^2 - c_RF) */
                        u1 += cqq * (-1.0 / r2 + 2.0 * krf * rr);
                        u2 += cqq * (2.0 / (r2 * rr) + 2.0 * krf);
                    }
                    g1 += u1 * rd / rr;
                    g2 += u2 * rd * rd / r2 + u1 / rr * (d2 - rd * rd / r2);
                }
            }
        }
    }
    free(X);
    free(A);
    double V = s->L * s->L * s->L, Ul = 0, Pl = 0;
    if (s->lrc) or_lrc(s, &Ul, &Pl);
    g1 *= 0.5;  /* each pair was visited from both molecules */
    g2 *= 0.5;
    out[0] = g1 / (3.0 * V) - Pl;
    out[1] = (g2 - 2.0 * g1) / (9.0 * V * V) + 2.0 * Pl / V;
}

/* Residual Massieu derivatives A^r_mn = beta^m rho^n d^(m+n)(A^r/(N k T)) /
 * d beta^m d rho^n (Eq. 1; k = 1) of the NVT ensemble, from canonical averages.
 * Written out from f = -(1/N) ln(Z_c / V^N), Z_c the configurational integral
 * taken over scaled centres, so that
 *   df/dbeta = <U>/N,  df/dV = beta <U_V>/N,  rho d/drho = -V d/dV,
 *   rho^2 d^2/drho^2 = 2 V d/dV + V^2 d^2/dV^2,
 *   d<X>/dbeta = -cov(X, U),  d<X>/dV = <X_V> - beta cov(X, U_V),
 * with U_V = dU/dV and U_VV = d2U/dV2 at fixed scaled centres.  This gives
 *   A10 = beta <U> / N                A01 = -beta V <U_V> / N
 *   A20 = -beta^2 var(U) / N          A11 = -(beta V / N) (<U_V> - beta cov(U, U_V))
 *   A02 = (beta / N) (2 V <U_V> + V^2 (<U_VV> - beta var(U_V)))
 *   A30 = beta^3 <dU^3> / N
 *   A21 = (beta^2 V / N) (2 cov(U, U_V) - beta <dU^2 dU_V>)
 *   A12 = (beta / N) (2 V (<U_V> - beta cov(U, U_V))
 *         + V^2 (<U_VV> - 2 beta var(U_V) - beta cov(U, U_VV) + beta^2 <dU dU_V^2>))
 * (dX = X - <X>).  acc holds the sample weight and weighted sums over samples of
 * x = U - U0, y = U_V - V0 and w = U_VV (the shifts keep the central moments
 * free of cancellation):
 *   acc = {n, x, x^2, x^3, y, y^2, x y, x^2 y, x y^2, w, x w}.
 * out = {A10, A01, A20, A11, A02, A30, A21, A12}. */
void or_massieu(const double *acc, double U0, double V0, double beta, double V, int N, double *out) {
    double n = acc[0];
    double mx = acc[1] / n, my = acc[4] / n, mw = acc[9] / n;
    double vx = acc[2] / n - mx * mx, vy = acc[5] / n - my * my, cxy = acc[6] / n - mx * my;
    double k3 = acc[3] / n - 3.0 * mx * acc[2] / n + 2.0 * mx * mx * mx;
    double m21 = acc[7] / n - 2.0 * mx * acc[6] / n - my * acc[2] / n + 2.0 * mx * mx * my;
    double m12 = acc[8] / n - 2.0 * my * acc[6] / n - mx * acc[5] / n + 2.0 * mx * my * my;
    double cxw = acc[10] / n - mx * mw;
    double U = U0 + mx, UV = V0 + my, b = beta;
    out[0] = b * U / N;
    out[1] = -b * V * UV / N;
    out[2] = -b * b * vx / N;
    out[3] = -(b * V / N) * (UV - b * cxy);
    out[4] = (b / N) * (2.0 * V * UV + V * V * (mw - b * vy));
    out[5] = b * b * b * k3 / N;
    out[6] = (b * b * V / N) * (2.0 * cxy - b * m21);
    out[7] = (b / N) * (2.0 * V * (UV - b * cxy) + V * V * (mw - 2.0 * b * vy - b * cxw + b * b * m12));
}

/* ------------------------------ Green-Kubo electric conductivity (Sec. 4, Eqs. 3-4) */
/* Electric current flux j_e = sum_k q_k v_k over the molecules with a net charge
 * q_k = sum_a q_a (the neutral ones drop out), v_k the centre velocities. */
void or_current(const or_system *s, const double *v, double *j) {
    j[0] = j[1] = j[2] = 0.0;
    for (int k = 0; k < s->N; ++k) {
        int sp = s->species[k];
        double qk = 0.0;
        for (int a = 0; a < s->n_sites[sp]; ++a) qk += s->charge[sp][a];
        for (int c = 0; c < 3; ++c) j[c] += qk * v[3 * k + c];
    }
}

/* Autocorrelation of a flux series j[t][3], t = 0 .. n-1, sampled every extended
 * time step, over all time origins: acf[m] = (1/(n - m)) sum_{t=m}^{n-1}
 * j(t).j(t-m) for m < min(n, n_lags) (0 beyond).  The dot product sums the three
 * spatial elements, as the 1/3 in the conductivity expects. */
void or_flux_acf(const double *j, int n, int n_lags, double *acf) {
    for (int m = 0; m < n_lags; ++m) {
        double c = 0.0;
        for (int t = m; t < n; ++t) c += dot3(j + 3 * t, j + 3 * (t - m));
        acf[m] = m < n ? c / (double)(n - m) : 0.0;
    }
}

/* sigma = 1/(3 V kB T) int_0^tmax <j_e(t).j_e(0)> dt with the trapezoidal rule over
 * the n_lags lags of spacing dt_ext.  Units: q in e, v in A/fs, V in A^3, T in K,
 * dt in fs -> sigma in S/m; reduced = 1: all quantities reduced, sigma reduced. */
double or_conductivity(const double *acf, int n_lags, double dt_ext, double V, double T, int reduced) {
    double integral = 0.0;
    for (int m = 0; m < n_lags; ++m) integral += ((m == 0 || m == n_lags - 1) ? 0.5 : 1.0) * acf[m];
    integral *= dt_ext;
    if (reduced) return integral / (3.0 * V * T);
    const double e = 1.602176634e-19, kB = 1.380649e-23;
    /* (e A/fs)^2 fs = e^2 1e10 m^2/s^2 1e-15 s; V in 1e-30 m^3 */
    return integral * e * e * 1e-5 / (3.0 * V * 1e-30 * kB * T);
}

/* ---------------------------- thermal conductivity of mixtures (Sec. 4, Eqs. 5-6) */
/* Microscopic heat flow of a configuration with centre velocities v and
 * space-frame angular momenta Lang:
 *   J_q = sum_k (E_k - h_{s(k)}) v_k + 1/2 sum_k sum_{l != k} r_kl (F_kl.v_k + tau_kl.w_k)
 * E_k = 1/2 M v_k^2 + 1/2 w_k.I.w_k + 1/2 sum_l u_kl (K), r_kl = R_k - R_l (minimum
 * image), F_kl and tau_kl the force and torque on k from l, w_k = A I^-1 A^T L_k
 * the angular velocity, h the per-molecule partial enthalpy of each species (K).
 * Reading of Eq. 6: its Gamma_kl is the orientational gradient of u, i.e. minus
 * the torque, so that the bracket is minus the power F_kl.v_k + tau_kl.w_k of the
 * pair on molecule k; without the h term J_q is then d/dt sum_k R_k E_k.  LJ and
 * point charges, reaction field or none (the pair sums of pair_ij).  J in K A/fs. */
void or_heat_flux(const or_system *s, const double *R, const double *q, const double *v, const double *Lang,
                  const double *h, double *J) {
    int N = s->N;
    uint32_t *X = (uint32_t *)malloc(sizeof(uint32_t) * 3 * N);
    lattice_all(s, R, X);
    uint64_t rc2 = or_rc2_lattice(s->rc, s->L);
    double *A = (double *)malloc(sizeof(double) * 9 * N), *w = (double *)malloc(sizeof(double) * 3 * N);
    for (int k = 0; k < N; ++k) {
        int sp = s->species[k];
        double Iinv[3], Lb[3], wb[3];
        or_rotation(q + 4 * k, A + 9 * k);
        mol_inv_inertia(s, sp, Iinv);
        matTvec(A + 9 * k, Lang + 3 * k, Lb);
        for (int c = 0; c < 3; ++c) wb[c] = Iinv[c] * Lb[c];
        matvec(A + 9 * k, wb, w + 3 * k);
    }
    double J0 = 0, J1 = 0, J2 = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : J0, J1, J2)
    for (int k = 0; k < N; ++k) {
        int sp = s->species[k];
        double uk = 0, jc[3] = {0, 0, 0};
        for (int l = 0; l < N; ++l) {
            if (l == k || !(lattice_d2(X + 3 * k, X + 3 * l) < rc2)) continue;
            double d[3], f[3] = {0, 0, 0}, t[3] = {0, 0, 0}, u[3] = {0, 0, 0}, Fkl[3], wo = 0;
            min_image(s, R + 3 * k, R + 3 * l, d);  /* R_l - R_k */
            pair_ij(s, k, l, A + 9 * k, A + 9 * l, d, f, t, u, Fkl, &wo);
            uk += u[0] + u[1] + u[2];
            double P = dot3(Fkl, v + 3 * k) + dot3(t, w + 3 * k);
            for (int c = 0; c < 3; ++c) jc[c] += 0.5 * (-d[c]) * P;
        }
        double Iinv[3], Lb[3];
        mol_inv_inertia(s, sp, Iinv);
        matTvec(A + 9 * k, Lang + 3 * k, Lb);
        double ke = 0.5 * mol_mass(s, sp) * dot3(v + 3 * k, v + 3 * k);
        for (int c = 0; c < 3; ++c) ke += 0.5 * Iinv[c] * Lb[c] * Lb[c];
        double Ek = ke / s->kconv + 0.5 * uk - h[sp];
        J0 += Ek * v[3 * k] + jc[0];
        J1 += Ek * v[3 * k + 1] + jc[1];
        J2 += Ek * v[3 * k + 2] + jc[2];
    }
    J[0] = J0;
    J[1] = J1;
    J[2] = J2;
    free(X);
    free(A);
    free(w);
}

/* lambda = 1/(V kB T^2) int <J^x(t) J^x(0)> dt, averaged over the three elements:
 * acf holds <J(t).J(0)> (the sum of the three), so lambda = trapz(acf) dt / (3 V T^2)
 * in K^2 A^2/fs^2 fs / (A^3 K^2) scaled to W/(m K) (kB in J/K, 1 A/fs = 1e5 m/s);
 * reduced = 1: reduced units. */
double or_thermal_conductivity(const double *acf, int n_lags, double dt_ext, double V, double T, int reduced) {
    double integral = 0.0;
    for (int m = 0; m < n_lags; ++m) integral += ((m == 0 || m == n_lags - 1) ? 0.5 : 1.0) * acf[m];
    integral *= dt_ext;
    if (reduced) return integral / (3.0 * V * T * T);
    const double kB = 1.380649e-23;
    /* (K A/fs)^2 fs -> kB^2 1e10 m^2/s^2 1e-15 s; / (V 1e-30 m^3 kB K^2) */
    return integral * kB * 1e-5 / (3.0 * V * 1e-30 * T * T);
}

/* ---------------------------------- residence time, solvation number (Sec. 4, Eq. 7) */
/* Residence correlation of molecules of species sj around molecules of species si
 * over a series of T configurations R[t][N][3] sampled every extended time step.
 * "Within r_shell" is the minimum-image centre distance, decided on the integer
 * centre lattice as the partner search decides the cut-off (R4).  Following Impey
 * et al., molecule k (of species sj, k != i) counts at lag tau for origin t0 and
 * centre i if it is in the shell at t0 and at t0 + tau and was never outside for
 * more than t_star consecutive samples in between.  For every origin t0 and centre
 * i with n_i(t0) > 0 shell members, the fraction (count at tau) / n_i(t0) enters
 * the average at lag tau, for tau < min(n_lags, T - t0):
 *   corr[tau] = sum over (t0, i) of fraction / number of (t0, i) terms.
 * The solvation number is the mean of n_i(t0) over all origins and centres. */
void or_residence(const or_system *s, const double *R, int T, int si, int sj, double r_shell, int t_star,
                  int n_lags, double *corr, double *solvation) {
    int N = s->N;
    uint64_t r2 = or_rc2_lattice(r_shell, s->L);
    uint32_t *X = (uint32_t *)malloc(sizeof(uint32_t) * 3 * N * (size_t)T);
    for (int t = 0; t < T; ++t) lattice_all(s, R + (size_t)t * 3 * N, X + (size_t)t * 3 * N);
    double *num = (double *)calloc(n_lags, sizeof(double));
    double *cnt = (double *)calloc(n_lags, sizeof(double));
    double nsum = 0.0, ncount = 0.0;
#define INSIDE(t, i, k) (lattice_d2(X + ((size_t)(t) * N + (i)) * 3, X + ((size_t)(t) * N + (k)) * 3) < r2)
    for (int t0 = 0; t0 < T; ++t0)
        for (int i = 0; i < N; ++i) {
            if (s->species[i] != si) continue;
            int n0 = 0;
            for (int k = 0; k < N; ++k)
                if (k != i && s->species[k] == sj && INSIDE(t0, i, k)) ++n0;
            nsum += n0;
            ncount += 1.0;
            if (n0 == 0) continue;
            for (int tau = 0; tau < n_lags && t0 + tau < T; ++tau) {
                int alive = 0;
                for (int k = 0; k < N; ++k) {
                    if (k == i || s->species[k] != sj || !INSIDE(t0, i, k)) continue;
                    int out = 0, gone = 0;
                    for (int u = 1; u <= tau && !gone; ++u) {  /* excursions up to tau */
                        if (INSIDE(t0 + u, i, k)) out = 0;
                        else if (++out > t_star) gone = 1;
                    }
                    if (!gone && INSIDE(t0 + tau, i, k)) ++alive;
                }
                num[tau] += (double)alive / n0;
                cnt[tau] += 1.0;
            }
        }
#undef INSIDE
    for (int tau = 0; tau < n_lags; ++tau) corr[tau] = cnt[tau] > 0 ? num[tau] / cnt[tau] : 0.0;
    *solvation = ncount > 0 ? nsum / ncount : 0.0;
    free(X);
    free(num);
    free(cnt);
}

/* ------------------------------------------------------ integrators (a5) */
/* thermo record per step: U, W, KE_tr, KE_rot, P (after the step) */
static void record(const or_system *s, const double *q, const double *v, const double *Lang, const double *terms,
                   double *out) {
    double ke[2];
    or_kinetic(s, q, v, Lang, ke);
    out[0] = terms[T_UTOT];
    out[1] = terms[T_WTOT];
    out[2] = ke[0];
    out[3] = ke[1];
    out[4] = or_pressure(s, ke[0], terms);
}

/* Velocity Verlet for molecules without rotational freedom (single sites):
 *   v(t+dt/2) = v(t) + dt/2 F(t)/M;  R(t+dt) = R(t) + dt v(t+dt/2);
 *   F(t+dt);  v(t+dt) = v(t+dt/2) + dt/2 F(t+dt)/M.
 * thermo (may be NULL) receives 5 numbers per step. */
void or_run_vv(const or_system *s, double *R, double *v, double dt, int nsteps, double *thermo) {
    int N = s->N;
    double *F = (double *)malloc(sizeof(double) * 3 * N), *tau = (double *)malloc(sizeof(double) * 3 * N);
    double *q = (double *)calloc(4 * N, sizeof(double)), *Lz = (double *)calloc(3 * N, sizeof(double));
    double terms[OR_NTERMS];
    for (int i = 0; i < N; ++i) q[4 * i] = 1.0;
    or_forces(s, R, q, F, tau, terms);
    for (int n = 0; n < nsteps; ++n) {
        for (int i = 0; i < N; ++i) {
            double M = mol_mass(s, s->species[i]);
            for (int k = 0; k < 3; ++k) {
                v[3 * i + k] += 0.5 * dt * s->kconv * F[3 * i + k] / M;
                R[3 * i + k] += dt * v[3 * i + k];
            }
        }
        or_forces(s, R, q, F, tau, terms);
        for (int i = 0; i < N; ++i) {
            double M = mol_mass(s, s->species[i]);
            for (int k = 0; k < 3; ++k) v[3 * i + k] += 0.5 * dt * s->kconv * F[3 * i + k] / M;
        }
        if (thermo) record(s, q, v, Lz, terms, thermo + 5 * n);
    }
    free(F); free(tau); free(q); free(Lz);
}

/* quaternion product p (x) r */
static void qmul(const double *p, const double *r, double *o) {
    o[0] = p[0] * r[0] - p[1] * r[1] - p[2] * r[2] - p[3] * r[3];
    o[1] = p[0] * r[1] + p[1] * r[0] + p[2] * r[3] - p[3] * r[2];
    o[2] = p[0] * r[2] - p[1] * r[3] + p[2] * r[0] + p[3] * r[1];
    o[3] = p[0] * r[3] + p[1] * r[2] - p[2] * r[1] + p[3] * r[0];
}

/* One rotational update q(t) -> q(t+dt) with the space-frame angular momentum L
 * held at its half-step value: implicit midpoint rule
 *   q1 = q0 + dt * 1/2 * qm (x) (0, w_b(qm)),   qm = (q0 + q1)/2,
 *   w_b = I^-1 A(qm/|qm|)^T L,
 * solved by n_iter fixed-point sweeps starting from q1 = q0, then q1 normalised. */
static void rotate(const double *Iinv, const double *q0, const double *Lsp, double dt, int n_iter, double *q1) {
    for (int k = 0; k < 4; ++k) q1[k] = q0[k];
    for (int it = 0; it < n_iter; ++it) {
        double qm[4], qh[4], A[9], Lb[3], w[4], dq[4];
        for (int k = 0; k < 4; ++k) qm[k] = 0.5 * (q0[k] + q1[k]);
        double nm = sqrt(qm[0] * qm[0] + qm[1] * qm[1] + qm[2] * qm[2] + qm[3] * qm[3]);
        for (int k = 0; k < 4; ++k) qh[k] = qm[k] / nm;
        or_rotation(qh, A);
        matTvec(A, Lsp, Lb);
        w[0] = 0;
        for (int k = 0; k < 3; ++k) w[k + 1] = Iinv[k] * Lb[k];
        qmul(qm, w, dq);
        for (int k = 0; k < 4; ++k) q1[k] = q0[k] + 0.5 * dt * dq[k];
    }
    double n1 = sqrt(q1[0] * q1[0] + q1[1] * q1[1] + q1[2] * q1[2] + q1[3] * q1[3]);
    for (int k = 0; k < 4; ++k) q1[k] /= n1;
}

/* Leapfrog for rigid molecules.  State: R(t), q(t), v(t-dt/2), L(t-dt/2).
 *   F(t), tau(t) from (R(t), q(t));
 *   v' = v + dt F/M,  L' = L + dt tau            (times kconv: energy -> mass units)
 *   if T0 > 0: lambda = sqrt(T0 / T'), T' = 2 (KE_tr(v') + KE_rot(L', q(t))) / N_dof,
 *              v' *= lambda, L' *= lambda        (isokinetic velocity scaling)
 *   R(t+dt) = R(t) + dt v';  q(t+dt) = rotate(q(t), L');  v, L <- v', L'.
 * thermo (may be NULL) receives 5 numbers per step (after the step, with the new
 * forces); tstat (may be NULL) receives the scaled temperature T' per step. */
void or_run_leapfrog(const or_system *s, double *R, double *q, double *v, double *Lang, double dt, int nsteps,
                     double T0, int n_iter, double *thermo, double *tstat) {
    int N = s->N;
    double *F = (double *)malloc(sizeof(double) * 3 * N), *tau = (double *)malloc(sizeof(double) * 3 * N);
    double terms[OR_NTERMS];
    int ndof = or_ndof(s);
    or_forces(s, R, q, F, tau, terms);
    for (int n = 0; n < nsteps; ++n) {
        for (int i = 0; i < N; ++i) {
            double M = mol_mass(s, s->species[i]);
            for (int k = 0; k < 3; ++k) {
                v[3 * i + k] += dt * s->kconv * F[3 * i + k] / M;
                Lang[3 * i + k] += dt * s->kconv * tau[3 * i + k];
            }
        }
        if (T0 > 0) {
            double ke[2];
            or_kinetic(s, q, v, Lang, ke);
            double Tp = 2.0 * (ke[0] + ke[1]) / ndof, lam = sqrt(T0 / Tp);
            for (int k = 0; k < 3 * N; ++k) { v[k] *= lam; Lang[k] *= lam; }
            if (tstat) {
                or_kinetic(s, q, v, Lang, ke);
                tstat[n] = 2.0 * (ke[0] + ke[1]) / ndof;
            }
        }
        for (int i = 0; i < N; ++i) {
            double Iinv[3], q1[4];
            mol_inv_inertia(s, s->species[i], Iinv);
            for (int k = 0; k < 3; ++k) R[3 * i + k] += dt * v[3 * i + k];
            if (Iinv[0] != 0 || Iinv[1] != 0 || Iinv[2] != 0) {
                rotate(Iinv, q + 4 * i, Lang + 3 * i, dt, n_iter, q1);
                for (int k = 0; k < 4; ++k) q[4 * i + k] = q1[k];
            }
        }
        or_forces(s, R, q, F, tau, terms);
        if (thermo) record(s, q, v, Lang, terms, thermo + 5 * n);
    }
    free(F); free(tau);
}

/* ------------------------------------------------------------- RDF (a7) */
/* Integer histogram of intermolecular LJ-site pairs at site minimum image,
 * r < r_max, bin = floor(r / (r_max / nbins)).  Site kinds t = (species, LJ site)
 * are numbered in species-then-site order; unordered kind pairs t1 <= t2 index
 * the rows of counts[n_pairs][nbins] in upper-triangle row-major order.
 * Each unordered molecule pair i < j contributes all its LJ-site pairs once. */
int or_rdf_kinds(const or_system *s, int *kind /* [OR_MAXSP][OR_MAXS] */) {
    int t = 0;
    for (int sp = 0; sp < OR_MAXSP; ++sp)
        for (int a = 0; a < OR_MAXS; ++a)
            kind[sp * OR_MAXS + a] = (sp < s->n_species && a < s->n_sites[sp] && s->lj[sp][a]) ? t++ : -1;
    return t;
}
static int pair_row(int t1, int t2, int T) {
    if (t1 > t2) { int x = t1; t1 = t2; t2 = x; }
    return t1 * T - t1 * (t1 - 1) / 2 + (t2 - t1);
}
void or_rdf_counts(const or_system *s, const double *R, const double *q, double r_max, int nbins,
                   long long *counts) {
    int kind[OR_MAXSP * OR_MAXS], T = or_rdf_kinds(s, kind), NP = T * (T + 1) / 2, N = s->N;
    double *pos = (double *)malloc(sizeof(double) * 3 * OR_MAXS * N), dr = r_max / nbins;
    or_site_positions(s, R, q, pos);
    memset(counts, 0, sizeof(long long) * NP * nbins);
#pragma omp parallel
    {
        long long *loc = (long long *)calloc((size_t)NP * nbins, sizeof(long long));
#pragma omp for schedule(dynamic, 8)
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j) {
                int si = s->species[i], sj = s->species[j];
                for (int a = 0; a < s->n_sites[si]; ++a) {
                    if (kind[si * OR_MAXS + a] < 0) continue;
                    for (int b = 0; b < s->n_sites[sj]; ++b) {
                        if (kind[sj * OR_MAXS + b] < 0) continue;
                        double d[3];
                        min_image(s, pos + (i * OR_MAXS + a) * 3, pos + (j * OR_MAXS + b) * 3, d);
                        double r = sqrt(dot3(d, d));
                        if (!(r < r_max)) continue;
                        int bin = (int)floor(r / dr);
                        if (bin >= nbins) continue;
                        loc[(size_t)pair_row(kind[si * OR_MAXS + a], kind[sj * OR_MAXS + b], T) * nbins + bin]++;
                    }
                }
            }
#pragma omp critical
        for (size_t k = 0; k < (size_t)NP * nbins; ++k) counts[k] += loc[k];
        free(loc);
    }
    free(pos);
}

/* Number of LJ-site pairs (as counted above) whose distance lies within delta of
 * each bin edge k*dr, k = 0..nbins (edge k = nbins is r_max), summed over kind
 * pairs.  A pair this close to an edge may fall on either side in a computation
 * with coarser rounding, so a comparison of histograms allows it to move. */
void or_rdf_edge_pairs(const or_system *s, const double *R, const double *q, double r_max, int nbins, double delta,
                       long long *near) {
    int kind[OR_MAXSP * OR_MAXS], N = s->N;
    or_rdf_kinds(s, kind);
    double *pos = (double *)malloc(sizeof(double) * 3 * OR_MAXS * N), dr = r_max / nbins;
    or_site_positions(s, R, q, pos);
    memset(near, 0, sizeof(long long) * (nbins + 1));
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            int si = s->species[i], sj = s->species[j];
            for (int a = 0; a < s->n_sites[si]; ++a) {
                if (kind[si * OR_MAXS + a] < 0) continue;
                for (int b = 0; b < s->n_sites[sj]; ++b) {
                    if (kind[sj * OR_MAXS + b] < 0) continue;
                    double d[3];
                    min_image(s, pos + (i * OR_MAXS + a) * 3, pos + (j * OR_MAXS + b) * 3, d);
                    double r = sqrt(dot3(d, d));
                    int k = (int)floor(r / dr + 0.5);
                    if (k >= 0 && k <= nbins && fabs(r - k * dr) < delta) near[k]++;
                }
            }
        }
    free(pos);
}
