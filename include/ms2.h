/*
 * ms2.h — C ABI of the GB300 molecular-dynamics hot path of the ms2 method
 * (Glass et al., "ms2: A molecular simulation tool for thermodynamic properties,
 * release 2.0", arXiv 1507.07548).
 *
 * One library call advances, inspects or serves systems of rigid multi-site
 * molecules (Lennard-Jones 12-6 sites, point charges, point dipoles) in a cubic
 * periodic box with a molecule-centre cut-off near half the box edge (paper,
 * Sec. "Hybrid MPI & OpenMP Parallelization": ~10^3 molecules, cut-off radius in
 * the range of half the box edge).  Electrostatics use the reaction field (Sec.
 * "Massieu potential derivatives", LRC paragraph) or Ewald summation (Sec.
 * "Algorithmic Developments", paragraph "Ewald summation").
 *
 * Conventions that hold for every call:
 *   - Every call returns an ms2_status; nothing is thrown across the ABI.  On
 *     failure ms2_last_error() returns a thread-local message.
 *   - Units are fixed: length Angstrom, time fs, mass g/mol, charge e, dipole
 *     e*Angstrom, energy and temperature K (k_B = 1), pressure K/Angstrom^3
 *     (1 K/A^3 = 13.80649 MPa).  With ms2_options.reduced = 1 all quantities are
 *     in Lennard-Jones reduced units instead (sigma = epsilon = m = k_B = 1).
 *   - Arrays are row-major FP64 on the HOST unless the name ends in _dev, in
 *     which case they are device pointers written asynchronously on the
 *     system's stream.  Inputs are copied at call time; the library keeps no
 *     pointer to caller memory after a call returns.
 *   - The library owns all device memory of a system or server.  It allocates it
 *     with ms2_options.dev_alloc / dev_free if both are set (e.g. a PyTorch
 *     caching allocator), else with cudaMalloc / cudaFree, on the current device.
 *   - All work of a system is queued on its stream (ms2_options.stream, or a
 *     stream the library creates).  Calls that return numbers to the host
 *     synchronise that stream first; ms2_step does not.
 *   - A system is not thread-safe: one host thread drives it at a time.
 */
#ifndef MS2_H
#define MS2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MS2_API __attribute__((visibility("default")))
#else
#define MS2_API
#endif

typedef struct ms2_system_s *ms2_system;
typedef struct ms2_batch_s *ms2_batch;
typedef struct ms2_server_s *ms2_server;

typedef enum {
    MS2_OK = 0,
    MS2_EINVAL = 1,    /* bad argument, unsupported model combination */
    MS2_ENOMEM = 2,    /* device allocation failed */
    MS2_EBUDGET = 3,   /* job can never fit the server's memory budget */
    MS2_ECUDA = 4,     /* a CUDA call failed (message has the CUDA error) */
    MS2_EUNSTABLE = 5, /* non-finite or exploding forces/energies detected */
    MS2_ETIMEOUT = 6,  /* a bounded wait gave up */
    MS2_ESTATE = 7     /* call not valid in the object's current state */
} ms2_status;

typedef enum { MS2_ELEC_NONE = 0, MS2_ELEC_RF = 1, MS2_ELEC_EWALD = 2 } ms2_elec;

/* site kind bits; a site may combine them (e.g. LJ + charge on a water oxygen).
 * An LJ site with sigma = epsilon = 0 is a dummy site: it interacts with nothing
 * but is sampled by the RDF (paper, Sec. "Property Calculations", RDF paragraph). */
enum { MS2_SITE_LJ = 1, MS2_SITE_CHARGE = 2, MS2_SITE_DIPOLE = 4 };

enum { MS2_INT_VERLET = 0, MS2_INT_LEAPFROG_Q = 1 };

/* One site of a rigid molecule.  pos is in the BODY frame: origin at the
 * molecule's centre of mass, axes along its principal axes of inertia (checked:
 * |centre of mass| and the off-diagonal inertia must vanish to 1e-9 relative).
 * dipole is the body-frame point-dipole vector (kind bit MS2_SITE_DIPOLE). */
typedef struct {
    int kind;
    double pos[3];
    double mass;
    double sigma, epsilon; /* LJ 12-6; unlike pairs mix by Lorentz-Berthelot */
    double charge;
    double dipole[3];
} ms2_site;

/* A potential model (paper: "potential model file"); at most 8 sites. */
typedef struct {
    int n_sites;
    const ms2_site *sites;
} ms2_model;

typedef struct {
    double eps_rf;            /* reaction-field dielectric constant; <= 0 or >= 1e30: conducting */
    int lrc;                  /* 1: analytic LJ long-range correction in U and P */
    double dt;                /* time step (fs, or reduced) */
    int thermostat;           /* 1: isokinetic velocity scaling to T every step (NVT) */
    unsigned long long seed;  /* initial lattice orientations and velocities */
    int integrator;           /* MS2_INT_VERLET (point molecules only) or MS2_INT_LEAPFROG_Q */
    int reduced;              /* 1: LJ reduced units */
    int quat_iters;           /* sweeps of the implicit quaternion midpoint rule; 0 -> 3 */
    int graph_chunk;          /* steps per captured CUDA graph; 0 -> 50 */
    int fp64;                 /* 1: site-pair arithmetic in FP64 too (point LJ models only) */
    int massieu;              /* 1: also sample the Massieu-derivative moments (ms2_massieu); LJ and
                                 point-charge models, reaction field or no electrostatics; not in batches */
    int fused_step;           /* 1 (default): a chunk of steps runs as one cooperative kernel where the
                                 system allows it (leapfrog, no Ewald, the whole system fits one SM's
                                 shared memory); results are bitwise those of the per-phase kernels.
                                 0: one kernel per phase, replayed as a CUDA graph */
    void *stream;             /* cudaStream_t to use, or NULL */
    void *(*dev_alloc)(size_t bytes, void *ctx);
    void (*dev_free)(void *ptr, void *ctx);
    void *alloc_ctx;
} ms2_options;

/* Fills *o with defaults: conducting RF, lrc = 1, dt = 2 fs, thermostat = 1,
 * seed = 1, leapfrog, real units, 3 quaternion sweeps, graph chunks of 50 steps,
 * FP32 site-pair arithmetic with FP64 state and sums. */
MS2_API ms2_status ms2_default_options(ms2_options *o);

/* Creates a system of sum(N_per_model) molecules: N_per_model[m] molecules of
 * models[m] (n_models <= 4), numbered model by model.  The box edge is `box`
 * if box > 0, else (N / rho)^(1/3) with rho the molecule number density; if
 * both are > 0 they must agree to 1e-12 relative.  Molecules start on a simple
 * cubic lattice (FCC for a single point-mass model when N = 4 m^3) with seeded
 * random orientations and Maxwell-Boltzmann velocities at temperature T.
 * Requires 0 < cutoff < box / 2 (molecule-centre minimum image, paper Sec.
 * "Hybrid MPI & OpenMP Parallelization").  Reaction field requires electrically
 * neutral molecules; net-charged molecules need MS2_ELEC_EWALD (the paper's
 * reason for adding Ewald summation).  Charges and dipoles may not both occur in
 * one system, and dipoles need MS2_ELEC_RF.  Ewald starts with alpha = 3.2/cutoff
 * and kmax = 8 per axis (change with ms2_ewald_params).
 * Errors: MS2_EINVAL (arguments), MS2_ENOMEM, MS2_ECUDA. */
MS2_API ms2_status ms2_create_system(const ms2_model *models, const int *N_per_model, int n_models, double box, double T,
                             double rho, double cutoff, ms2_elec elec, const ms2_options *opt, ms2_system *out);
MS2_API ms2_status ms2_destroy_system(ms2_system sys);

/* Basic facts: molecule count, box edge, cut-off, degrees of freedom. */
MS2_API ms2_status ms2_system_info(ms2_system sys, int *N, double *box, double *cutoff, int *ndof);

/* Advances n >= 0 time steps (asynchronous).  Each step: interaction partner
 * search, site-pair energies/forces/torques (+ Ewald reciprocal space), then the
 * integrator (velocity Verlet, or leapfrog with the quaternion implicit
 * midpoint rule), with isokinetic scaling when the thermostat is on.  Paper,
 * Sec. "Hybrid MPI & OpenMP Parallelization": the partner search, the energy
 * and the force calculation are the loops over molecules that make up an MD
 * step; the paper names no integrator or thermostat (the leapfrog, quaternion
 * rule and isokinetic scaling are this library's stated readings).
 * Errors: MS2_EINVAL (n < 0); failures of the work show at the next read. */
MS2_API ms2_status ms2_step(ms2_system sys, long long n);

/* Potential energy U (incl. LRC and Ewald constants), molecular virial W
 * (sum over pairs of (R_i - R_j).F_ij, + reciprocal part; excl. LRC), kinetic
 * temperature of the stored velocities and pressure P = (2 KE_tr/3 + W/3)/V + P_LRC,
 * for the current configuration.  Any pointer may be NULL.  Paper, Sec.
 * "Massieu potential derivatives": U and its volume derivative (W = -3V dU/dV
 * at fixed scaled centres and orientations) are the NVT ensemble's sampled
 * quantities; the LRC follows the same section's LRC paragraph.  Synchronises
 * the system stream.  Errors: MS2_EUNSTABLE (non-finite or exploding forces),
 * MS2_ETIMEOUT (a bounded wait of the last fused launch ran out; the state is
 * then unspecified until ms2_set_state), MS2_ECUDA. */
MS2_API ms2_status ms2_energy_virial(ms2_system sys, double *U, double *W, double *T_inst, double *P);

/* The 16-number breakdown of the current configuration, in this order:
 * U_lj, U_qq (RF or Ewald real space), U_dd, U_rec, U_self, U_intra, U_bg,
 * U_lrc, U_total, W_pair, W_rec, W_bg, W_total, P_lrc, n_pairs (unique
 * molecule pairs within the cut-off), KE_total. */
MS2_API ms2_status ms2_energy_terms(ms2_system sys, double terms[16]);

/* Molecule forces F (N x 3) and space-frame torques tau (N x 3) of the current
 * configuration, in K/Angstrom and K (paper, Sec. "Hybrid MPI & OpenMP
 * Parallelization": every pair force acts on both molecules, and the same holds
 * for torques; here each molecule's owner sums its own, so no write is shared).
 * Caller-owned host arrays; synchronises the system stream.  Errors as
 * ms2_energy_virial. */
MS2_API ms2_status ms2_forces_torques(ms2_system sys, double *F, double *tau);
/* Same, into device buffers of 3N doubles each, queued on the system stream. */
MS2_API ms2_status ms2_forces_torques_dev(ms2_system sys, double *F_dev, double *tau_dev);

/* Ewald splitting parameter and k box |n_x| <= kx, |n_y| <= ky, |n_z| <= kz
 * (k = 2 pi n / box); paper, Sec. "Algorithmic Developments", paragraph "Ewald
 * summation" (real-space erfc sum within the cut-off plus the reciprocal sum
 * over these k vectors, tin-foil boundary).  MS2_EINVAL unless the system uses MS2_ELEC_EWALD or if
 * alpha <= 0 or a kmax is outside 1..64.  Recomputes forces. */
MS2_API ms2_status ms2_ewald_params(ms2_system sys, double alpha, int kx, int ky, int kz);

/* State for checkpoint/restart (no counterpart in the paper; the quantities
 * its MD integrates): centres R (N x 3), unit quaternions q (N x 4,
 * (w, x, y, z), body -> space), centre velocities v (N x 3) and space-frame
 * angular momenta Lang (N x 3, g/mol*A^2/fs) — for the leapfrog these are the
 * values half a step behind R and q — and the step counter.  Any pointer may be
 * NULL.  set_state renormalises a q whose squared norm differs from 1 by more
 * than 1e-13 and takes the others bit for bit.  It validates and stages the
 * state on the host, queues the copy and returns without waiting for it; the
 * forces, energies and site build of the new state are evaluated by the next
 * call that reads them (energies, forces, terms, partner counts, offsets, an RDF
 * sample, a batch step) or by the next ms2_step, whose fused kernel evaluates
 * the state first.  Results are the same either way, bit for bit. */
MS2_API ms2_status ms2_get_state(ms2_system sys, double *R, double *q, double *v, double *Lang, long long *step);
MS2_API ms2_status ms2_set_state(ms2_system sys, const double *R, const double *q, const double *v, const double *Lang);

/* Diagnostics of the last force evaluation: partner count of each molecule
 * (int, N), and site offsets A(q_i) b_a (N x n_site_slots x 3, FP64 copies of
 * the FP32 values the pair kernels use; unused slots are 0). */
MS2_API ms2_status ms2_partner_counts(ms2_system sys, int *counts);
/* Per-molecule shares of the last force evaluation (N x 4): half of each
 * molecule's summed pair energies (LJ, charge-charge, dipole-dipole) and of its
 * pair virial, so that the column sums are U_lj, U_qq, U_dd and W_pair. */
MS2_API ms2_status ms2_molecule_energies(ms2_system sys, double *out);
MS2_API ms2_status ms2_site_offsets(ms2_system sys, double *offsets, int *n_site_slots);

/* Radial distribution function between LJ sites (paper Eq. 2).  rdf_setup
 * clears the histogram and samples every `every` steps (0: only on
 * ms2_rdf_sample) into n_bins bins of width r_max / n_bins; r_max <= min(cutoff,
 * box/2).  Kinds are the LJ sites (model, site) in model-then-site order; kind
 * pairs t1 <= t2 are rows in upper-triangle row-major order.  ms2_rdf returns
 * the raw counts (rows x n_bins, may be NULL), g(r) normalised by the ideal-gas
 * pair count of each shell (may be NULL), the number of samples and the rows. */
MS2_API ms2_status ms2_rdf_setup(ms2_system sys, double r_max, int n_bins, int every);
MS2_API ms2_status ms2_rdf_sample(ms2_system sys);
MS2_API ms2_status ms2_rdf(ms2_system sys, long long *counts, double *g, int *n_samples, int *n_rows);

/* Running averages since the last reset over the steps taken: <U>, <P>, <T>,
 * and the block-averaged standard errors of <U> and <P> (blocks of 100 steps). */
MS2_API ms2_status ms2_averages(ms2_system sys, double out[5], long long *n_steps);
MS2_API ms2_status ms2_reset_averages(ms2_system sys);

/* ----------------------------------------------------------------- batch */
/* Paper, Sec. "Introduction": the tool serves high-throughput work, many
 * independent simulations of ~10^3 molecules (e.g. the state points of a
 * phase diagram); each system here is one such simulation, and batching them
 * onto one GPU has no counterpart in the paper.  Arguments: systems[0..n) are
 * the caller's systems (n >= 1, each in at most one batch; the batch keeps the
 * handles, not copies); *out receives the batch.  ms2_batch_step advances
 * every system by n >= 0 steps (asynchronous); read results per system.
 * Errors: MS2_EINVAL (a system the batch kernels do not take, see below),
 * MS2_ENOMEM, MS2_ECUDA.
 * A batch advances many independent systems together: per chunk of steps, one
 * cooperative persistent kernel per model kind (slot pattern) runs every phase
 * of a step (drift and site build, partner search and site-pair forces, RDF
 * samples, reduction, thermostat, record) over all of the kind's systems at
 * once, spread over the whole GPU at molecule granularity, with a bounded grid
 * barrier between phases.  A system's results depend only on the system (bit
 * for bit the same alone or in any batch).  The systems must be leapfrog
 * systems with the reaction field or no electrostatics, or 3-site water (with
 * or without single-site ions) under Ewald summation, whose whole configuration
 * fits one block's shared memory (about 3700 three-site molecules).  For the
 * Ewald kind, the reciprocal-space tasks of the single-system path (structure
 * factor, sums, forces; paper Sec. "Algorithmic Developments", paragraph "Ewald
 * summation") run over all its systems between grid barriers after the pair
 * phase.  The block shape comes from the autotuner cache.  Where it pays
 * (a list shorter than 3N/4), a system also gets device memory for candidate
 * lists: 2 bytes x N x (2.5 x the molecules within 1.2 r_c + 64, at most N), rebuilt at
 * the start of every chunk of steps and whenever a molecule has moved 0.1 r_c;
 * the partners found are those of the full search.  A barrier wait
 * that runs out (2 s) marks every system of the kind so that its next
 * ms2_energy_virial returns MS2_ETIMEOUT.  The systems stay
 * usable on their own: the batch runs on a stream of its own, waits for work
 * already queued on the systems' streams and makes their later work wait for
 * it.  Destroy a batch before any of its systems. */
MS2_API ms2_status ms2_batch_create(const ms2_system *systems, int n, ms2_batch *out);
MS2_API ms2_status ms2_batch_step(ms2_batch b, long long n);
MS2_API ms2_status ms2_batch_destroy(ms2_batch b);

/* ----------------------------------------------------------------- serve */
/* A simulation job: model mix entry, size and state point, steps, outputs.
 * The server builds the system itself (ms2_create_system defaults with this
 * seed).  arrival_time (s, on the server's clock, which starts at
 * ms2_serve_open) is when the job becomes eligible.  R0 (N x 3) and q0 (N x 4),
 * if not NULL, replace the lattice start's centres and orientations (a restart
 * from a checkpoint); they are copied at submit and checked at admission as by
 * ms2_set_state (a failure retires the job with that status). */
typedef struct {
    const ms2_model *models;
    const int *N_per_model;
    int n_models;
    double T, rho, cutoff;
    ms2_elec elec;
    long long steps;
    double arrival_time;
    unsigned long long seed;
    int rdf_bins;         /* 0: no RDF output */
    int rdf_every;
    const double *R0;     /* optional start: centres, N x 3 */
    const double *q0;     /* optional start: unit quaternions, N x 4 */
} ms2_job;

typedef struct {
    long long job_id;
    ms2_status status;
    double U_avg, U_err, P_avg, P_err, T_avg;
    double t_arrive, t_admit, t_done; /* server clock, s */
    int n_rows, n_bins;
    double g[4096];                   /* g(r), n_rows x n_bins (first kind pair rows) */
} ms2_job_result;

/* Opens a server whose resident job state may use at most hbm_budget_bytes of
 * device memory; a scheduler thread admits eligible jobs in arrival order as
 * budget and slots free up, advances all resident jobs together chunk by chunk
 * (continuous batching), and retires finished ones.  max_slots <= 1024.  A job's
 * path depends on the job alone: a job the batch kernels take (see
 * ms2_batch_create) always steps in the server's batch, a batch of one when it
 * is the only such job, and any other job with its own single-system kernels.
 * So a job's results are bit for bit the same alone and in any mix of other
 * jobs.  All the server's systems share one stream.  The admission estimate of a
 * job's device memory includes the batch's candidate lists; a batch that cannot
 * be built retires its jobs with the error. */
/* (Serving has no counterpart in the paper; each job is one simulation as in
 * its Sec. "Introduction".)  opt: the defaults of the jobs' systems (NULL:
 * ms2_default_options); *out receives the server.  Errors: MS2_EINVAL, MS2_ECUDA. */
MS2_API ms2_status ms2_serve_open(size_t hbm_budget_bytes, int max_slots, const ms2_options *opt, ms2_server *out);
/* Queues a job (never blocks); the job's arrays are copied, *job_id receives its
 * id.  MS2_EBUDGET if it alone exceeds the budget; MS2_EINVAL for bad models or
 * sizes (failures found at admission are reported in the job's result). */
MS2_API ms2_status ms2_serve_submit(ms2_server s, const ms2_job *job, long long *job_id);
/* Copies up to max finished results out (oldest first) and removes them. */
MS2_API ms2_status ms2_serve_poll(ms2_server s, ms2_job_result *out, int max, int *n_done);
/* Blocks until all submitted jobs finished or timeout_s passed (MS2_ETIMEOUT). */
MS2_API ms2_status ms2_serve_drain(ms2_server s, double timeout_s);
MS2_API ms2_status ms2_serve_close(ms2_server s);

/* ------------------------------------------------- Massieu derivatives */
/* Paper Sec. 2, Eq. 1: A_mn = beta^m rho^n d^(m+n)(F/(N k T)) / d beta^m d rho^n
 * (beta = 1/T, rho = N/V) splits into an ideal and a residual part; the
 * residual parts of the NVT ensemble are canonical moments of the potential
 * energy U and of its volume derivatives U_V = dU/dV, U_VV = d2U/dV2 taken at
 * fixed scaled centres and orientations (the scaling of the molecular virial):
 *   A10 = beta <U>/N                  A01 = -beta V <U_V>/N
 *   A20 = -beta^2 var(U)/N            A11 = -(beta V/N) (<U_V> - beta cov(U,U_V))
 *   A02 = (beta/N) (2 V <U_V> + V^2 (<U_VV> - beta var(U_V)))
 *   A30 = beta^3 <dU^3>/N             A21 = (beta^2 V/N) (2 cov(U,U_V) - beta <dU^2 dU_V>)
 *   A12 = (beta/N) (2 V (<U_V> - beta cov(U,U_V))
 *         + V^2 (<U_VV> - 2 beta var(U_V) - beta cov(U,U_VV) + beta^2 <dU dU_V^2>))
 * (dX = X - <X>; N molecules; energies in K, k = 1; beta = 1/T0 of the
 * thermostat).  U_V = -W/(3V) - P_LRC and U_VV include the long-range parts
 * -P_LRC and 2 P_LRC/V.  The paper does not offer these with Ewald summation;
 * point dipoles are not covered either.  Needs ms2_options.massieu = 1 at
 * creation, otherwise MS2_ESTATE. */
/* U_V and U_VV of the current configuration. */
MS2_API ms2_status ms2_volume_derivatives(ms2_system sys, double *dUdV, double *d2UdV2);
/* A^r_mn, mn = 10, 01, 20, 11, 02, 30, 21, 12, from the samples of every step
 * since ms2_reset_averages (MS2_ESTATE without samples); *n_samples may be NULL. */
MS2_API ms2_status ms2_massieu(ms2_system sys, double A[8], long long *n_samples);

/* ----------------------------------------------------- residence time */
/* Paper Sec. 4, Eq. 7: tau_j = int <(1/n_ij(0)) sum_k Theta_k(t) Theta_k(0)> dt for
 * molecules of species j around molecules of species i, with the tolerance of
 * Impey et al.  Readings: "within r_ij" is the minimum-image centre distance
 * below r_shell, decided exactly on the integer centre lattice like the cut-off;
 * a member counts at lag t if it is in the shell at the origin and at t and was
 * never outside for more than t_star consecutive samples in between; the average
 * runs over all origins (one every `every` steps) and centres with a non-empty
 * shell.  The solvation number n_ij is the mean shell count.  Setup (re)allocates
 * and zeroes the state; MS2_EINVAL for bad species, r_shell outside (0, L/2),
 * every < 1, n_lags outside 2..4096 or t_star outside 0..254.  Sampling systems
 * step with the per-phase kernels and are not batched. */
MS2_API ms2_status ms2_residence_setup(ms2_system sys, int species_i, int species_j, double r_shell, int every,
                                       int n_lags, int t_star);
/* corr (n_lags values, may be NULL), tau = trapezoidal integral of corr (fs, or
 * reduced time), the solvation number and the sample count (each may be NULL). */
MS2_API ms2_status ms2_residence(ms2_system sys, double *corr, double *tau, double *solvation, long long *n_samples);

/* ------------------------------------------- Green-Kubo conductivity */
/* Paper Sec. 4, Eqs. 3-4: sigma = 1/(3 V kB T) int_0^inf <j_e(t).j_e(0)> dt with
 * the electric current flux j_e = sum_k q_k v_k over the net-charged molecules
 * (q_k = sum of the molecule's site charges; neutral molecules drop out), sampled
 * every `every` MD steps (the extended time step).  Reading: v_k is the stored
 * centre velocity after the step (the half-step velocity of the leapfrog, the one
 * the reported temperature uses).  The autocorrelation runs over all time origins
 * on the device: a ring of the last n_lags samples and one sum per lag in sample
 * order.  Setup (re)allocates and zeroes the sampling state; MS2_EINVAL for
 * every < 1 or n_lags outside 2..2^20.  Systems that sample are not batched. */
MS2_API ms2_status ms2_conductivity_setup(ms2_system sys, int every, int n_lags);
/* The flux j_e (e A/fs, or reduced) of the last sample. */
MS2_API ms2_status ms2_current(ms2_system sys, double j[3]);
/* sigma (S/m; reduced units for reduced systems) from the trapezoidal integral of
 * the autocorrelation over the n_lags lags, T = T0; acf (n_lags values of
 * <j(t).j(0)>, may be NULL) and *n_samples (may be NULL).  MS2_ESTATE without setup. */
MS2_API ms2_status ms2_conductivity(ms2_system sys, double *sigma, double *acf, long long *n_samples);

/* ------------------------------------ Green-Kubo thermal conductivity */
/* Paper Sec. 4, Eqs. 5-6: lambda = 1/(3 V kB T^2) int_0^inf <J_q(t).J_q(0)> dt with
 * the microscopic heat flux of a mixture of rigid molecules
 *   J_q = sum_k (E_k - h_k) v_k + 1/2 sum_k sum_{l != k} (R_k - R_l) (F_kl.v_k + tau_kl.w_k),
 *   E_k = M_k v_k^2 / 2 + w_k.I_k w_k / 2 + 1/2 sum_{l != k} u_kl,
 * F_kl and tau_kl the force and torque (about R_k) of l on k, h_k the partial
 * molar enthalpy of k's component (h[species], energy units per molecule: K, or
 * reduced; h may be NULL for zeros).  Reading: Gamma_kl of the paper is the
 * torque of l on k, entering as tau_kl.w_k (the sign that makes J_q the time
 * derivative of sum_k R_k E_k); v_k, w_k are taken at the integer time of the
 * forces, v = v(n - 1/2) + dt/2 F/M and L = L(n - 1/2) + dt/2 tau (the leapfrog
 * half-step mean without the thermostat factor; the velocity-Verlet state as is).
 * Sampled every `every` steps: on such a step a second pair pass forms
 * sum_l d_kl P_kl with the integer-time site velocities (no change to the
 * trajectory).  Pairwise interactions only: MS2_EINVAL for Ewald systems, the
 * FP64 pair path, 8-slot models, every < 1, n_lags outside 2..2^20 or a
 * non-finite h.  Setup (re)allocates and zeroes the sampling state.  Systems
 * that sample are not batched. */
MS2_API ms2_status ms2_heat_setup(ms2_system sys, int every, int n_lags, const double *h);
/* The heat flux J_q (K A/fs with energies in K, or reduced) of the last sample. */
MS2_API ms2_status ms2_heat_flux(ms2_system sys, double J[3]);
/* lambda (W/(m K); reduced units for reduced systems) from the trapezoidal
 * integral of the autocorrelation over the n_lags lags, T = T0; acf (n_lags
 * values of <J_q(t).J_q(0)>, may be NULL) and *n_samples (may be NULL).
 * MS2_ESTATE without setup. */
MS2_API ms2_status ms2_thermal_conductivity(ms2_system sys, double *lambda, double *acf, long long *n_samples);

/* Kernel timing: with on = 1, every subsequently enqueued batch of steps
 * records CUDA events (on the system stream) around its last step and around
 * that step's pair kernel and Ewald kernels.  ms2_last_step_times synchronises
 * and returns, in ms: [0] pair kernel, [1] Ewald reciprocal kernels, [2] the whole
 * last step, [3] that step minus [0] and [1].  When the last chunk ran as one
 * fused kernel (ms2_options.fused_step), [2] is the chunk's time per step,
 * [0] the pair phase of its last step and [1] its reciprocal-space task phases
 * (device timer; 0 without Ewald). */
MS2_API ms2_status ms2_enable_timing(ms2_system sys, int on);
/* *fused = 1 if the next chunk of steps runs as the fused cooperative kernel
 * (ms2_options.fused_step and a system it takes; an RDF histogram too large for
 * shared memory sends the chunk to the per-phase kernels), else 0. */
MS2_API ms2_status ms2_step_kernel(ms2_system sys, int *fused);
/* Diagnostic of the fused step with timing on: device-timer durations (ms) of
 * the last step of the last chunk: [0] drift and site build, with the thermostat
 * factor the drifting warps form first from the previous step's totals, [2]
 * staging, pair and RDF, [3] unit reduction (each until the slowest block is
 * done), [1] and [4] the grid barriers after [0] and [3], [5] the rest of the
 * step on block 0's first warp (the totals of its record run on other warps,
 * beside the next drift),
 * [6] kernel entry to that last step, [7] the whole last step, [8] its end to
 * the kernel's exit (write-back of the block-held state); Ewald systems (whose
 * reciprocal-space tasks run between [2] and the reduction, inside [3]):
 * [9] structure-factor tasks, [10] sum tasks, [11] force tasks, each until the
 * grid barrier after it ends (block 0's clock), else 0.  MS2_ESTATE if timing
 * is off or the last chunk ran as per-phase kernels. */
MS2_API ms2_status ms2_last_step_phases(ms2_system sys, double out[12]);
MS2_API ms2_status ms2_last_step_times(ms2_system sys, double out[4]);

/* Fault-path hook (tests of failure detection; no counterpart in the paper).
 * what = MS2_FAULT_BARRIER: the next fused launch of sys (ms2_step) limits each
 * grid-barrier wait to wait_s seconds (1e-6 <= wait_s <= 2) and makes its first
 * barrier wait for one arrival more than the grid has.  That wait runs out, the
 * kernel raises its sticky timeout flag, every other wait ends at once and the
 * launch returns; the next ms2_energy_virial reports MS2_ETIMEOUT, clears the
 * flag, and the state is unspecified until ms2_set_state.  No wait is
 * unbounded and no memory access leaves its buffer.  MS2_EINVAL for another
 * `what` or wait_s out of range; MS2_ESTATE if the system has no fused kernel
 * (ms2_step_kernel). */
enum { MS2_FAULT_BARRIER = 1 };
MS2_API ms2_status ms2_fault_inject(ms2_system sys, int what, double wait_s);

/* ------------------------------------------------------- allocation-free */
/* Forces, torques, potential energy and molecular virial of ONE configuration
 * without allocating any device memory.  For callers that cannot call
 * cudaMalloc: code running inside a pre-reserved memory pool or under a strict
 * memory cap, plugins that are handed a stream and buffers by a host
 * application owning all allocations, and sections that must not risk the
 * implicit device synchronisation an allocation can cause.  (This convenience
 * has no counterpart in the paper.)
 * Inputs (device, row-major FP64): centres R_dev (N x 3), unit quaternions
 * q_dev (N x 4); models/N_per_model/box/cutoff/elec/opt as for
 * ms2_create_system (box > 0 required; MS2_ELEC_NONE or MS2_ELEC_RF only;
 * opt->fp64 must be 0: the site-pair arithmetic is FP32 here).
 * Outputs (device, FP64): F_dev (N x 3), tau_dev (N x 3), UW_dev[2] = {U, W}
 * (pair energy + LJ long-range correction; molecular pair virial).  All work is
 * queued on `stream` (a cudaStream_t, NULL = default stream); nothing is
 * synchronised.
 * Working memory is one library-owned __device__ array of
 * ms2_noalloc_scratch_bytes() bytes (about 2.9 MB) that every GPU loading the
 * library holds until the process exits.  Limits: N <= 4096 molecules, at most
 * 4 site slots per molecule; larger inputs return MS2_EINVAL.  The first call on
 * a device looks up the array's device address; make that first call before
 * any stream capture.  Every call shares the array: calls that overlap on the
 * GPU race, so serialise them (one stream, or events). */
MS2_API ms2_status ms2_forces_noalloc(const ms2_model *models, const int *N_per_model, int n_models, double box,
                                      double cutoff, ms2_elec elec, const ms2_options *opt, const double *R_dev,
                                      const double *q_dev, double *F_dev, double *tau_dev, double *UW_dev,
                                      void *stream);
MS2_API size_t ms2_noalloc_scratch_bytes(void);

/* ------------------------------------------------------------------ misc */
MS2_API const char *ms2_last_error(void);
/* Number of kernels this library has launched in the process (graph nodes
 * counted per replay). */
MS2_API long long ms2_kernel_launches(void);
MS2_API const char *ms2_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MS2_H */
