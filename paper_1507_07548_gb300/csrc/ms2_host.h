// Host-side structures shared by the C-ABI, batch and serving translation units.
#pragma once
#include <map>
#include <tuple>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ms2.h"
#include "ms2_internal.cuh"

// Device memory owner: user hooks (e.g. a PyTorch caching allocator) or cudaMalloc.
struct DevAlloc {
    void *(*fa)(size_t, void *) = nullptr;
    void (*ff)(void *, void *) = nullptr;
    void *ctx = nullptr;
    std::vector<void *> live;
    size_t bytes = 0;
    cudaError_t alloc(void **p, size_t n);
    void release_all();
};

struct GraphEntry {
    cudaGraphExec_t exec;
    long long nodes;
};

struct ms2_system_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevAlloc al;
    SysParams hp;
    SysParams *dP = nullptr;
    DevSys d;
    int N = 0, ns = 1;
    std::vector<int> species;
    double rc = 0;
    bool lrc = true, reduced = false, fp64 = false;
    unsigned ljm = 0, qm = 0, dm = 0;
    int tile = 0;  // tile layout of the pair kernel: dipole slots kept + 256 x (molecular dipoles kept)
    bool multi_used = false;
    void *pair_fn = nullptr;
    int wpb = 8, jsplit = 1, TJ = 32;
    size_t pair_smem = 0;
    int tune_wpb = 0, tune_jsplit = 0;
    // fused step (k_step.cu): null when the per-phase kernels run every step
    void *step_fn = nullptr;
    void *fuse_fn = nullptr;  // the variant when the system is fusable (decides the decomposition)
    void *step_heat_fn = nullptr;  // the fused variant with the heat-flux pass (heat sampling on), or null
    int step_grid = 0, Np = 0, bar_parity = 0, mcap = 0, nunits = 1;
    size_t step_smem_max = 0;
    int last_launch_steps = 0;
    bool last_fused = false;
    // Ewald
    double alpha = 0;
    float2 *AS = nullptr;
    int ny_per_chunk = 1;
    // energy constants
    double uconst = 0, wbg = 0, ulrc = 0, plrc = 0;
    long long step = 0;
    int graph_chunk = 50;
    std::map<std::tuple<int, int, int, int, int>, GraphEntry> graphs;  // (steps, RDF, conductivity, residence, heat phase)
    long long launch_acc = 0;
    // RDF
    int rdf_every = 0, rdf_samples = 0, rdf_cap = 0;
    int gk_every = 0;  // conductivity: extended time step (0: off)
    int res_every = 0;  // residence time: extended time step (0: off)
    int hf_every = 0;   // thermal conductivity: extended time step (0: off)
    void *heat_fn = nullptr;  // heat-flux power pass matching pair_fn
    ResArgs res{};
    double rdf_rmax = 0;
    // host staging of the state
    std::vector<double> hR, hq, hv, hL;
    // page-locked staging: two upload buffers of 13N doubles (used alternately,
    // each guarded by the event of its last copy) and one download buffer of 13N
    double *pinned = nullptr;
    double *hscal = nullptr;   // page-locked copy target of the system scalars
    cudaEvent_t up_ev[2] = {nullptr, nullptr};
    int up_k = 0;
    // set_state leaves forces, energies and site build stale; the next query
    // evaluates them, or the next fused step does it in its prologue
    bool stale = false;
    // fault-path test: the next fused launch's first grid barrier waits for one
    // arrival more than the grid has, each wait limited to fault_wait_ns
    int fault_barrier = 0;
    int sms = 1;  // multiprocessors of the device (queried at creation)
    unsigned long long fault_wait_ns = 0;
    // timing events: [0] step start, [1] before pair, [2] after pair, [3] after Ewald, [4] step end
    bool timing = false;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    size_t mum_bytes() const { return d.mum ? 3 * sizeof(float) * (size_t)N : 0; }
    size_t mu_bytes() const { return d.mu ? 3 * sizeof(float) * (size_t)ns * N : 0; }
};

// Candidate lists of the batch kernels: capacity per molecule = MS2_LIST_CAP x
// the ideal-gas count within r_c + skin, + 64, at most the system (batch.cu; the
// server's admission estimate uses the same bound)
constexpr double MS2_LIST_CAP = 2.5;

ms2_status ms2_fail(ms2_status st, const char *fmt, ...);
ms2_status ms2_fail_cuda(cudaError_t e, const char *what, const char *file, int line);
// raises (never lowers) a kernel's dynamic shared-memory limit on the current device
cudaError_t ms2_allow_smem(const void *fn, size_t bytes);
void ms2_unit_constants(bool reduced, double *coulomb, double *kconv);
ms2_status ms2_eval_forces(ms2_system s);
ms2_status ms2_ensure_forces(ms2_system s);  // evaluates after ms2_set_state, else nothing
ms2_status ms2_validate_models(const ms2_model *models, int n_models, ms2_elec elec);
// residence-time sampling (k_residence.cu)
void ms2_launch_residence(cudaStream_t st, const SysParams *P, const DevSys &S, const ResArgs &a);
size_t ms2_residence_state_doubles(int M);
// fused step kernel (k_step.cu)
size_t ms2_step_smem_bytes(int NS, int tile, bool multi, int Np, int mcap, int js, int rdf_cells, size_t ews);
size_t ms2_step_ewald_scratch(int kx, int ky, int kz, int ny_per_chunk, int skc);
int ms2_step_threads();
void *ms2_pick_step_kernel(int ns, unsigned ljm, unsigned qm, unsigned dm, int elec, bool multi, bool mass, bool heat);
cudaError_t ms2_launch_step(void *fn, int grid, size_t smem, cudaStream_t st, const SysParams *P, const DevSys &S,
                            const StepArgs &A);
