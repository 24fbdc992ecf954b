// Serving: a request loop for simulation jobs with state resident on the GPU.
//
// A scheduler thread owns all device work.  Between chunks of steps it
//   1. retires finished jobs (averages and RDF copied out, memory released),
//   2. admits eligible jobs (arrival time reached) in arrival order while the
//      memory budget and the slot table allow (head-of-line: a job that does
//      not fit yet blocks the ones behind it, so admission is FIFO-fair),
//   3. advances every resident job by one chunk.
// Jobs that arrive while others run are admitted at the next chunk boundary
// (continuous batching).  A job's path is a function of the job alone: a job the
// batch kernels take always steps in the batch (a batch of one when it is the
// only such job), any other job with its own single-system kernels (the fused
// step where the system allows, each chunk on the whole GPU).  A batched
// system's results depend only on the system, so every job gives the same bits
// alone and in any mix.  (A path chosen by the load would not: the batch and
// the single-system kernels split the pair sums differently and agree only
// within the parity tolerances, and trajectories amplify that difference.)
// All systems of a server share one stream, so cooperative launches never
// overlap each other or the batch.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "ms2_host.h"

bool ms2_batch_accepts(ms2_system s);  // batch.cu
ms2_status ms2_batch_create_opt(const ms2_system *systems, int n, ms2_batch *out, bool tune_shapes,
                                void *(*fa)(size_t, void *), void (*ff)(void *, void *), void *ctx);
ms2_status ms2_scalars_enqueue(ms2_system s);  // capi.cu: the system scalars to the host, queued
ms2_status ms2_scalars_status(ms2_system s);   // capi.cu: their status, after a synchronisation

namespace {

struct JobSpec {
    long long id = 0;
    std::vector<std::vector<ms2_site>> sites;
    std::vector<int> counts;
    double T = 0, rho = 0, cutoff = 0, arrival = 0;
    ms2_elec elec = MS2_ELEC_NONE;
    long long steps = 0;
    unsigned long long seed = 1;
    int rdf_bins = 0, rdf_every = 0;
    std::vector<double> R0, q0;  // optional start (empty: the lattice start)
    size_t bytes = 0;
};

struct Slot {
    JobSpec job;
    ms2_system sys = nullptr;
    long long remaining = 0;
    double t_admit = 0;
    bool batched = false;
};

// device bytes a system will hold (mirrors the allocations of ms2_create_system)
size_t estimate_bytes(const JobSpec &j) {
    long long N = 0;
    int ns = 1;
    for (size_t m = 0; m < j.counts.size(); ++m) {
        N += j.counts[m];
        ns = std::max(ns, (int)j.sites[m].size());
    }
    const int nsp = ns <= 1 ? 1 : (ns <= 4 ? 4 : 8);  // padded slots (upper bound)
    size_t b = (size_t)N * (23 * 8 + 4 + 12 + 2 * 12 * nsp + 12 + 8 * 12 * 4 + 4 + 8);
    // in a batch: reduction-unit partials and candidate lists (16-bit slots,
    // MS2_LIST_CAP x the ideal-gas count within 1.2 r_c + 64 per molecule, at most
    // the system; an upper bound of the batch's allocation, which takes lists
    // only where they are short)
    const double V = N / std::max(j.rho, 1e-300), rl = 1.2 * j.cutoff;
    const double frac = std::min(1.0, 4.18879020478639098 * rl * rl * rl / V);
    const double lcap = std::min(MS2_LIST_CAP * frac * N + 64.0, (double)N + 32.0);
    b += (size_t)N * (8 * 32 + 16) + (size_t)N * 2 * (size_t)lcap;
    if (j.elec == MS2_ELEC_EWALD) {
        const size_t M = (size_t)N * nsp;
        b += M * (12 + 4 + 3 * 9 * 8 + 17 * 3 * 4) + 17 * 17 * 9 * 8 * 2;
    }
    return b + (1 << 20);
}

// Device blocks the server's batches reuse: a batch is rebuilt whenever a job is
// admitted or retires, and cudaMalloc/cudaFree (which synchronises the device)
// on every rebuild would stall the loop.  Sizes are rounded up to 1/8 steps of a
// power of two so that blocks fit the next batch's similar requests.
struct DevCache {
    std::multimap<size_t, void *> free_;
    std::map<void *, size_t> size_;
    static size_t round(size_t n) {
        size_t p = 256;
        while (p < n) p <<= 1;
        const size_t step = std::max<size_t>(p >> 3, 256);
        return (n + step - 1) / step * step;
    }
    static void *alloc(size_t n, void *ctx) {
        DevCache *c = (DevCache *)ctx;
        n = round(n);
        auto it = c->free_.lower_bound(n);
        if (it != c->free_.end() && it->first <= n + (n >> 2)) {
            void *p = it->second;
            c->free_.erase(it);
            return p;
        }
        void *p = nullptr;
        if (cudaMalloc(&p, n) != cudaSuccess) {
            c->trim();  // give the cached blocks back and try once more
            if (cudaMalloc(&p, n) != cudaSuccess) return nullptr;
        }
        c->size_[p] = n;
        return p;
    }
    static void release(void *p, void *ctx) {
        DevCache *c = (DevCache *)ctx;
        auto it = c->size_.find(p);
        if (it != c->size_.end()) c->free_.emplace(it->second, p);
    }
    void trim() {
        for (auto &kv : free_) {
            cudaFree(kv.second);
            size_.erase(kv.second);
        }
        free_.clear();
    }
    ~DevCache() {
        for (auto &kv : size_) cudaFree(kv.first);
    }
};

}  // namespace

struct ms2_server_s {
    size_t budget = 0;
    int max_slots = 0;
    ms2_options opt;
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<JobSpec> queue;
    std::deque<ms2_job_result> done;
    std::vector<Slot> slots;
    size_t resident = 0;
    long long next_id = 1, outstanding = 0;
    bool stop = false;
    int chunk = 100;
    std::thread th;
    ms2_batch batch = nullptr;
    bool batch_dirty = true;
    DevCache cache;  // device blocks of the rebuilt batches
    cudaStream_t stream = nullptr;  // shared by all the server's systems

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

static void finish_slot(ms2_server S, Slot &sl, ms2_status st) {
    ms2_job_result r;
    memset(&r, 0, sizeof r);
    r.job_id = sl.job.id;
    r.status = st;
    r.t_arrive = sl.job.arrival;
    r.t_admit = sl.t_admit;
    if (sl.sys) {
        double av[5];
        long long n = 0;
        if (st == MS2_OK) st = ms2_averages(sl.sys, av, &n);
        if (st == MS2_OK) {
            r.U_avg = av[0];
            r.P_avg = av[1];
            r.T_avg = av[2];
            r.U_err = av[3];
            r.P_err = av[4];
        }
        if (st == MS2_OK && sl.job.rdf_bins > 0) {
            int ns = 0, rows = 0;
            std::vector<double> g;
            ms2_rdf(sl.sys, nullptr, nullptr, &ns, &rows);
            g.resize((size_t)rows * sl.job.rdf_bins);
            ms2_rdf(sl.sys, nullptr, g.data(), &ns, &rows);
            const int keep = std::min<int>(rows, 4096 / sl.job.rdf_bins);
            r.n_rows = keep;
            r.n_bins = sl.job.rdf_bins;
            for (int k = 0; k < keep * sl.job.rdf_bins; ++k) r.g[k] = g[k];
        }
        r.status = st;
        S->resident -= std::min(S->resident, sl.job.bytes);
        ms2_destroy_system(sl.sys);
        sl.sys = nullptr;
    }
    r.t_done = S->now();
    std::lock_guard<std::mutex> lk(S->mu);
    S->done.push_back(r);
    S->outstanding -= 1;
    S->cv.notify_all();
}

static void admit(ms2_server S) {
    for (;;) {
        JobSpec j;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->queue.empty()) return;
            const JobSpec &h = S->queue.front();
            if (h.arrival > S->now()) return;
            if ((int)S->slots.size() >= S->max_slots || S->resident + h.bytes > S->budget) return;
            j = h;
            S->queue.pop_front();
        }
        Slot sl;
        sl.job = j;
        sl.t_admit = S->now();
        std::vector<ms2_model> models(j.sites.size());
        for (size_t m = 0; m < j.sites.size(); ++m) {
            models[m].n_sites = (int)j.sites[m].size();
            models[m].sites = j.sites[m].data();
        }
        ms2_options o = S->opt;
        o.seed = j.seed;
        o.stream = (void *)S->stream;
        ms2_status st = ms2_create_system(models.data(), j.counts.data(), (int)models.size(), 0.0, j.T, j.rho,
                                          j.cutoff, j.elec, &o, &sl.sys);
        if (st == MS2_OK && (!j.R0.empty() || !j.q0.empty()))
            st = ms2_set_state(sl.sys, j.R0.empty() ? nullptr : j.R0.data(), j.q0.empty() ? nullptr : j.q0.data(),
                               nullptr, nullptr);
        if (st == MS2_OK && j.rdf_bins > 0) {
            int N = 0;
            double box = 0, rc = 0;
            ms2_system_info(sl.sys, &N, &box, &rc, nullptr);
            st = ms2_rdf_setup(sl.sys, std::min(rc, 0.5 * box), j.rdf_bins, j.rdf_every > 0 ? j.rdf_every : 10);
        }
        if (st == MS2_OK) st = ms2_reset_averages(sl.sys);
        if (st != MS2_OK) {
            S->resident += j.bytes;  // finish_slot releases it
            finish_slot(S, sl, st);
            continue;
        }
        S->resident += j.bytes;
        sl.remaining = j.steps;
        sl.batched = ms2_batch_accepts(sl.sys);  // the job's own property, never the load
        S->slots.push_back(sl);
        S->batch_dirty = true;
    }
}

static void advance(ms2_server S) {
    long long m = S->chunk;
    for (const Slot &sl : S->slots) m = std::min(m, sl.remaining);
    if (m <= 0) return;
    std::vector<ms2_system> bs;
    for (const Slot &sl : S->slots)
        if (sl.batched) bs.push_back(sl.sys);
    if (S->batch_dirty) {
        if (S->batch) ms2_batch_destroy(S->batch);
        S->batch = nullptr;
        ms2_status st = MS2_OK;
        if (!bs.empty())
            st = ms2_batch_create_opt(bs.data(), (int)bs.size(), &S->batch, false, &DevCache::alloc, &DevCache::release,
                                      &S->cache);
        S->batch_dirty = false;
        if (st != MS2_OK) {
            // no silent change of path (it would change the jobs' results):
            // the batched jobs retire with the failure
            S->batch = nullptr;
            for (Slot &sl : S->slots)
                if (sl.batched) sl.remaining = -1 - (long long)st;
            return;
        }
    }
    // unbatched jobs first (they run on their own streams), then the batch
    for (Slot &sl : S->slots)
        if (!sl.batched) ms2_step(sl.sys, m);
    if (S->batch) ms2_batch_step(S->batch, m);
    // every job's scalars to the host in one round (one synchronisation), then
    // the status of each: a failed job retires with it
    std::vector<ms2_status> qst(S->slots.size(), MS2_OK);
    for (size_t k = 0; k < S->slots.size(); ++k) qst[k] = ms2_scalars_enqueue(S->slots[k].sys);
    cudaStreamSynchronize(S->stream);
    for (size_t k = 0; k < S->slots.size(); ++k) {
        Slot &sl = S->slots[k];
        const ms2_status st = qst[k] != MS2_OK ? qst[k] : ms2_scalars_status(sl.sys);
        sl.remaining -= m;
        if (st != MS2_OK) sl.remaining = -1 - (long long)st;  // failed job: retire with its status
    }
}

static void retire(ms2_server S) {
    bool changed = false, any = false;
    for (const Slot &sl : S->slots)
        if (sl.remaining <= 0) any = true;
    if (any && S->batch) {  // the batch references the systems: release it first
        ms2_batch_destroy(S->batch);
        S->batch = nullptr;
        S->batch_dirty = true;
    }
    for (size_t k = 0; k < S->slots.size();) {
        Slot &sl = S->slots[k];
        if (sl.remaining <= 0) {
            const ms2_status st = sl.remaining < 0 ? (ms2_status)(-1 - sl.remaining) : MS2_OK;
            finish_slot(S, sl, st);
            S->slots.erase(S->slots.begin() + k);
            changed = true;
        } else {
            ++k;
        }
    }
    if (changed) S->batch_dirty = true;
}

static void scheduler(ms2_server S) {
    cudaSetDevice(S->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop) break;
            if (S->slots.empty()) {
                // idle: wait for a job or for the next arrival time
                if (S->queue.empty()) {
                    S->cv.wait_for(lk, std::chrono::milliseconds(50));
                    continue;
                }
                const double wait = S->queue.front().arrival - S->now();
                if (wait > 0) {
                    S->cv.wait_for(lk, std::chrono::duration<double>(std::min(wait, 0.05)));
                    continue;
                }
            }
        }
        admit(S);
        if (!S->slots.empty()) advance(S);
        retire(S);
    }
    if (S->batch) ms2_batch_destroy(S->batch);
    S->batch = nullptr;
    for (Slot &sl : S->slots) finish_slot(S, sl, MS2_ESTATE);
    S->slots.clear();
}

extern "C" ms2_status ms2_serve_open(size_t hbm_budget_bytes, int max_slots, const ms2_options *opt,
                                     ms2_server *out) {
    if (!out) return ms2_fail(MS2_EINVAL, "null output handle");
    if (hbm_budget_bytes == 0 || max_slots < 1 || max_slots > 1024)
        return ms2_fail(MS2_EINVAL, "need a budget > 0 and 1 <= max_slots <= 1024");
    ms2_server S = new ms2_server_s();
    S->budget = hbm_budget_bytes;
    S->max_slots = max_slots;
    ms2_default_options(&S->opt);
    if (opt) S->opt = *opt;
    cudaGetDevice(&S->device);
    {
        const cudaError_t e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete S;
            return ms2_fail_cuda(e, "server stream", __FILE__, __LINE__);
        }
    }
    S->t0 = std::chrono::steady_clock::now();
    S->th = std::thread(scheduler, S);
    *out = S;
    return MS2_OK;
}

extern "C" ms2_status ms2_serve_submit(ms2_server S, const ms2_job *job, long long *job_id) {
    if (!S || !job) return ms2_fail(MS2_EINVAL, "null argument");
    if (!job->models || !job->N_per_model || job->n_models < 1 || job->n_models > MS2_MAXSP)
        return ms2_fail(MS2_EINVAL, "job needs 1..%d models", MS2_MAXSP);
    if (job->steps < 1) return ms2_fail(MS2_EINVAL, "job needs steps >= 1");
    if (job->rdf_bins < 0 || job->rdf_bins > 4096) return ms2_fail(MS2_EINVAL, "rdf_bins must be 0..4096");
    ms2_status st = ms2_validate_models(job->models, job->n_models, job->elec);
    if (st != MS2_OK) return st;
    JobSpec j;
    for (int m = 0; m < job->n_models; ++m) {
        j.sites.emplace_back(job->models[m].sites, job->models[m].sites + job->models[m].n_sites);
        j.counts.push_back(job->N_per_model[m]);
    }
    j.T = job->T;
    j.rho = job->rho;
    j.cutoff = job->cutoff;
    j.elec = job->elec;
    j.steps = job->steps;
    j.arrival = job->arrival_time;
    j.seed = job->seed;
    j.rdf_bins = job->rdf_bins;
    j.rdf_every = job->rdf_every;
    {
        long long N = 0;
        for (int c : j.counts) N += c;
        if (job->R0) j.R0.assign(job->R0, job->R0 + 3 * N);
        if (job->q0) j.q0.assign(job->q0, job->q0 + 4 * N);
    }
    j.bytes = estimate_bytes(j);
    if (j.bytes > S->budget)
        return ms2_fail(MS2_EBUDGET, "job needs ~%zu bytes of device memory, budget is %zu", j.bytes, S->budget);
    std::lock_guard<std::mutex> lk(S->mu);
    j.id = S->next_id++;
    // keep the queue in arrival order (stable for equal times)
    auto it = std::upper_bound(S->queue.begin(), S->queue.end(), j,
                               [](const JobSpec &a, const JobSpec &b) { return a.arrival < b.arrival; });
    S->queue.insert(it, j);
    S->outstanding += 1;
    if (job_id) *job_id = j.id;
    S->cv.notify_all();
    return MS2_OK;
}

extern "C" ms2_status ms2_serve_poll(ms2_server S, ms2_job_result *out, int max, int *n_done) {
    if (!S || (!out && max > 0)) return ms2_fail(MS2_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    int k = 0;
    while (k < max && !S->done.empty()) {
        out[k++] = S->done.front();
        S->done.pop_front();
    }
    if (n_done) *n_done = k;
    return MS2_OK;
}

extern "C" ms2_status ms2_serve_drain(ms2_server S, double timeout_s) {
    if (!S) return ms2_fail(MS2_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(S->mu);
    const bool ok = S->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return S->outstanding == 0; });
    if (!ok) return ms2_fail(MS2_ETIMEOUT, "%lld jobs still outstanding after %.1f s", S->outstanding, timeout_s);
    return MS2_OK;
}

extern "C" ms2_status ms2_serve_close(ms2_server S) {
    if (!S) return MS2_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    int dev = 0;
    cudaGetDevice(&dev);
    cudaSetDevice(S->device);  // the stream and the block cache belong to the server's device
    if (S->stream) cudaStreamDestroy(S->stream);  // after every system of the server is gone
    delete S;
    cudaSetDevice(dev);
    return MS2_OK;
}
