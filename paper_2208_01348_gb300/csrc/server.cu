// Serving loop: EELS map / spectrum requests of different lattices admitted
// by device-memory footprint and run concurrently.
//
// Each request is one eels_solve (all its (energy, beam) points).  Requests
// wait in arrival order; a free worker takes the first waiting request whose
// footprint fits the unreserved part of the memory budget (so a small request
// may pass a large one that does not fit yet).  Every worker owns a CUDA
// stream and runs its request in a context of its own, so requests that
// arrive while others run are admitted as soon as a worker and memory free
// up, and their kernels overlap on the device.  Each request's arithmetic is
// independent of the others (per-system reductions use a fixed block
// partition), so its results are the same bits alone or in the mix.
// Device buffers are allocated stream-ordered, so one request's allocation
// or release does not stall the streams of the others.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/eelsdda.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    long long id = 0;
    // copies of the request
    int nx = 0, ny = 0, nz = 0;
    double d_nm = 0;
    double origin_nm[3] = {0, 0, 0};
    std::vector<uint8_t> occ;
    eels_opts opts{};
    std::vector<double> energies;
    std::vector<eels_c128> eps_p, eps_h;
    std::vector<eels_beam> beams;
    int n_mat = 0;
    size_t footprint = 0;
    // results
    std::vector<double> p_eels, p_cl, p_ext, p_abs;
    std::vector<eels_point_stats> stats;
    int state = EELS_JOB_QUEUED;
    int code = EELS_OK;
    std::string err;
    double t_submit = 0, t_start = 0, t_end = 0;
};

}  // namespace

struct eels_server {
    eels_server_opts o{};
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Job*> queue;
    std::map<long long, std::unique_ptr<Job>> jobs;
    size_t in_use = 0;
    int running = 0, running_max = 0, completed = 0;
    long long next_id = 1;
    bool stop = false;
    std::vector<std::thread> workers;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// First waiting job that fits the unreserved budget (nullptr if none).
Job* pick_admissible(eels_server* s) {
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        Job* j = *it;
        if (j->footprint <= s->o.hbm_budget - s->in_use) {
            s->queue.erase(it);
            return j;
        }
    }
    return nullptr;
}

void run_job(eels_server* s, Job* j, cudaStream_t st) {
    const int ne = (int)j->energies.size(), nb = (int)j->beams.size();
    const size_t np = (size_t)ne * nb;
    j->p_eels.assign(np, 0.0);
    j->p_cl.assign(j->opts.n_dir > 0 ? np : 0, 0.0);
    j->p_ext.assign(np, 0.0);
    j->p_abs.assign(np, 0.0);
    j->stats.assign(np, eels_point_stats{});
    if (s->o.flags & EELS_SERVER_DRYRUN) {
        // scheduler-only mode: hold the slot for a time that grows with the work
        std::this_thread::sleep_for(std::chrono::microseconds(200 + (long long)(np * 20)));
        j->code = EELS_OK;
        return;
    }
    eels_ctx* ctx = nullptr;
    int rc = eels_create(&ctx, s->o.device, st);
    if (rc == EELS_OK) {
        eels_grid g{j->nx, j->ny, j->nz, j->d_nm, j->occ.data(), {j->origin_nm[0], j->origin_nm[1], j->origin_nm[2]}};
        rc = eels_set_grid(ctx, &g);
        if (rc == EELS_OK)
            rc = eels_solve(ctx, &j->opts, ne, j->energies.data(), j->n_mat, j->eps_p.data(), j->eps_h.data(), nb,
                            j->beams.data(), j->p_eels.data(), j->opts.n_dir > 0 ? j->p_cl.data() : nullptr,
                            j->p_ext.data(), j->p_abs.data(), nullptr, j->stats.data());
        if (rc != EELS_OK) j->err = eels_last_error(ctx);
        eels_destroy(ctx);
    }
    j->code = rc;
}

void worker_main(eels_server* s) {
    cudaStream_t st = nullptr;
    if (!(s->o.flags & EELS_SERVER_DRYRUN)) {
        cudaSetDevice(s->o.device);
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    }
    for (;;) {
        Job* j = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || (j = pick_admissible(s)) != nullptr; });
            if (!j) break;   // stopping
            s->in_use += j->footprint;
            s->running += 1;
            s->running_max = std::max(s->running_max, s->running);
            j->state = EELS_JOB_RUNNING;
            j->t_start = s->now();
        }
        run_job(s, j, st);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->in_use -= j->footprint;
            s->running -= 1;
            s->completed += 1;
            j->t_end = s->now();
            j->state = (j->code == EELS_OK || j->code == EELS_E_NOT_CONVERGED) ? EELS_JOB_DONE : EELS_JOB_FAILED;
        }
        s->cv.notify_all();
    }
    if (st) cudaStreamDestroy(st);
}

void fill_info(const Job* j, eels_job_info* info) {
    if (!info) return;
    info->state = j->state;
    info->code = j->code;
    info->t_submit = j->t_submit;
    info->t_start = j->t_start;
    info->t_end = j->t_end;
    info->footprint = j->footprint;
    info->n_points = (int)(j->energies.size() * j->beams.size());
}

}  // namespace

// A single asynchronous eels_solve: copies of the inputs, the thread that
// runs it, and its return code.
struct eels_job {
    eels_opts opts{};
    std::vector<double> energies;
    std::vector<eels_c128> eps_p, eps_h;
    std::vector<eels_beam> beams;
    int n_mat = 0;
    std::thread worker;
    std::mutex mu;
    bool done = false;
    int code = EELS_OK;
};

extern "C" {

int eels_server_create(eels_server** out, const eels_server_opts* o) {
    if (!out || !o || o->max_concurrent < 1) return EELS_E_INVALID_ARG;
    *out = nullptr;
    auto* s = new eels_server();
    s->o = *o;
    if (!(o->flags & EELS_SERVER_DRYRUN)) {
        int n = 0;
        if (cudaGetDeviceCount(&n) != cudaSuccess || o->device < 0 || o->device >= n) {
            cudaGetLastError();
            delete s;
            return EELS_E_CUDA;
        }
        if (s->o.hbm_budget == 0) {
            size_t fr = 0, tot = 0;
            cudaSetDevice(o->device);
            if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { delete s; return EELS_E_CUDA; }
            s->o.hbm_budget = (size_t)(0.8 * (double)fr);
        }
    } else if (s->o.hbm_budget == 0) {
        delete s;
        return EELS_E_INVALID_ARG;
    }
    s->t0 = Clock::now();
    for (int i = 0; i < s->o.max_concurrent; ++i) s->workers.emplace_back(worker_main, s);
    *out = s;
    return EELS_OK;
}

int eels_server_submit(eels_server* s, const eels_grid* g, const eels_opts* o, int n_energy, const double* energy_eV,
                       int n_mat, const eels_c128* eps_p, const eels_c128* eps_h, int n_beam, const eels_beam* beams,
                       long long* job_id) {
    if (!s || !g || !o || !g->occ || n_energy <= 0 || n_beam <= 0 || n_mat <= 0 || !energy_eV || !eps_p || !eps_h ||
        !beams || !job_id)
        return EELS_E_INVALID_ARG;
    auto j = std::make_unique<Job>();
    j->nx = g->nx; j->ny = g->ny; j->nz = g->nz; j->d_nm = g->d_nm;
    for (int a = 0; a < 3; ++a) j->origin_nm[a] = g->origin_nm[a];
    j->occ.assign(g->occ, g->occ + (size_t)g->nx * g->ny * g->nz);
    j->opts = *o;
    j->energies.assign(energy_eV, energy_eV + n_energy);
    j->eps_p.assign(eps_p, eps_p + (size_t)n_energy * n_mat);
    j->eps_h.assign(eps_h, eps_h + n_energy);
    j->beams.assign(beams, beams + n_beam);
    j->n_mat = n_mat;
    // memory share per request: the largest batch whose footprint fits
    // budget / max_concurrent (at least one system)
    const size_t share = s->o.hbm_budget / (size_t)s->o.max_concurrent;
    const int n_sys = n_energy * n_beam;
    int batch = o->max_batch > 0 ? std::min(o->max_batch, n_sys) : n_sys;
    size_t fp = 0;
    int rc = eels_query_footprint(g, o, 1, &fp);
    if (rc != EELS_OK) return rc;
    if (fp > s->o.hbm_budget) return EELS_E_OOM;
    while (batch > 1) {
        rc = eels_query_footprint(g, o, batch, &fp);
        if (rc != EELS_OK) return rc;
        if (fp <= share) break;
        batch = std::max(1, batch / 2);
    }
    eels_query_footprint(g, o, batch, &fp);
    j->opts.max_batch = batch;
    j->footprint = fp;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        j->id = s->next_id++;
        j->t_submit = s->now();
        *job_id = j->id;
        s->queue.push_back(j.get());
        s->jobs[j->id] = std::move(j);
    }
    s->cv.notify_all();
    return EELS_OK;
}

int eels_server_poll(eels_server* s, long long job, eels_job_info* info) {
    if (!s) return EELS_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job);
    if (it == s->jobs.end()) return EELS_E_INVALID_ARG;
    fill_info(it->second.get(), info);
    return EELS_OK;
}

int eels_server_wait(eels_server* s, long long job, double* p_eels, double* p_cl, double* p_ext, double* p_abs,
                     eels_point_stats* stats, eels_job_info* info) {
    if (!s) return EELS_E_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job);
    if (it == s->jobs.end()) return EELS_E_INVALID_ARG;
    Job* j = it->second.get();
    s->cv.wait(lk, [&] { return j->state == EELS_JOB_DONE || j->state == EELS_JOB_FAILED; });
    fill_info(j, info);
    const size_t np = j->p_eels.size();
    if (j->state == EELS_JOB_DONE) {
        if (p_eels) std::memcpy(p_eels, j->p_eels.data(), np * sizeof(double));
        if (p_cl && !j->p_cl.empty()) std::memcpy(p_cl, j->p_cl.data(), np * sizeof(double));
        if (p_ext) std::memcpy(p_ext, j->p_ext.data(), np * sizeof(double));
        if (p_abs) std::memcpy(p_abs, j->p_abs.data(), np * sizeof(double));
        if (stats) std::memcpy(stats, j->stats.data(), np * sizeof(eels_point_stats));
    }
    return j->code;
}

int eels_server_stats(eels_server* s, int* running_max, int* completed, size_t* in_use) {
    if (!s) return EELS_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (running_max) *running_max = s->running_max;
    if (completed) *completed = s->completed;
    if (in_use) *in_use = s->in_use;
    return EELS_OK;
}

void eels_server_destroy(eels_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->queue.clear();   // requests never admitted are dropped
    }
    s->cv.notify_all();
    for (auto& t : s->workers) t.join();
    delete s;
}

// ---- one request on the caller's context, in a host thread ----

int eels_solve_async(eels_ctx* ctx, const eels_opts* opts, int n_energy, const double* energy_eV, int n_mat,
                     const eels_c128* eps_p, const eels_c128* eps_h, int n_beam, const eels_beam* beams,
                     double* p_eels, double* p_cl, double* p_ext, double* p_abs, eels_c128* p_out,
                     eels_point_stats* stats, eels_job** job) {
    if (!job) return EELS_E_INVALID_ARG;
    *job = nullptr;
    if (!ctx || !opts || n_energy <= 0 || n_beam <= 0 || n_mat <= 0 || !energy_eV || !eps_p || !eps_h || !beams ||
        !p_eels)
        return EELS_E_INVALID_ARG;
    auto* j = new eels_job();
    j->opts = *opts;
    j->energies.assign(energy_eV, energy_eV + n_energy);
    j->eps_p.assign(eps_p, eps_p + (size_t)n_energy * n_mat);
    j->eps_h.assign(eps_h, eps_h + n_energy);
    j->beams.assign(beams, beams + n_beam);
    j->n_mat = n_mat;
    j->worker = std::thread([j, ctx, p_eels, p_cl, p_ext, p_abs, p_out, stats] {
        const int code = eels_solve(ctx, &j->opts, (int)j->energies.size(), j->energies.data(), j->n_mat,
                                    j->eps_p.data(), j->eps_h.data(), (int)j->beams.size(), j->beams.data(), p_eels,
                                    p_cl, p_ext, p_abs, p_out, stats);
        std::lock_guard<std::mutex> lk(j->mu);
        j->code = code;
        j->done = true;
    });
    *job = j;
    return EELS_OK;
}

int eels_job_poll(eels_job* job, int* done) {
    if (!job || !done) return EELS_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(job->mu);
    *done = job->done ? 1 : 0;
    return EELS_OK;
}

int eels_job_wait(eels_job* job) {
    if (!job) return EELS_E_INVALID_ARG;
    job->worker.join();
    const int code = job->code;
    delete job;
    return code;
}

}  // extern "C"
