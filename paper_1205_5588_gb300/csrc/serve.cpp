// serve.cpp — continuous-batching server for hysteresis-loop and temperature-scan jobs (the
// paper's two kinds of runs, Sec. 3, Fig. 3, Fig. 5) on one GPU.
//
// Clients submit jobs (a height map, layers, seed, initial state and a schedule) at any time.
// A worker thread admits queued jobs while the device-memory budget allows (each admitted job
// holds its film on the device until it finishes), then advances every admitted film by at most
// `sweeps_per_tick` sweeps in one batched launch (isf_batch_run_sweeps), retires the films whose
// schedule is done, and repeats: jobs that arrive while a tick runs join the next one, so their
// work overlaps with the jobs already on the GPU.  Each film keeps its own RNG key and sweep
// counter, so a job's result is the same alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "capi_internal.h"

using namespace isf;

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    int64_t id = 0;
    std::vector<uint8_t> heights;
    int32_t rows = 0, cols = 0, layers = 0;
    uint32_t flags = 0;
    uint64_t seed = 0;
    int32_t init = 0;
    std::vector<double> T, h;
    std::vector<int32_t> eq, meas;
    double J = 1.0, h_s = 0.0;
    // state
    int32_t state = 0;            // ISF_JOB_*
    isf_lattice* lat = nullptr;
    size_t bytes = 0;
    int64_t attempts = 0;
    Clock::time_point t_submit, t_admit, t_done;
    int64_t tick_first = -1, tick_last = -1, tick_count = 0;   // the batched launches it ran in
    std::vector<isf_step_obs> result;
    int32_t err = 0;
    std::string msg;
};

int fail(int code, const std::string& m) { return set_last_error(code, m.c_str()); }

}  // namespace

struct isf_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    std::deque<Job*> queue;
    std::vector<Job*> active;
    std::unordered_map<int64_t, Job*> jobs;
    size_t budget = 0, used = 0, peak = 0;
    int64_t sweeps_per_tick = 0;
    int64_t next_id = 1;
    bool stop = false;
    int device = 0;
    // statistics
    int64_t submitted = 0, completed = 0, failed = 0, ticks = 0, attempts_done = 0;
    double busy_s = 0.0;
    Clock::time_point t0;
    int32_t worker_err = 0;
    std::string worker_msg;
};

namespace {

size_t job_bytes(const Job& j) {
    const size_t film = isf_lattice_bytes(j.rows, j.cols, j.layers, j.flags);
    if (!film) return 0;
    return film + j.T.size() * (kTableStride * 4 + 8 + sizeof(StepRec)) + 4096;
}

void finish(isf_server* S, Job* j, int32_t state) {
    j->state = state;
    j->t_done = Clock::now();
    if (j->lat) {
        isf_lattice_destroy(j->lat);
        j->lat = nullptr;
    }
    S->used -= j->bytes;
    j->bytes = 0;
    if (state == ISF_JOB_DONE) ++S->completed;
    else ++S->failed;
}

void worker_main(isf_server* S) {
    cudaSetDevice(S->device);
    cudaStream_t stream = nullptr;
    isf_batch* batch = nullptr;
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess || isf_batch_create(&batch)) {
        std::lock_guard<std::mutex> lock(S->mu);
        S->worker_err = ISF_ERR_CUDA;
        S->worker_msg = "server worker could not start";
        S->stop = true;
        S->cv_done.notify_all();
        return;
    }
    for (;;) {
        std::vector<Job*> admit;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            S->cv_work.wait(lock, [&] { return S->stop || !S->queue.empty() || !S->active.empty(); });
            if (S->stop && S->queue.empty() && S->active.empty()) break;
            // admission by device memory: a job enters when its film fits the budget
            while (!S->queue.empty()) {
                Job* j = S->queue.front();
                if (j->bytes > S->budget) {
                    S->queue.pop_front();
                    j->err = ISF_ERR_OOM;
                    j->msg = "job needs more device memory than the whole budget";
                    j->state = ISF_JOB_FAILED;
                    j->t_done = Clock::now();
                    ++S->failed;
                    continue;
                }
                if (S->used + j->bytes > S->budget) break;
                S->queue.pop_front();
                S->used += j->bytes;
                S->peak = std::max(S->peak, S->used);
                admit.push_back(j);
            }
        }
        for (Job* j : admit) {
            int rc = isf_lattice_create(j->heights.data(), j->rows, j->cols, j->layers, j->flags, j->seed, j->init,
                                        stream, &j->lat);
            if (!rc) rc = isf_set_schedule(j->lat, (int32_t)j->T.size(), j->T.data(), j->h.data(), j->eq.data(),
                                           j->meas.data(), j->J, j->h_s);
            std::lock_guard<std::mutex> lock(S->mu);
            if (rc) {
                j->err = rc;
                j->msg = isf_last_error();
                finish(S, j, ISF_JOB_FAILED);
                S->cv_done.notify_all();
                continue;
            }
            int64_t n_occ = 0, total = 0;
            isf_lattice_info(j->lat, &n_occ, nullptr, nullptr, nullptr);
            for (size_t k = 0; k < j->T.size(); ++k) total += (int64_t)j->eq[k] + j->meas[k];
            j->attempts = n_occ * total;
            j->state = ISF_JOB_RUNNING;
            j->t_admit = Clock::now();
            S->active.push_back(j);
        }
        std::vector<Job*> act;
        {
            std::lock_guard<std::mutex> lock(S->mu);
            act = S->active;
        }
        if (act.empty()) continue;
        const isf::TraceRange trace("isf_server_tick");
        isf_batch_clear(batch);
        for (Job* j : act) isf_batch_add(batch, j->lat);
        const auto t_start = Clock::now();
        int rc = isf_batch_run_sweeps(batch, S->sweeps_per_tick, stream);
        cudaError_t ce = rc ? cudaSuccess : cudaStreamSynchronize(stream);
        const double dt = std::chrono::duration<double>(Clock::now() - t_start).count();
        std::vector<Job*> done;
        for (Job* j : act)
            if (rc || ce != cudaSuccess || sweeps_remaining(j->lat) == 0) done.push_back(j);
        for (Job* j : done) {
            if (!rc && ce == cudaSuccess) {
                j->result.resize(j->T.size());
                int32_t n = 0;
                const int r2 = isf_read_observables(j->lat, j->result.data(), (int32_t)j->result.size(), &n);
                if (r2) { j->err = r2; j->msg = isf_last_error(); }
            } else {
                j->err = rc ? rc : ISF_ERR_CUDA;
                j->msg = rc ? isf_last_error() : cudaGetErrorString(ce);
            }
        }
        std::lock_guard<std::mutex> lock(S->mu);
        S->busy_s += dt;
        for (Job* j : act) {
            if (j->tick_first < 0) j->tick_first = S->ticks;
            j->tick_last = S->ticks;
            ++j->tick_count;
        }
        ++S->ticks;
        for (Job* j : done) {
            if (!j->err) S->attempts_done += j->attempts;
            finish(S, j, j->err ? ISF_JOB_FAILED : ISF_JOB_DONE);
            S->active.erase(std::find(S->active.begin(), S->active.end(), j));
        }
        if (!done.empty()) S->cv_done.notify_all();
    }
    isf_batch_destroy(batch);
    cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

int isf_server_create(size_t device_budget_bytes, int64_t sweeps_per_tick, isf_server** out) {
    if (!out || device_budget_bytes == 0 || sweeps_per_tick < 1) return fail(ISF_ERR_ARG, "bad arguments");
    isf_server* S = new (std::nothrow) isf_server();
    if (!S) return fail(ISF_ERR_OOM, "host allocation failed");
    if (cudaGetDevice(&S->device) != cudaSuccess) { delete S; return fail(ISF_ERR_CUDA, "cudaGetDevice"); }
    S->budget = device_budget_bytes;
    S->sweeps_per_tick = sweeps_per_tick;
    S->t0 = Clock::now();
    try {
        S->worker = std::thread(worker_main, S);
    } catch (...) {
        delete S;
        return fail(ISF_ERR_OOM, "cannot start the worker thread");
    }
    *out = S;
    return ISF_OK;
}

int isf_server_submit(isf_server* S, const isf_job* in, int64_t* id) {
    if (!S || !in || !id || !in->heights || !in->T || !in->h || !in->sweeps_eq || !in->sweeps_meas || in->nsteps < 1)
        return fail(ISF_ERR_ARG, "bad arguments");
    Job* j = new (std::nothrow) Job();
    if (!j) return fail(ISF_ERR_OOM, "host allocation failed");
    j->rows = in->rows; j->cols = in->cols; j->layers = in->layers; j->flags = in->flags;
    j->seed = in->seed; j->init = in->init; j->J = in->J; j->h_s = in->h_s;
    j->bytes = job_bytes(*j);
    if (!j->bytes) { delete j; return fail(ISF_ERR_ARG, "invalid film shape or flags"); }
    j->heights.assign(in->heights, in->heights + (size_t)in->rows * in->cols);
    j->T.assign(in->T, in->T + in->nsteps);
    j->h.assign(in->h, in->h + in->nsteps);
    j->eq.assign(in->sweeps_eq, in->sweeps_eq + in->nsteps);
    j->meas.assign(in->sweeps_meas, in->sweeps_meas + in->nsteps);
    j->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->stop) { delete j; return fail(ISF_ERR_STATE, "server is stopping"); }
        j->id = S->next_id++;
        S->jobs[j->id] = j;
        S->queue.push_back(j);
        ++S->submitted;
        *id = j->id;
    }
    S->cv_work.notify_one();
    return ISF_OK;
}

int isf_server_wait(isf_server* S, int64_t id, double timeout_s, int32_t* state) {
    if (!S || !state) return fail(ISF_ERR_ARG, "bad arguments");
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return fail(ISF_ERR_ARG, "unknown job id");
    Job* j = it->second;
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    S->cv_done.wait_until(lock, until, [&] { return j->state >= ISF_JOB_DONE || S->worker_err; });
    *state = j->state;
    if (j->state < ISF_JOB_DONE && S->worker_err) return fail(S->worker_err, S->worker_msg);
    return ISF_OK;
}

int isf_server_poll(isf_server* S, int64_t id, int32_t* state, isf_step_obs* out, int32_t max, int32_t* n_out,
                    double* latency_s) {
    if (!S || !state) return fail(ISF_ERR_ARG, "bad arguments");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return fail(ISF_ERR_ARG, "unknown job id");
    Job* j = it->second;
    *state = j->state;
    if (n_out) *n_out = 0;
    if (j->state == ISF_JOB_FAILED) return fail(j->err ? j->err : ISF_ERR_STATE, j->msg);
    if (j->state != ISF_JOB_DONE) return ISF_OK;
    if (latency_s) *latency_s = std::chrono::duration<double>(j->t_done - j->t_submit).count();
    const int32_t n = std::min<int32_t>((int32_t)j->result.size(), std::max(max, 0));
    if (out && n) std::memcpy(out, j->result.data(), (size_t)n * sizeof(isf_step_obs));
    if (n_out) *n_out = n;
    return ISF_OK;
}

int isf_server_job_ticks(isf_server* S, int64_t id, int64_t* out3) {
    if (!S || !out3) return fail(ISF_ERR_ARG, "bad arguments");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return fail(ISF_ERR_ARG, "unknown job id");
    out3[0] = it->second->tick_first;
    out3[1] = it->second->tick_last;
    out3[2] = it->second->tick_count;
    return ISF_OK;
}

int isf_server_release(isf_server* S, int64_t id) {
    if (!S) return fail(ISF_ERR_ARG, "bad arguments");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return fail(ISF_ERR_ARG, "unknown job id");
    if (it->second->state < ISF_JOB_DONE) return fail(ISF_ERR_STATE, "job not finished");
    delete it->second;
    S->jobs.erase(it);
    return ISF_OK;
}

int isf_server_stats(isf_server* S, int64_t* out8, double* out4) {
    if (!S) return fail(ISF_ERR_ARG, "bad arguments");
    std::lock_guard<std::mutex> lock(S->mu);
    if (out8) {
        const int64_t v[8] = {S->submitted, S->completed, S->failed, (int64_t)S->active.size(), (int64_t)S->queue.size(),
                              S->ticks, S->attempts_done, (int64_t)S->peak};
        std::memcpy(out8, v, sizeof v);
    }
    if (out4) {
        out4[0] = S->busy_s;
        out4[1] = std::chrono::duration<double>(Clock::now() - S->t0).count();
        out4[2] = (double)S->used;
        out4[3] = (double)S->budget;
    }
    return ISF_OK;
}

void isf_server_destroy(isf_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto& kv : S->jobs) {
        if (kv.second->lat) isf_lattice_destroy(kv.second->lat);
        delete kv.second;
    }
    delete S;
}

}  // extern "C"
