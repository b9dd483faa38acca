// batch.cpp — batched films: many independent films, each with its own height map, seed and
// temperature / field schedule (the paper's temperature scans and hysteresis loops, Sec. 3,
// Fig. 3, Fig. 5, run for many samples at once), advanced to the end of their schedules by one
// persistent launch per size class, optionally replayed from a captured CUDA graph.
//
// Classes: films whose int8 layout fits one CTA's shared memory go to a single-CTA queue
// kernel (A); films that need a cluster go to a cluster queue kernel (B, K CTAs per film);
// the remaining films (bit-packed ones, periodic-column ones, and int8 ones too large for a
// cluster's shared memory) keep their state in global memory and go to a queue kernel that runs
// each on one CTA (D, up to 2^20 lattice sites) or on one cluster of 8 CTAs (E, up to 2^24).
// The four launches run concurrently on forked streams and every CTA / cluster pulls films from
// its queue (longest first).  Larger films (C) run after them on the multi-CTA global-memory
// path, one launch each.  Every film keeps its own RNG key and
// sweep counter, so its trajectory is the one it has alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "capi_internal.h"

using namespace isf;

struct isf_batch {
    std::vector<isf_lattice*> films;
    int32_t threads_a = 0, K_b = 0, threads_b = 0;   // 0 = tuned or default
    bool use_graph = false;
    // device-side queues: class A entries, then class B entries; class D entries
    ResArgs* d_desc = nullptr;
    size_t cap = 0;
    unsigned* d_next = nullptr;  // queue counters of A, B, D, E; films D and E took from A and B
    ResArgs* h_desc = nullptr;   // pinned staging
    SweepArgs* d_gdesc = nullptr;   // class D entries, then class E entries
    SweepArgs* h_gdesc = nullptr;
    size_t gcap = 0;
    cudaStream_t sa = nullptr, sb = nullptr, sd = nullptr, se = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_a = nullptr, ev_b = nullptr, ev_d = nullptr, ev_e = nullptr, ev_done = nullptr;
    bool pending = false;
    // one single-kernel graph per queue kernel (A, B, D, E), for the launch shape in gsig
    cudaGraphExec_t gx[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t gsig[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    // last run
    int32_t n_a = 0, n_b = 0, n_c = 0, units_a = 0, units_b = 0, used_K = 0, used_ta = 0, used_tb = 0;
    int32_t n_d = 0, units_d = 0, n_e = 0, units_e = 0;
    int device = 0;
};

namespace {

constexpr int kDefaultThreadsA = 256;
constexpr int kDefaultK = 16;
constexpr int kDefaultThreadsB = 512;
constexpr int kThreadsD = 256;                      // one CTA per film, state in global memory
constexpr int64_t kMaxSitesD = (int64_t)1 << 20;    // larger films take a cluster (class E)
constexpr int kKE = 8, kThreadsE = 256;             // one cluster of 8 CTAs per film, global memory
constexpr int64_t kMaxSitesE = (int64_t)1 << 24;    // larger films take the whole GPU (class C)

int fail(int code, const std::string& msg) { return set_last_error(code, msg.c_str()); }

int cuda_fail(cudaError_t e, const char* what) {
    return fail(ISF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define CUDA_TRY(expr, what)                                  \
    do {                                                      \
        cudaError_t e_ = (cudaError_t)(expr);                 \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);    \
    } while (0)

int ensure_streams(isf_batch* b) {
    if (b->sa) return ISF_OK;
    CUDA_TRY(cudaGetDevice(&b->device), "cudaGetDevice");
    CUDA_TRY(cudaStreamCreateWithFlags(&b->sa, cudaStreamNonBlocking), "stream");
    CUDA_TRY(cudaStreamCreateWithFlags(&b->sb, cudaStreamNonBlocking), "stream");
    CUDA_TRY(cudaStreamCreateWithFlags(&b->sd, cudaStreamNonBlocking), "stream");
    CUDA_TRY(cudaStreamCreateWithFlags(&b->se, cudaStreamNonBlocking), "stream");
    CUDA_TRY(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming), "event");
    CUDA_TRY(cudaEventCreateWithFlags(&b->ev_a, cudaEventDisableTiming), "event");
    CUDA_TRY(cudaEventCreateWithFlags(&b->ev_b, cudaEventDisableTiming), "event");
    CUDA_TRY(cudaEventCreateWithFlags(&b->ev_d, cudaEventDisableTiming), "event");
    CUDA_TRY(cudaEventCreateWithFlags(&b->ev_e, cudaEventDisableTiming), "event");
    CUDA_TRY(cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming), "event");
    CUDA_TRY(cudaMalloc(&b->d_next, 6 * sizeof(unsigned)), "cudaMalloc");
    CUDA_TRY(cudaMemset(b->d_next, 0, 6 * sizeof(unsigned)), "cudaMemset");
    return ISF_OK;
}

void drop_graphs(isf_batch* b) {
    for (cudaGraphExec_t& g : b->gx)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
}

int ensure_gcapacity(isf_batch* b, size_t n) {
    if (n <= b->gcap) return ISF_OK;
    if (b->d_gdesc) cudaFree(b->d_gdesc);
    if (b->h_gdesc) cudaFreeHost(b->h_gdesc);
    b->d_gdesc = nullptr;
    b->h_gdesc = nullptr;
    b->gcap = 0;
    drop_graphs(b);
    CUDA_TRY(cudaMalloc(&b->d_gdesc, n * sizeof(SweepArgs)), "cudaMalloc batch queue");
    CUDA_TRY(cudaMallocHost(&b->h_gdesc, n * sizeof(SweepArgs)), "cudaMallocHost batch queue");
    b->gcap = n;
    return ISF_OK;
}

int ensure_capacity(isf_batch* b, size_t n) {
    if (n <= b->cap) return ISF_OK;
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->h_desc) cudaFreeHost(b->h_desc);
    b->d_desc = nullptr;
    b->h_desc = nullptr;
    b->cap = 0;
    drop_graphs(b);
    CUDA_TRY(cudaMalloc(&b->d_desc, n * sizeof(ResArgs)), "cudaMalloc batch queue");
    CUDA_TRY(cudaMallocHost(&b->h_desc, n * sizeof(ResArgs)), "cudaMallocHost batch queue");
    b->cap = n;
    return ISF_OK;
}

// One queue kernel launched on its stream, or (graph mode) its single-kernel graph, captured from
// that launch the first time and replayed after.  The kernels are launched, graph or not, in the
// same host order, so they reach the GPU in a fixed order: the sibling kernel nodes of one graph
// do not, and which persistent kernel the hardware places first decides how the SMs are shared.
// Returns a cudaError_t value.
template <class F>
int launch_on(isf_batch* b, int cls, cudaStream_t st, F&& launch) {
    if (!b->use_graph) return launch(st);
    if (!b->gx[cls]) {
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
        if (ce != cudaSuccess) return (int)ce;
        const int e = launch(st);
        ce = cudaStreamEndCapture(st, &g);
        if (e || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return e ? e : (int)ce;
        }
        ce = cudaGraphInstantiate(&b->gx[cls], g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) { b->gx[cls] = nullptr; return (int)ce; }
    }
    return (int)cudaGraphLaunch(b->gx[cls], st);
}

// The launch sequence: queue uploads, counters, fork, the persistent launches, join.
int enqueue(isf_batch* b, cudaStream_t s, int n_a, int n_b, int K, int ta, int tb, uint32_t smem_a,
            uint32_t smem_b, int units_a, int units_b, int n_d, int units_d, int n_e, int units_e) {
    const size_t n = (size_t)n_a + n_b;
    if (n)
        CUDA_TRY(cudaMemcpyAsync(b->d_desc, b->h_desc, n * sizeof(ResArgs), cudaMemcpyHostToDevice, s), "upload queue");
    if (n_d + n_e)
        CUDA_TRY(cudaMemcpyAsync(b->d_gdesc, b->h_gdesc, (size_t)(n_d + n_e) * sizeof(SweepArgs),
                                 cudaMemcpyHostToDevice, s), "upload queue");
    CUDA_TRY(cudaMemsetAsync(b->d_next, 0, 6 * sizeof(unsigned), s), "reset queue");
    CUDA_TRY(cudaEventRecord(b->ev_fork, s), "fork");
    if (n_d) {
        CUDA_TRY(cudaStreamWaitEvent(b->sd, b->ev_fork, 0), "fork");
        // once its own films are done, it takes the single-CTA resident films not yet started
        const StealQueue steal{b->d_desc, n_a, b->d_next + 0, b->d_next + 4};
        int e = launch_on(b, 2, b->sd, [&](cudaStream_t st) {
            return launch_batch_global(b->d_gdesc, n_d, b->d_next + 2, kThreadsD, units_d, st, steal);
        });
        if (e) return cuda_fail((cudaError_t)e, "batch launch (one CTA per film, global memory)");
        CUDA_TRY(cudaEventRecord(b->ev_d, b->sd), "join");
        CUDA_TRY(cudaStreamWaitEvent(s, b->ev_d, 0), "join");
    }
    if (n_e) {
        CUDA_TRY(cudaStreamWaitEvent(b->se, b->ev_fork, 0), "fork");
        // once its own films are done, it takes the resident cluster films not yet started
        const StealQueue steal{b->d_desc + n_a, n_b, b->d_next + 1, b->d_next + 5};
        int e = launch_on(b, 3, b->se, [&](cudaStream_t st) {
            return launch_batch_cluster_global(b->d_gdesc + n_d, n_e, b->d_next + 3, kKE, kThreadsE, units_e, st, steal);
        });
        if (e) return cuda_fail((cudaError_t)e, "batch launch (one cluster per film, global memory)");
        CUDA_TRY(cudaEventRecord(b->ev_e, b->se), "join");
        CUDA_TRY(cudaStreamWaitEvent(s, b->ev_e, 0), "join");
    }
    if (n_a) {
        CUDA_TRY(cudaStreamWaitEvent(b->sa, b->ev_fork, 0), "fork");
        int e = launch_on(b, 0, b->sa, [&](cudaStream_t st) {
            return launch_batch(b->d_desc, n_a, b->d_next, 1, ta, smem_a, units_a, st);
        });
        if (e) return cuda_fail((cudaError_t)e, "batch launch (single-CTA films)");
        CUDA_TRY(cudaEventRecord(b->ev_a, b->sa), "join");
        CUDA_TRY(cudaStreamWaitEvent(s, b->ev_a, 0), "join");
    }
    if (n_b) {
        CUDA_TRY(cudaStreamWaitEvent(b->sb, b->ev_fork, 0), "fork");
        int e = launch_on(b, 1, b->sb, [&](cudaStream_t st) {
            return launch_batch(b->d_desc + n_a, n_b, b->d_next + 1, K, tb, smem_b, units_b, st);
        });
        if (e) return cuda_fail((cudaError_t)e, "batch launch (cluster films)");
        CUDA_TRY(cudaEventRecord(b->ev_b, b->sb), "join");
        CUDA_TRY(cudaStreamWaitEvent(s, b->ev_b, 0), "join");
    }
    return ISF_OK;
}

struct Item {
    isf_lattice* L;
    int64_t nsweeps;
    ResPlan plan;
    double work;
};

// ---- autotuner --------------------------------------------------------------------------------
// A probe: a film shape (layers, row and column size classes) on a device at a launch shape
// (cluster size K, threads); its time in ms, negative when the shape does not run.
struct TuneKey {
    std::string dev;
    int K, threads, L, rh_bucket, ch_bucket;
    bool operator==(const TuneKey& o) const {
        return dev == o.dev && K == o.K && threads == o.threads && L == o.L && rh_bucket == o.rh_bucket &&
               ch_bucket == o.ch_bucket;
    }
};
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, double>> g_tune_cache;

int bucket(int v) {
    int b = 1;
    while (b < v) b *= 2;
    return b;
}

std::string device_name() {
    int dev = 0;
    cudaDeviceProp p{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    return p.name;
}

// Time `sweeps` sweeps of a throw-away copy of film L with the resident kernel at (K, threads).
double probe(const isf_lattice* L, int K, int threads, int sweeps, cudaStream_t s) {
    isf_lattice* P = nullptr;
    if (isf_lattice_create(L->heights.data(), L->lay.R, L->lay.C, L->lay.L, L->lay.flags, L->seed, 0, s, &P)) return -1;
    const double T = L->nsteps ? L->T[L->nsteps / 2] : 3.0, h = 0.0;
    const int32_t eq = 0, meas = sweeps;
    double best = -1;
    if (!isf_set_schedule(P, 1, &T, &h, &eq, &meas, 1.0, 0.0) && !isf_set_path(P, ISF_PATH_RESIDENT) &&
        !isf_set_launch(P, K, threads) && !isf_set_item_sites(P, 16)) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        for (int rep = 0; rep < 2; ++rep) {
            isf_set_schedule(P, 1, &T, &h, &eq, &meas, 1.0, 0.0);
            cudaEventRecord(a, s);
            const int rc = isf_run_sweeps(P, -1, s);
            cudaEventRecord(b, s);
            if (rc || cudaEventSynchronize(b) != cudaSuccess) { best = -1; break; }
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            if (rep > 0) best = ms;   // the first run warms the path
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
    isf_lattice_destroy(P);
    cudaGetLastError();
    return best;
}

}  // namespace

extern "C" {

int isf_batch_create(isf_batch** out) {
    if (!out) return fail(ISF_ERR_ARG, "out is NULL");
    *out = new (std::nothrow) isf_batch();
    if (!*out) return fail(ISF_ERR_OOM, "host allocation failed");
    return ISF_OK;
}

int isf_batch_add(isf_batch* b, isf_lattice* L) {
    if (!b || !L) return fail(ISF_ERR_ARG, "bad arguments");
    if (!L->nsteps) return fail(ISF_ERR_STATE, "the film has no schedule");
    if (L->f.slab) return fail(ISF_ERR_STATE, "a slab film advances by isf_run_pass, not in a batch");
    if (std::find(b->films.begin(), b->films.end(), L) != b->films.end()) return fail(ISF_ERR_ARG, "film already in the batch");
    b->films.push_back(L);
    return ISF_OK;
}

int isf_batch_clear(isf_batch* b) {
    if (!b) return fail(ISF_ERR_ARG, "batch is NULL");
    b->films.clear();
    return ISF_OK;
}

int isf_batch_set_launch(isf_batch* b, int32_t threads_single, int32_t cluster_K, int32_t threads_cluster) {
    auto bad_threads = [](int32_t t) { return t != 0 && (t % 32 || t < 64 || t > 512); };
    if (!b || cluster_K < 0 || cluster_K > 16 || bad_threads(threads_single) || bad_threads(threads_cluster))
        return fail(ISF_ERR_ARG, "threads: 0 or multiples of 32 in 64..512; cluster size 0..16");
    b->threads_a = threads_single;
    b->K_b = cluster_K;
    b->threads_b = threads_cluster;
    return ISF_OK;
}

int isf_batch_set_graph(isf_batch* b, int32_t on) {
    if (!b) return fail(ISF_ERR_ARG, "batch is NULL");
    b->use_graph = on != 0;
    return ISF_OK;
}

namespace {
// Probe time of a film's shape at (K, threads), cached for the process.
double cached_probe(const isf_lattice* L, int K, int threads, const std::string& dev, cudaStream_t s) {
    const TuneKey key{dev, K, threads, L->lay.L, bucket(L->lay.Rh), bucket(L->lay.Ch)};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (auto& kv : g_tune_cache)
            if (kv.first == key) return kv.second;
    }
    const double t = probe(L, K, threads, 20, s);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.push_back({key, t});
    return t;
}
}  // namespace

int isf_batch_tune(isf_batch* b, void* cuda_stream) {
    if (!b) return fail(ISF_ERR_ARG, "batch is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const std::string dev = device_name();
    const int ths[4] = {128, 256, 384, 512};
    // single-CTA class: the threads that run its largest film fastest
    const isf_lattice* rep0 = nullptr;
    double rep0_work = 0;
    std::vector<const isf_lattice*> cluster_films;
    for (isf_lattice* L : b->films) {
        if (L->lay.packed || (L->lay.flags & ISF_PERIODIC_X)) continue;
        ResPlan p;
        const double w = (double)L->lay.L * L->lay.Rh * L->lay.Ch;
        if (resident_plan(L->f, 1, 0, 16, &p) == 0) {
            if (w > rep0_work) { rep0_work = w; rep0 = L; }
        } else if (resident_plan(L->f, 16, 0, 16, &p) == 0) {
            cluster_films.push_back(L);
        }
        cudaGetLastError();
    }
    if (rep0) {
        double best_t = 1e300;
        int best_th = kDefaultThreadsA;
        for (int th : ths) {
            const double t = cached_probe(rep0, 1, th, dev, s);
            if (t > 0 && t < best_t) { best_t = t; best_th = th; }
        }
        b->threads_a = best_th;
    }
    // cluster class: for each cluster size, the films that fit it queue over the co-resident
    // clusters, so the size is chosen by (probe time of the largest film that fits) x (rounds of
    // the queue); films that fit only the larger size run on the global-memory cluster kernel
    double best_score = 1e300;
    for (int K : {8, 16}) {
        const isf_lattice* rep = nullptr;
        double rep_work = 0;
        int n_fit = 0;
        for (const isf_lattice* L : cluster_films) {
            ResPlan p;
            if (resident_plan(L->f, K, 0, 16, &p) != 0) { cudaGetLastError(); continue; }
            ++n_fit;
            const double w = (double)L->lay.L * L->lay.Rh * L->lay.Ch;
            if (w > rep_work) { rep_work = w; rep = L; }
        }
        if (!rep) continue;
        for (int th : ths) {
            const double t = cached_probe(rep, K, th, dev, s);
            ResPlan p;
            int units = 0;
            if (t <= 0 || resident_plan(rep->f, K, th, 16, &p) != 0 || batch_units_possible(K, th, p.smem, &units) ||
                units < 1) {
                cudaGetLastError();
                continue;
            }
            const double score = t * (double)((n_fit + units - 1) / units);
            if (score < best_score) { best_score = score; b->K_b = K; b->threads_b = th; }
        }
    }
    return set_last_error(ISF_OK, "");
}

namespace {
// Units of the four classes (in: what each could keep resident alone; out: its share of the GPU
// by work: that share of its resident units, at least one, at most one per film; what the caps
// leave over goes to the others by their work).
void share_units(const std::vector<Item>& A, const std::vector<Item>& B, const std::vector<Item>& D,
                 const std::vector<Item>& E, int* ua, int* ub, int* ud, int* ue) {
    const std::vector<Item>* cls[4] = {&A, &B, &D, &E};
    int* u[4] = {ua, ub, ud, ue};
    double w[4] = {0.0, 0.0, 0.0, 0.0}, wt = 0.0;
    int maxu[4], cap[4];
    for (int x = 0; x < 4; ++x) {
        for (const Item& it : *cls[x]) w[x] += it.work;
        wt += w[x];
        maxu[x] = *u[x];
        cap[x] = std::min<int>(*u[x], (int)cls[x]->size());
    }
    if (wt <= 0.0) return;
    double used = 0.0, w_open = 0.0;     // fraction of the GPU taken; work of the classes below their cap
    for (int x = 0; x < 4; ++x) {
        if (cls[x]->empty() || maxu[x] < 1) continue;
        *u[x] = std::max(1, std::min(cap[x], (int)(w[x] / wt * maxu[x])));
        used += (double)*u[x] / maxu[x];
        if (*u[x] < cap[x]) w_open += w[x];
    }
    const double left = 1.0 - used;
    if (left > 0.0 && w_open > 0.0) {
        for (int x = 0; x < 4; ++x) {
            if (cls[x]->empty() || maxu[x] < 1 || *u[x] >= cap[x]) continue;
            *u[x] = std::min(cap[x], *u[x] + (int)(left * w[x] / w_open * maxu[x]));
        }
    }
}
}  // namespace

int isf_batch_run(isf_batch* b, void* cuda_stream) { return isf_batch_run_sweeps(b, -1, cuda_stream); }

int isf_batch_run_sweeps(isf_batch* b, int64_t max_sweeps, void* cuda_stream) {
    const isf::TraceRange trace("isf_batch_run_sweeps");
    if (!b) return fail(ISF_ERR_ARG, "batch is NULL");
    if (max_sweeps < -1 || max_sweeps == 0) return fail(ISF_ERR_ARG, "max_sweeps must be >= 1 or -1");
    int rc = ensure_streams(b);
    if (rc) return rc;
    CUDA_TRY(cudaSetDevice(b->device), "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (b->pending) {   // the staging buffer may still be read by the previous run's upload
        CUDA_TRY(cudaEventSynchronize(b->ev_done), "previous batch");
        b->pending = false;
    }
    const int ta = b->threads_a ? b->threads_a : kDefaultThreadsA;
    const int K = b->K_b ? b->K_b : kDefaultK;
    const int tb = b->threads_b ? b->threads_b : kDefaultThreadsB;
    std::vector<Item> A, B, D, E;
    std::vector<isf_lattice*> C;
    // a film in global memory takes one CTA (class D) only if its work is at most an even share
    // of the whole batch's work per such CTA; a larger one would finish last on its own CTA, so it
    // takes a cluster (class E)
    double total_work = 0.0;
    for (isf_lattice* L : b->films) {
        int64_t n = sweeps_remaining(L);
        if (max_sweeps > 0 && n > max_sweeps) n = max_sweeps;
        if (n > 0) total_work += (double)n * L->lay.L * L->lay.Rh * L->lay.Ch;
    }
    int d_units = 0;
    if (batch_global_units(kThreadsD, &d_units) || d_units < 1) {
        cudaGetLastError();
        d_units = 1;
    }
    const double d_limit = total_work / d_units;
    for (isf_lattice* L : b->films) {
        if (L->device != b->device) return fail(ISF_ERR_ARG, "all films of a batch must be on one device");
        int64_t n = sweeps_remaining(L);
        if (max_sweeps > 0 && n > max_sweeps) n = max_sweeps;
        if (n <= 0) continue;
        Item it{L, n, {}, (double)n * L->lay.L * L->lay.Rh * L->lay.Ch};
        // the queue kernels hold int8 films without periodic columns
        const bool queueable = !L->lay.packed && !(L->lay.flags & ISF_PERIODIC_X);
        const int64_t sites = (int64_t)L->lay.L * L->lay.R * L->lay.C;
        if (queueable && resident_plan(L->f, 1, ta, 16, &it.plan) == 0) A.push_back(it);
        else if (queueable && resident_plan(L->f, K, tb, 16, &it.plan) == 0) B.push_back(it);
        else if (sites <= kMaxSitesD && it.work <= d_limit) D.push_back(it);
        else if (sites <= kMaxSitesE) E.push_back(it);
        else C.push_back(L);
        cudaGetLastError();
    }
    // With films on the cluster global-memory kernel, the cluster-resident films join its queue:
    // launched first, that kernel holds the SMs a resident cluster would need, and it runs these
    // films about as fast per SM; a resident cluster kernel placed beside it only leaves some of
    // them on fewer SMs, from run to run (the bench's int8 batch: 10.7 s, or 13 s).
    if (!E.empty() && !B.empty()) {
        E.insert(E.end(), B.begin(), B.end());
        B.clear();
    }
    auto longest_first = [](const Item& x, const Item& y) { return x.work > y.work; };
    std::sort(A.begin(), A.end(), longest_first);
    std::sort(B.begin(), B.end(), longest_first);
    std::sort(D.begin(), D.end(), longest_first);
    std::sort(E.begin(), E.end(), longest_first);
    const int n_a = (int)A.size(), n_b = (int)B.size(), n_d = (int)D.size(), n_e = (int)E.size();
    rc = ensure_capacity(b, (size_t)n_a + n_b + 1);
    if (rc) return rc;
    rc = ensure_gcapacity(b, (size_t)n_d + n_e + 1);
    if (rc) return rc;
    for (int i = 0; i < n_d; ++i) b->h_gdesc[i] = sweep_args(D[i].L, D[i].nsweeps);
    for (int i = 0; i < n_e; ++i) b->h_gdesc[n_d + i] = sweep_args(E[i].L, E[i].nsweeps);
    int units_e = 0;
    if (n_e) {
        int e = batch_cluster_global_units(kKE, kThreadsE, &units_e);
        if (e || units_e < 1) return fail(ISF_ERR_CUDA, "cluster global-memory batch kernel cannot be resident");
    }
    int units_d = 0;
    if (n_d) {
        int e = batch_global_units(kThreadsD, &units_d);
        if (e || units_d < 1) return fail(ISF_ERR_CUDA, "global-memory batch kernel cannot be resident");
    }
    uint32_t smem_a = 0, smem_b = 0;
    for (int i = 0; i < n_a; ++i) {
        b->h_desc[i] = make_res_args(sweep_args(A[i].L, A[i].nsweeps), A[i].plan);
        smem_a = std::max(smem_a, A[i].plan.smem);
    }
    for (int i = 0; i < n_b; ++i) {
        b->h_desc[n_a + i] = make_res_args(sweep_args(B[i].L, B[i].nsweeps), B[i].plan);
        smem_b = std::max(smem_b, B[i].plan.smem);
    }
    int units_a = 0, units_b = 0;
    if (n_a) {
        int e = batch_units_possible(1, ta, smem_a, &units_a);
        if (e || units_a < 1) return fail(ISF_ERR_CUDA, "single-CTA batch kernel cannot be resident");
    }
    if (n_b) {
        int e = batch_units_possible(K, tb, smem_b, &units_b);
        if (e || units_b < 1) return fail(ISF_ERR_CUDA, "cluster batch kernel cannot be resident");
    }
    // The persistent queue kernels run at once.  Sized alone, each would take the whole GPU, and
    // the one the hardware places first would hold its SMs until its queue drains while the
    // others wait, so the batch's time would depend on the placement.  When all the work is on the
    // two global-memory classes (bit-packed, periodic-column or over-sized films: the same code
    // per site, so work is a fair measure of time), the GPU is shared in proportion to their work
    // and both kernels are resident from the start.  With resident int8 classes the same sharing
    // measured slower (27 s for the bench's int8 batch against 10.7), so those batches keep
    // whole-GPU grids, and the order of the launches (global-memory kernels, then the single-CTA
    // and the cluster kernel: the fastest order measured) is fixed, with or without graphs.
    if (A.empty() && B.empty()) share_units(A, B, D, E, &units_a, &units_b, &units_d, &units_e);
    units_a = std::min(units_a, n_a);
    units_b = std::min(units_b, n_b);
    units_d = std::min(units_d, n_d);
    units_e = std::min(units_e, n_e);
    if (n_a || n_b || n_d || n_e) {
        const int64_t sig[12] = {n_a, n_b, K, ta, tb, (int64_t)smem_a << 32 | smem_b, units_a, units_b, n_d, units_d,
                                 n_e, units_e};
        if (b->use_graph && std::memcmp(sig, b->gsig, sizeof sig)) {
            drop_graphs(b);
            std::memcpy(b->gsig, sig, sizeof sig);
        }
        rc = enqueue(b, s, n_a, n_b, K, ta, tb, smem_a, smem_b, units_a, units_b, n_d, units_d, n_e, units_e);
        if (rc) return rc;
        CUDA_TRY(cudaEventRecord(b->ev_done, s), "batch done");
        b->pending = true;
    }
    for (const Item& it : A) {
        advance_cursor(it.L, it.nsweeps);
        it.L->last = s;
        it.L->last_path = ISF_PATH_RESIDENT; it.L->last_ctas = 1; it.L->last_threads = ta;
    }
    for (const Item& it : B) {
        advance_cursor(it.L, it.nsweeps);
        it.L->last = s;
        it.L->last_path = ISF_PATH_RESIDENT; it.L->last_ctas = K; it.L->last_threads = tb;
    }
    for (const Item& it : D) {
        advance_cursor(it.L, it.nsweeps);
        it.L->last = s;
        it.L->last_path = ISF_PATH_GLOBAL; it.L->last_ctas = 1; it.L->last_threads = kThreadsD;
        it.L->last_sites = it.L->lay.packed ? 32 : 16;
    }
    for (const Item& it : E) {
        advance_cursor(it.L, it.nsweeps);
        it.L->last = s;
        it.L->last_path = ISF_PATH_GLOBAL; it.L->last_ctas = kKE; it.L->last_threads = kThreadsE;
        it.L->last_sites = it.L->lay.packed ? 32 : 16;
    }
    for (isf_lattice* L : C) {
        const int32_t saved = L->path;
        L->path = ISF_PATH_GLOBAL;
        int64_t n = sweeps_remaining(L);
        if (max_sweeps > 0 && n > max_sweeps) n = max_sweeps;
        rc = isf_run_sweeps(L, n, s);
        L->path = saved;
        if (rc) return rc;
    }
    b->n_a = n_a; b->n_b = n_b; b->n_c = (int)C.size(); b->n_d = n_d; b->n_e = n_e;
    b->units_a = units_a; b->units_b = units_b; b->units_d = units_d; b->units_e = units_e;
    b->used_K = K; b->used_ta = ta; b->used_tb = tb;
    return set_last_error(ISF_OK, "");
}

int isf_batch_info(isf_batch* b, int32_t* out12) {
    if (!b || !out12) return fail(ISF_ERR_ARG, "bad arguments");
    const int32_t v[12] = {b->n_a, b->n_b, b->n_c, b->units_a, b->units_b, b->used_K, b->used_ta, b->used_tb,
                           b->n_d, b->units_d, b->n_e, b->units_e};
    std::memcpy(out12, v, sizeof v);
    return ISF_OK;
}

int isf_batch_taken(isf_batch* b, int32_t* out2) {
    if (!b || !out2) return fail(ISF_ERR_ARG, "bad arguments");
    unsigned v[2] = {0u, 0u};
    if (b->d_next) {
        CUDA_TRY(cudaSetDevice(b->device), "cudaSetDevice");
        if (b->pending) CUDA_TRY(cudaEventSynchronize(b->ev_done), "batch sync");
        CUDA_TRY(cudaMemcpy(v, b->d_next + 4, sizeof v, cudaMemcpyDeviceToHost), "read counters");
    }
    out2[0] = (int32_t)v[0];
    out2[1] = (int32_t)v[1];
    return ISF_OK;
}

void isf_batch_destroy(isf_batch* b) {
    if (!b) return;
    if (b->sa) {
        cudaSetDevice(b->device);
        if (b->pending) cudaEventSynchronize(b->ev_done);
        drop_graphs(b);
        cudaStreamDestroy(b->sa);
        cudaStreamDestroy(b->sb);
        cudaStreamDestroy(b->sd);
        cudaStreamDestroy(b->se);
        cudaEventDestroy(b->ev_fork);
        cudaEventDestroy(b->ev_a);
        cudaEventDestroy(b->ev_b);
        cudaEventDestroy(b->ev_d);
        cudaEventDestroy(b->ev_e);
        cudaEventDestroy(b->ev_done);
        if (b->d_desc) cudaFree(b->d_desc);
        if (b->h_desc) cudaFreeHost(b->h_desc);
        if (b->d_gdesc) cudaFree(b->d_gdesc);
        if (b->h_gdesc) cudaFreeHost(b->h_gdesc);
        if (b->d_next) cudaFree(b->d_next);
    }
    delete b;
}

}  // extern "C"
