// noalloc.cu — isf_run_noalloc: a whole schedule on one small film without allocating any
// memory, for callers that are not allowed to call cudaMalloc / cudaFree.
//
// Who needs it: code that runs inside a process whose device memory is owned by someone else's
// pool (a framework allocator that has reserved the free memory, so a foreign cudaMalloc fails
// or fragments it), latency-bound loops where cudaMalloc/cudaFree would synchronise the device
// and stall unrelated streams, and deployments that forbid dynamic allocation after start-up.
//
// How: the film layout, its running state, the threshold tables and the step records are
// carved out of one file-scope device array of ISF_NOALLOC_MAX_BYTES, which every GPU that
// loads the library holds until the process exits.  The kernels are the library's own
// (init, recompute, sweep, unpack), given addresses inside that array.  In host code the array's
// name is only a host-side stand-in, so its device address is fetched with cudaGetSymbolAddress
// once per device (with that device current) on the first call there and kept for the process
// (a cudaDeviceReset would make it stale; the library is not to be used across one).  Every call
// synchronises its stream and stages through host stack buffers, so no call may be made while a
// stream is being captured.  All calls share the array and each call clears what must start at
// zero; two calls whose work overlaps on the GPU (on different streams or host threads) race on
// it and must not be issued.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "isf_internal.h"
#include "../../include/isingfilm.h"

namespace isf {
int set_last_error(int code, const char* msg);   // capi.cpp
}

using namespace isf;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[ISF_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

inline size_t round256(size_t v) { return (v + 255) & ~size_t(255); }

int scratch_on(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return set_last_error(ISF_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return set_last_error(ISF_ERR_CUDA, cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[dev];
    return ISF_OK;
}

int cuda_err(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return ISF_OK;
    char buf[200];
    std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return set_last_error(ISF_ERR_CUDA, buf);
}

}  // namespace

extern "C" int isf_run_noalloc(const uint8_t* heights, int32_t rows, int32_t cols, int32_t layers, uint32_t flags,
                               uint64_t seed, int32_t init, int32_t nsteps, const double* T, const double* h,
                               const int32_t* sweeps_eq, const int32_t* sweeps_meas, double J, double h_s,
                               int8_t* dev_spins_out, isf_step_obs* obs_out, void* cuda_stream) {
    // ---- arguments (all on the host, before any device work) ----
    if (!heights || !T || !h || !sweeps_eq || !sweeps_meas || !dev_spins_out || !obs_out)
        return set_last_error(ISF_ERR_ARG, "isf_run_noalloc: a pointer argument is NULL");
    if (init < ISF_INIT_RANDOM || init > ISF_INIT_DOWN) return set_last_error(ISF_ERR_ARG, "init must be ISF_INIT_*");
    if (nsteps < 1) return set_last_error(ISF_ERR_ARG, "nsteps must be >= 1");
    Layout lay;
    const char* why = "";
    int rc = make_layout(rows, cols, layers, flags, &lay, &why);
    if (rc) return set_last_error(rc, why);
    rc = check_colouring(lay, &why);
    if (rc) return set_last_error(rc, why);
    for (size_t p = 0; p < (size_t)rows * (size_t)cols; ++p)
        if (heights[p] > layers) return set_last_error(ISF_ERR_ARG, "a height exceeds the number of layers");
    if (!std::isfinite(J) || !std::isfinite(h_s)) return set_last_error(ISF_ERR_SCHEDULE, "J and h_s must be finite");
    bool use_gate = false;
    for (int32_t k = 0; k < nsteps; ++k) {
        if (std::isnan(T[k]) || T[k] < 0.0) return set_last_error(ISF_ERR_SCHEDULE, "T must be >= 0 (inf allowed)");
        if (!std::isfinite(h[k])) return set_last_error(ISF_ERR_SCHEDULE, "h must be finite");
        if (sweeps_eq[k] < 0 || sweeps_meas[k] < 0) return set_last_error(ISF_ERR_SCHEDULE, "sweep counts must be >= 0");
        const int64_t tot = (int64_t)sweeps_eq[k] + sweeps_meas[k];
        if (tot < 1 || tot > 0x7FFFFFFF) return set_last_error(ISF_ERR_SCHEDULE, "every step needs 1 .. 2^31-1 sweeps");
    }
    // ---- where everything goes inside the fixed array ----
    const size_t tab_off = round256(lay.total_bytes);
    const size_t eq_off = round256(tab_off + (size_t)nsteps * kTableStride * 4);
    const size_t tot_off = round256(eq_off + (size_t)nsteps * 4);
    const size_t rec_off = round256(tot_off + (size_t)nsteps * 4);
    const size_t need = round256(rec_off + (size_t)nsteps * sizeof(StepRec));
    if (need > (size_t)ISF_NOALLOC_MAX_BYTES) {
        char buf[200];
        std::snprintf(buf, sizeof buf,
                      "isf_run_noalloc: this film and schedule need %zu bytes of scratch; the fixed array holds %zu",
                      need, (size_t)ISF_NOALLOC_MAX_BYTES);
        return set_last_error(ISF_ERR_ARG, buf);
    }
    int dev = 0;
    if ((rc = cuda_err(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    unsigned char* base = nullptr;
    if ((rc = scratch_on(dev, &base))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    // ---- the film, as isf_lattice_create lays it out, inside the array ----
    DevFilm f{};
    f.R = rows; f.C = cols; f.L = layers;
    f.Rh = lay.Rh; f.Ch = lay.Ch; f.Qw = lay.Qw;
    f.flags = flags; f.packed = lay.packed ? 1 : 0;
    f.key0 = (uint32_t)seed; f.key1 = (uint32_t)(seed >> 32);
    f.P = lay.P; f.ls8 = lay.ls8; f.cs8 = lay.cs8; f.nck = (int32_t)lay.nck;
    f.Wp = lay.Wp; f.lsw = lay.lsw; f.csw = lay.csw; f.nw = (int32_t)lay.nw;
    if (lay.packed) {
        f.sp = reinterpret_cast<uint32_t*>(base);
        f.op = f.sp + 4 * lay.csw;
    } else {
        f.s8 = base;
    }
    f.heights = base + lay.heights_off;
    fill_neighbour_classes(lay, &f);
    FilmState* st = reinterpret_cast<FilmState*>(base + lay.state_off);
    uint32_t* d_tab = reinterpret_cast<uint32_t*>(base + tab_off);
    int32_t* d_eq = reinterpret_cast<int32_t*>(base + eq_off);
    int32_t* d_tot = reinterpret_cast<int32_t*>(base + tot_off);
    StepRec* d_rec = reinterpret_cast<StepRec*>(base + rec_off);

    // the previous call's contents stay in the array: clear the state block and the records
    if ((rc = cuda_err(cudaMemsetAsync(st, 0, sizeof(FilmState), s), "clear state"))) return rc;
    if ((rc = cuda_err(cudaMemsetAsync(d_rec, 0, (size_t)nsteps * sizeof(StepRec), s), "clear records"))) return rc;
    if ((rc = cuda_err(cudaMemcpyAsync(base + lay.heights_off, heights, (size_t)rows * cols, cudaMemcpyHostToDevice, s),
                       "copy heights"))) return rc;
    if ((rc = cuda_err((cudaError_t)launch_init(f, init, s), "init kernel"))) return rc;
    if ((rc = cuda_err((cudaError_t)launch_recompute(f, st, s), "recompute kernel"))) return rc;
    long long red[4];
    if ((rc = cuda_err(cudaMemcpyAsync(red, st->red, sizeof red, cudaMemcpyDeviceToHost, s), "read counts"))) return rc;
    if ((rc = cuda_err(cudaStreamSynchronize(s), "synchronise"))) return rc;
    const long long n_occ = red[2];
    const long long mb[2] = {red[0], red[1] / 2};
    if ((rc = cuda_err(cudaMemcpyAsync(&st->M, mb, sizeof mb, cudaMemcpyHostToDevice, s), "write state"))) return rc;

    // tables and step lengths, a chunk of steps at a time through stack buffers
    constexpr int kChunk = 32;
    uint32_t tab[kChunk * kTableStride];
    int32_t eqc[kChunk], totc[kChunk];
    int64_t total = 0;
    for (int32_t k0 = 0; k0 < nsteps; k0 += kChunk) {
        const int32_t n = nsteps - k0 < kChunk ? nsteps - k0 : kChunk;
        for (int32_t i = 0; i < n; ++i) {
            const int32_t k = k0 + i;
            build_step_table(T[k], h[k], J, h_s, &tab[(size_t)i * kTableStride]);
            if (tab[(size_t)i * kTableStride + kGateSlot] != kAlways) use_gate = true;
            eqc[i] = sweeps_eq[k];
            totc[i] = sweeps_eq[k] + sweeps_meas[k];
            total += totc[i];
        }
        if ((rc = cuda_err(cudaMemcpyAsync(d_tab + (size_t)k0 * kTableStride, tab, (size_t)n * kTableStride * 4,
                                           cudaMemcpyHostToDevice, s), "copy tables"))) return rc;
        if ((rc = cuda_err(cudaMemcpyAsync(d_eq + k0, eqc, (size_t)n * 4, cudaMemcpyHostToDevice, s), "copy schedule"))) return rc;
        if ((rc = cuda_err(cudaMemcpyAsync(d_tot + k0, totc, (size_t)n * 4, cudaMemcpyHostToDevice, s), "copy schedule"))) return rc;
        if ((rc = cuda_err(cudaStreamSynchronize(s), "synchronise"))) return rc;   // stack buffers reused next
    }

    // ---- the sweeps ----
    SweepArgs a{};
    a.f = f;
    a.st = st;
    a.tables = d_tab;
    a.step_eq = d_eq;
    a.step_total = d_tot;
    a.recs = d_rec;
    a.sweep0 = 0;
    a.nsweeps = total;
    a.k0 = 0;
    a.pos0 = 0;
    a.nsteps = nsteps;
    a.use_gate = use_gate ? 1 : 0;
    const int threads = 256;
    int maxc = 0;
    if ((rc = cuda_err((cudaError_t)sweep_max_ctas_for(f, threads, &maxc), "occupancy query"))) return rc;
    if (maxc < 1) return set_last_error(ISF_ERR_CUDA, "sweep kernel cannot be resident");
    const int64_t items = sweep_items_per_pass(f);
    int64_t ctas = (items + threads - 1) / threads;
    if (ctas < 1) ctas = 1;
    if (ctas > maxc) ctas = maxc;
    if ((rc = cuda_err((cudaError_t)launch_sweeps(a, (int)ctas, threads, s), "sweep kernel launch"))) return rc;

    // ---- outputs: spins to the caller's device buffer, records to the caller's host array ----
    if ((rc = cuda_err((cudaError_t)launch_unpack(f, dev_spins_out, s), "unpack kernel"))) return rc;
    int err = 0;
    if ((rc = cuda_err(cudaMemcpyAsync(&err, &st->error, sizeof err, cudaMemcpyDeviceToHost, s), "read status"))) return rc;
    if ((rc = cuda_err(cudaStreamSynchronize(s), "synchronise"))) return rc;
    if (err) return set_last_error(err, "a sweep kernel stopped: bounded wait expired");
    StepRec rec[kChunk];
    for (int32_t k0 = 0; k0 < nsteps; k0 += kChunk) {
        const int32_t n = nsteps - k0 < kChunk ? nsteps - k0 : kChunk;
        if ((rc = cuda_err(cudaMemcpyAsync(rec, d_rec + k0, (size_t)n * sizeof(StepRec), cudaMemcpyDeviceToHost, s),
                           "read records"))) return rc;
        if ((rc = cuda_err(cudaStreamSynchronize(s), "synchronise"))) return rc;
        for (int32_t i = 0; i < n; ++i) {
            const int32_t k = k0 + i;
            const StepRec& r = rec[i];
            isf_step_obs& o = obs_out[k];
            o.T = T[k]; o.h = h[k];
            o.M_last = r.M_last; o.B_last = r.B_last; o.n_meas = r.n_meas;
            o.sumM = r.sumM; o.sumAbsM = r.sumAbsM; o.sumB = r.sumB;
            for (int w = 0; w < 2; ++w) { o.sumM2[w] = r.sumM2[w]; o.sumB2[w] = r.sumB2[w]; o.sumMB[w] = r.sumMB[w]; }
            double d[6];
            derive_record(r, T[k], h[k], J, n_occ, d);
            o.m = d[0]; o.abs_m = d[1]; o.e = d[2]; o.chi = d[3]; o.chi_abs = d[4]; o.C = d[5];
        }
    }
    return set_last_error(ISF_OK, "");
}
