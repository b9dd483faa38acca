// capi.cpp — the C ABI (include/isingfilm.h): film lifetime, schedule, sweeps, read-out.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "capi_internal.h"

using namespace isf;

namespace isf {
// The item lists (and their per-entry records) are kept only for films whose word or byte
// offsets, neighbour offsets included, fit 32 bits.
bool lists_fit_32_bits(const Layout& lay) {
    return lay.packed ? (4 * lay.csw + 2 * lay.lsw) < ((int64_t)1 << 31)
                      : (4 * lay.cs8 + 2 * lay.ls8) < ((int64_t)1 << 31);
}
}  // namespace isf

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(ISF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define CUDA_TRY(expr, what)                         \
    do {                                             \
        cudaError_t e_ = (cudaError_t)(expr);        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

void free_schedule(isf_lattice* L) {
    if (L->sched) cudaFree(L->sched);
    L->sched = nullptr;
    L->d_tables = nullptr; L->d_eq = nullptr; L->d_tot = nullptr; L->d_recs = nullptr;
    L->nsteps = 0;
    L->T.clear(); L->h.clear(); L->eq.clear(); L->tot.clear();
    L->k = 0; L->pos = 0;
}

// Sync with the last stream this film ran on and surface any status word a kernel set.
int sync_film(isf_lattice* L) {
    CUDA_TRY(cudaSetDevice(L->device), "cudaSetDevice");
    CUDA_TRY(L->last ? cudaStreamSynchronize(L->last) : cudaDeviceSynchronize(), "synchronise");
    unsigned long long chk[4];
    CUDA_TRY((cudaError_t)read_checks(chk), "read checks");
    if (chk[0])
        return fail(ISF_ERR_STATE, "a resident kernel skipped an out-of-range access (check " + std::to_string(chk[0]) +
                                       ": " + std::to_string(chk[1]) + ", " + std::to_string(chk[2]) + ")");
    int err = 0, where = 0;
    CUDA_TRY(cudaMemcpy(&err, &L->st->error, sizeof(int), cudaMemcpyDeviceToHost), "read status");
    if (err) {
        CUDA_TRY(cudaMemcpy(&where, &L->st->error_where, sizeof(int), cudaMemcpyDeviceToHost), "read status");
        return fail(err, "a sweep kernel stopped: bounded wait expired (barrier " + std::to_string(where) + ")");
    }
    return ISF_OK;
}

int recompute(isf_lattice* L, cudaStream_t s, long long red[4]) {
    int e = launch_recompute(L->f, L->st, s);
    if (e) return cuda_fail((cudaError_t)e, "recompute kernel");
    CUDA_TRY(cudaMemcpyAsync(red, L->st->red, 4 * sizeof(long long), cudaMemcpyDeviceToHost, s), "read recompute");
    CUDA_TRY(cudaStreamSynchronize(s), "recompute sync");
    return ISF_OK;
}

// A slab's place in its whole film: counter rows, row offset, own colour-rows.
struct SlabWindow {
    int32_t cRh, cj0, jlo, jhi;
};

int create_common(const uint8_t* heights, int32_t rows, int32_t cols, int32_t layers, uint32_t flags,
                  uint64_t seed, int32_t init, void* cuda_stream, void* dev_buf, size_t dev_bytes,
                  isf_lattice** out, const SlabWindow* sw = nullptr) {
    if (!out) return fail(ISF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!heights) return fail(ISF_ERR_ARG, "heights is NULL");
    if (init < ISF_INIT_RANDOM || init > ISF_INIT_DOWN) return fail(ISF_ERR_ARG, "init must be ISF_INIT_*");
    Layout lay;
    const char* why = "";
    int rc = make_layout(rows, cols, layers, flags, &lay, &why);
    if (rc) return fail(rc, why);
    rc = check_colouring(lay, &why);
    if (rc) return fail(rc, why);
    const size_t n_px = (size_t)rows * (size_t)cols;
    for (size_t p = 0; p < n_px; ++p)
        if (heights[p] > layers) return fail(ISF_ERR_ARG, "a height exceeds the number of layers");

    isf_lattice* L = new (std::nothrow) isf_lattice();
    if (!L) return fail(ISF_ERR_OOM, "host allocation failed");
    L->lay = lay;
    L->seed = seed;
    L->init = init;
    L->heights.assign(heights, heights + n_px);
    cudaError_t e = cudaGetDevice(&L->device);
    if (e != cudaSuccess) { delete L; return cuda_fail(e, "cudaGetDevice"); }
    if (dev_buf) {
        if (dev_bytes < lay.total_bytes) { delete L; return fail(ISF_ERR_OOM, "caller buffer smaller than isf_lattice_bytes"); }
        if (reinterpret_cast<uintptr_t>(dev_buf) % 256) { delete L; return fail(ISF_ERR_ARG, "caller buffer must be 256-byte aligned"); }
        L->dev = static_cast<uint8_t*>(dev_buf);
    } else {
        e = cudaMalloc(&L->dev, lay.total_bytes);
        if (e != cudaSuccess) { delete L; cudaGetLastError(); return fail(ISF_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e)); }
        L->owns_dev = true;
    }
    DevFilm& f = L->f;
    f.R = rows; f.C = cols; f.L = layers;
    f.Rh = lay.Rh; f.Ch = lay.Ch; f.Qw = lay.Qw;
    f.flags = flags; f.packed = lay.packed ? 1 : 0;
    f.key0 = (uint32_t)seed; f.key1 = (uint32_t)(seed >> 32);
    f.P = lay.P; f.ls8 = lay.ls8; f.cs8 = lay.cs8; f.nck = (int32_t)lay.nck;
    f.Wp = lay.Wp; f.lsw = lay.lsw; f.csw = lay.csw; f.nw = (int32_t)lay.nw;
    if (lay.packed) {
        f.sp = reinterpret_cast<uint32_t*>(L->dev);
        f.op = f.sp + 4 * lay.csw;
    } else {
        f.s8 = L->dev;
    }
    f.heights = L->dev + lay.heights_off;
    fill_neighbour_classes(lay, &f);
    L->st = reinterpret_cast<FilmState*>(L->dev + lay.state_off);
    if (sw) {
        f.slab = 1;
        f.cRh = sw->cRh; f.cj0 = sw->cj0; f.jlo = sw->jlo; f.jhi = sw->jhi;
    }
    // item lists (with their per-entry records) for films whose indices and neighbour offsets
    // fit 32 bits; the kernels walk every item of the others
    f.narrow = lists_fit_32_bits(lay) ? 1 : 0;
    std::vector<uint32_t> items;
    if (f.narrow && build_word_items(lay, heights, items, f.nitems, &f.item_wbits, &f.item_jbits,
                                     sw ? sw->jlo : 0, sw ? sw->jhi : lay.Rh,
                                     (sw || !lay.packed) ? nullptr : &L->roff_h)) {
        f.items = reinterpret_cast<const uint32_t*>(L->dev + lay.items_off);
        f.item_cap = lay.items_cap;
    } else {
        L->roff_h.clear();
    }
    if (f.items) {
        f.ient = reinterpret_cast<const uint32_t*>(L->dev + lay.ient_off);
        if (lay.packed) f.ivq = reinterpret_cast<const uint32_t*>(L->dev + lay.ivq_off);
    }

    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    auto bail = [&](int code) { isf_lattice_destroy(L); return code; };
    e = cudaMemsetAsync(L->st, 0, sizeof(FilmState), s);
    if (e != cudaSuccess) return bail(cuda_fail(e, "memset state"));
    if (f.items) {
        // host vector stays alive until the stream synchronisation at the end of set-up
        e = cudaMemcpyAsync(L->dev + lay.items_off, items.data(), items.size() * sizeof(uint32_t),
                            cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return bail(cuda_fail(e, "copy word lists"));
    }
    if (!L->roff_h.empty()) {
        e = cudaMemcpyAsync(L->dev + lay.roff_off, L->roff_h.data(), L->roff_h.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return bail(cuda_fail(e, "copy word-list row offsets"));
    }
    e = cudaMemcpyAsync(L->dev + lay.heights_off, heights, n_px, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return bail(cuda_fail(e, "copy heights"));
    int ke = launch_init(f, init, s);
    if (ke) return bail(cuda_fail((cudaError_t)ke, "init kernel"));
    if (f.ient) {
        ke = launch_init_entries(f, s);
        if (ke) return bail(cuda_fail((cudaError_t)ke, "word-list entries kernel"));
    }

    long long red[4];
    rc = recompute(L, s, red);
    if (rc) return bail(rc);
    L->n_occ = red[2];
    L->n_bonds = red[3] / 2;
    long long mb[2] = {red[0], red[1] / 2};
    if (sw) {
        // a slab's running M, B count its own changes from zero; its share of the whole film's
        // M and 2B (over its own sites, neighbours in the halo included) is kept on the host
        L->slab_m0 = red[0];
        L->slab_b2 = red[1];
        mb[0] = 0;
        mb[1] = 0;
    }
    e = cudaMemcpyAsync(&L->st->M, mb, sizeof(mb), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bail(cuda_fail(e, "write state"));
    L->last = s;
    *out = L;
    g_err.clear();
    return ISF_OK;
}

}  // namespace

namespace isf {
// Last-error setter for the library's other translation units.
int set_last_error(int code, const char* msg) {
    g_err = msg;
    return code;
}

int64_t sweeps_remaining(const isf_lattice* L) {
    int64_t r = 0;
    for (int32_t k = L->k; k < L->nsteps; ++k) r += L->tot[k];
    return r - L->pos;
}

SweepArgs sweep_args(const isf_lattice* L, int64_t nsweeps) {
    SweepArgs a{};
    a.f = L->f;
    a.st = L->st;
    a.tables = L->d_tables;
    a.step_eq = L->d_eq;
    a.step_total = L->d_tot;
    a.recs = L->d_recs;
    a.trace = L->d_trace;
    a.trace_begin = L->trace_n;
    a.trace_cap = L->trace_cap;
    a.sweep0 = L->sweep;
    a.nsweeps = nsweeps;
    a.k0 = L->k;
    a.pos0 = L->pos;
    a.nsteps = L->nsteps;
    a.use_gate = L->use_gate ? 1 : 0;
    return a;
}

void advance_cursor(isf_lattice* L, int64_t nsweeps) {
    L->sweep += nsweeps;
    if (L->d_trace) L->trace_n = std::min<int64_t>(L->trace_cap, L->trace_n + nsweeps);
    int64_t left = nsweeps;
    while (left > 0) {
        const int64_t room = L->tot[L->k] - L->pos;
        if (left >= room) { left -= room; L->k += 1; L->pos = 0; }
        else { L->pos += (int32_t)left; left = 0; }
    }
}
}  // namespace isf

extern "C" {

const char* isf_last_error(void) { return g_err.c_str(); }

size_t isf_lattice_bytes(int32_t rows, int32_t cols, int32_t layers, uint32_t flags) {
    Layout lay;
    const char* why = "";
    if (make_layout(rows, cols, layers, flags, &lay, &why)) return 0;
    return lay.total_bytes;
}

int isf_lattice_create(const uint8_t* heights, int32_t rows, int32_t cols, int32_t layers, uint32_t flags,
                       uint64_t seed, int32_t init, void* cuda_stream, isf_lattice** out) {
    return create_common(heights, rows, cols, layers, flags, seed, init, cuda_stream, nullptr, 0, out);
}

int isf_lattice_create_in(const uint8_t* heights, int32_t rows, int32_t cols, int32_t layers, uint32_t flags,
                          uint64_t seed, int32_t init, void* cuda_stream, void* dev_buf, size_t dev_bytes,
                          isf_lattice** out) {
    if (!dev_buf) return fail(ISF_ERR_ARG, "dev_buf is NULL");
    return create_common(heights, rows, cols, layers, flags, seed, init, cuda_stream, dev_buf, dev_bytes, out);
}

int isf_lattice_create_slab(const uint8_t* heights, int32_t rows, int32_t cols, int32_t layers, uint32_t flags,
                            uint64_t seed, int32_t init, int32_t y0, int32_t y1, void* cuda_stream,
                            isf_lattice** out) {
    if (!out) return fail(ISF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!heights) return fail(ISF_ERR_ARG, "heights is NULL");
    Layout whole;
    const char* why = "";
    int rc = make_layout(rows, cols, layers, flags, &whole, &why);   // the whole film must be valid
    if (rc) return fail(rc, why);
    rc = check_colouring(whole, &why);
    if (rc) return fail(rc, why);
    const bool py = (flags & ISF_PERIODIC_Y) != 0;
    if (y0 < 0 || y1 > rows || y1 - y0 < 2 || (y0 & 1) || ((y1 & 1) && y1 != rows))
        return fail(ISF_ERR_ARG, "slab rows [y0, y1): 0 <= y0 < y1 <= rows, y0 even, y1 even or rows, at least 2 rows");
    // one halo row pair on each side (whole-film rows wrap when periodic in y)
    const int32_t ya = (y0 > 0 || py) ? y0 - 2 : y0;
    const int32_t yb = (y1 < rows || py) ? y1 + 2 : y1;
    const int32_t lr = yb - ya;
    std::vector<uint8_t> local((size_t)lr * cols);
    for (int32_t r = 0; r < lr; ++r) {
        const int32_t y = ((ya + r) % rows + rows) % rows;
        std::memcpy(&local[(size_t)r * cols], heights + (size_t)y * cols, (size_t)cols);
    }
    SlabWindow sw;
    sw.cRh = whole.Rh;
    sw.cj0 = ya / 2;                              // ya is even (possibly -2)
    sw.jlo = (y0 - ya) / 2;
    sw.jhi = (yb == y1) ? (lr + 1) / 2 : (y1 - ya) / 2;
    rc = create_common(local.data(), lr, cols, layers, flags & ~(uint32_t)ISF_PERIODIC_Y, seed, init, cuda_stream,
                       nullptr, 0, out, &sw);
    if (rc) return rc;
    (*out)->slab_y0 = y0; (*out)->slab_y1 = y1; (*out)->slab_ya = ya; (*out)->slab_rows = rows;
    return ISF_OK;
}

int isf_slab_info(isf_lattice* L, int32_t* out6, size_t* halo_bytes, int64_t* out3) {
    if (!L || !out6 || !halo_bytes || !out3) return fail(ISF_ERR_ARG, "bad arguments");
    if (!L->f.slab) return fail(ISF_ERR_STATE, "not a slab film");
    const int32_t v[6] = {L->slab_y0, L->slab_y1, L->slab_ya, L->lay.R, L->f.jlo, L->f.jhi};
    std::memcpy(out6, v, sizeof v);
    *halo_bytes = (size_t)L->lay.L * (L->lay.packed ? (size_t)L->lay.Wp * 4 : (size_t)L->lay.P);
    out3[0] = L->slab_m0;
    out3[1] = L->slab_b2;
    out3[2] = L->n_occ;
    return ISF_OK;
}

// Device address and pitch of colour-row j (local) of colour c, layer 0; layers follow at the
// returned pitch.  int8: the whole padded row; packed: the spin bit-plane row.
static void slab_row(const isf_lattice* L, int32_t c, int32_t j, uint8_t** p, size_t* width, size_t* pitch) {
    const Layout& lay = L->lay;
    if (lay.packed) {
        *p = reinterpret_cast<uint8_t*>(L->f.sp + (int64_t)c * lay.csw + lay.lsw + (int64_t)(j + 1) * lay.Wp);
        *width = (size_t)lay.Wp * 4;
        *pitch = (size_t)lay.lsw * 4;
    } else {
        *p = L->f.s8 + (int64_t)c * lay.cs8 + lay.ls8 + (int64_t)(j + 1) * lay.P;
        *width = (size_t)lay.P;
        *pitch = (size_t)lay.ls8;
    }
}

int isf_slab_export(isf_lattice* L, int32_t colour, int32_t side, void* dev_buf, void* cuda_stream) {
    if (!L || !dev_buf || colour < 0 || colour > 3 || (side != 0 && side != 1)) return fail(ISF_ERR_ARG, "bad arguments");
    if (!L->f.slab) return fail(ISF_ERR_STATE, "not a slab film");
    uint8_t* p;
    size_t w, pitch;
    slab_row(L, colour, side == 0 ? L->f.jlo : L->f.jhi - 1, &p, &w, &pitch);
    CUDA_TRY(cudaSetDevice(L->device), "cudaSetDevice");
    CUDA_TRY(cudaMemcpy2DAsync(dev_buf, w, p, pitch, w, (size_t)L->lay.L, cudaMemcpyDeviceToDevice,
                               static_cast<cudaStream_t>(cuda_stream)), "export halo rows");
    return ISF_OK;
}

int isf_slab_import(isf_lattice* L, int32_t colour, int32_t side, const void* dev_buf, void* cuda_stream) {
    if (!L || !dev_buf || colour < 0 || colour > 3 || (side != 0 && side != 1)) return fail(ISF_ERR_ARG, "bad arguments");
    if (!L->f.slab) return fail(ISF_ERR_STATE, "not a slab film");
    const int32_t j = side == 0 ? L->f.jlo - 1 : L->f.jhi;
    if (j < 0 || j >= L->lay.Rh) return fail(ISF_ERR_ARG, "this slab has no halo on that side (edge of an open film)");
    uint8_t* p;
    size_t w, pitch;
    slab_row(L, colour, j, &p, &w, &pitch);
    CUDA_TRY(cudaSetDevice(L->device), "cudaSetDevice");
    CUDA_TRY(cudaMemcpy2DAsync(p, pitch, dev_buf, w, w, (size_t)L->lay.L, cudaMemcpyDeviceToDevice,
                               static_cast<cudaStream_t>(cuda_stream)), "import halo rows");
    return ISF_OK;
}

int isf_run_pass(isf_lattice* L, int32_t colour, void* cuda_stream) {
    if (!L || colour < 0 || colour > 3) return fail(ISF_ERR_ARG, "bad arguments");
    if (!L->f.slab) return fail(ISF_ERR_STATE, "isf_run_pass is for slab films (whole films: isf_run_sweeps)");
    if (!L->nsteps) return fail(ISF_ERR_STATE, "no schedule set");
    if (colour != L->pass_next) return fail(ISF_ERR_STATE, "colour passes run in the order 0, 1, 2, 3");
    if (sweeps_remaining(L) < 1) return fail(ISF_ERR_SCHEDULE, "past the end of the schedule");
    CUDA_TRY(cudaSetDevice(L->device), "cudaSetDevice");
    SweepArgs a = sweep_args(L, 1);
    a.pass_plus1 = colour + 1;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int threads = L->threads ? std::min(L->threads, 512) : 256;
    int maxc = 0;
    int e = sweep_max_ctas_for(L->f, threads, &maxc);
    if (e) return cuda_fail((cudaError_t)e, "occupancy query");
    if (maxc < 1) return fail(ISF_ERR_CUDA, "sweep kernel cannot be resident with this block size");
    int ctas = L->ctas;
    if (ctas <= 0) ctas = (int)std::max<int64_t>(1, (sweep_items_per_pass(L->f) + threads - 1) / threads);
    if (ctas > maxc) ctas = maxc;
    e = launch_sweeps(a, ctas, threads, s);
    if (e) return cuda_fail((cudaError_t)e, "sweep kernel launch");
    L->last_path = ISF_PATH_GLOBAL; L->last_ctas = ctas; L->last_threads = threads;
    L->last_sites = L->lay.packed ? 32 : 16;
    L->last = s;
    if (colour == 3) {
        advance_cursor(L, 1);
        L->pass_next = 0;
    } else {
        L->pass_next = colour + 1;
    }
    return ISF_OK;
}

int isf_fold_series(int32_t nsteps, const double* T, const double* h, const int32_t* sweeps_eq,
                    const int32_t* sweeps_meas, double J, int64_t n_occ, const int64_t* M, const int64_t* B,
                    isf_step_obs* out) {
    if (nsteps < 1 || !T || !h || !sweeps_eq || !sweeps_meas || !M || !B || !out) return fail(ISF_ERR_ARG, "bad arguments");
    int64_t t = 0;
    for (int32_t k = 0; k < nsteps; ++k) {
        if (sweeps_eq[k] < 0 || sweeps_meas[k] < 0 || sweeps_eq[k] + (int64_t)sweeps_meas[k] < 1)
            return fail(ISF_ERR_SCHEDULE, "every step needs at least one sweep");
        StepRec r{};
        __int128 m2 = 0, b2 = 0, mb = 0;
        t += sweeps_eq[k];
        for (int32_t i = 0; i < sweeps_meas[k]; ++i, ++t) {
            const long long m = M[t], b = B[t];
            r.n_meas += 1;
            r.sumM += m;
            r.sumAbsM += m < 0 ? -m : m;
            r.sumB += b;
            m2 += (__int128)m * m;
            b2 += (__int128)b * b;
            mb += (__int128)m * b;
        }
        r.M_last = M[t - 1];
        r.B_last = B[t - 1];
        const unsigned __int128 um2 = (unsigned __int128)m2, ub2 = (unsigned __int128)b2, umb = (unsigned __int128)mb;
        r.sumM2[0] = (unsigned long long)um2; r.sumM2[1] = (unsigned long long)(um2 >> 64);
        r.sumB2[0] = (unsigned long long)ub2; r.sumB2[1] = (unsigned long long)(ub2 >> 64);
        r.sumMB[0] = (unsigned long long)umb; r.sumMB[1] = (unsigned long long)(umb >> 64);
        isf_step_obs& o = out[k];
        o.T = T[k]; o.h = h[k];
        o.M_last = r.M_last; o.B_last = r.B_last; o.n_meas = r.n_meas;
        o.sumM = r.sumM; o.sumAbsM = r.sumAbsM; o.sumB = r.sumB;
        std::memcpy(o.sumM2, r.sumM2, sizeof o.sumM2);
        std::memcpy(o.sumB2, r.sumB2, sizeof o.sumB2);
        std::memcpy(o.sumMB, r.sumMB, sizeof o.sumMB);
        double d[6];
        derive_record(r, T[k], h[k], J, n_occ, d);
        o.m = d[0]; o.abs_m = d[1]; o.e = d[2]; o.chi = d[3]; o.chi_abs = d[4]; o.C = d[5];
    }
    return ISF_OK;
}

void isf_lattice_destroy(isf_lattice* L) {
    if (!L) return;
    cudaSetDevice(L->device);
    if (L->last) cudaStreamSynchronize(L->last);
    else cudaDeviceSynchronize();
    free_schedule(L);
    if (L->d_trace) cudaFree(L->d_trace);
    if (L->owns_dev && L->dev) cudaFree(L->dev);
    delete L;
}

int isf_set_schedule(isf_lattice* L, int32_t nsteps, const double* T, const double* h,
                     const int32_t* sweeps_eq, const int32_t* sweeps_meas, double J, double h_s) {
    if (!L) return fail(ISF_ERR_ARG, "lattice is NULL");
    if (nsteps < 1) return fail(ISF_ERR_ARG, "nsteps must be >= 1");
    if (!T || !h || !sweeps_eq || !sweeps_meas) return fail(ISF_ERR_ARG, "schedule array is NULL");
    if (!std::isfinite(J) || !std::isfinite(h_s)) return fail(ISF_ERR_SCHEDULE, "J and h_s must be finite");
    for (int32_t k = 0; k < nsteps; ++k) {
        if (std::isnan(T[k]) || T[k] < 0.0) return fail(ISF_ERR_SCHEDULE, "T must be >= 0 (inf allowed)");
        if (!std::isfinite(h[k])) return fail(ISF_ERR_SCHEDULE, "h must be finite");
        if (sweeps_eq[k] < 0 || sweeps_meas[k] < 0) return fail(ISF_ERR_SCHEDULE, "sweep counts must be >= 0");
        if ((int64_t)sweeps_eq[k] + sweeps_meas[k] < 1) return fail(ISF_ERR_SCHEDULE, "every step needs at least one sweep");
        if ((int64_t)sweeps_eq[k] + sweeps_meas[k] > 0x7FFFFFFF) return fail(ISF_ERR_SCHEDULE, "too many sweeps in a step");
    }
    int rc = sync_film(L);
    if (rc) return rc;
    free_schedule(L);
    const size_t tb = align256((size_t)nsteps * kTableStride * 4);
    const size_t ib = align256((size_t)nsteps * 4);
    const size_t rb = align256((size_t)nsteps * sizeof(StepRec));
    cudaError_t e = cudaMalloc(&L->sched, tb + 2 * ib + rb);
    if (e != cudaSuccess) { cudaGetLastError(); L->sched = nullptr; return fail(ISF_ERR_OOM, "cudaMalloc schedule"); }
    L->d_tables = reinterpret_cast<uint32_t*>(L->sched);
    L->d_eq = reinterpret_cast<int32_t*>(L->sched + tb);
    L->d_tot = reinterpret_cast<int32_t*>(L->sched + tb + ib);
    L->d_recs = reinterpret_cast<StepRec*>(L->sched + tb + 2 * ib);
    std::vector<uint32_t> tables((size_t)nsteps * kTableStride);
    L->use_gate = false;
    for (int32_t k = 0; k < nsteps; ++k) {
        build_step_table(T[k], h[k], J, h_s, &tables[(size_t)k * kTableStride]);
        if (tables[(size_t)k * kTableStride + kGateSlot] != kAlways) L->use_gate = true;
    }
    L->T.assign(T, T + nsteps);
    L->h.assign(h, h + nsteps);
    L->eq.assign(sweeps_eq, sweeps_eq + nsteps);
    L->tot.resize(nsteps);
    for (int32_t k = 0; k < nsteps; ++k) L->tot[k] = sweeps_eq[k] + sweeps_meas[k];
    L->J = J;
    L->h_s = h_s;
    CUDA_TRY(cudaMemcpy(L->d_tables, tables.data(), tables.size() * 4, cudaMemcpyHostToDevice), "upload tables");
    CUDA_TRY(cudaMemcpy(L->d_eq, L->eq.data(), (size_t)nsteps * 4, cudaMemcpyHostToDevice), "upload schedule");
    CUDA_TRY(cudaMemcpy(L->d_tot, L->tot.data(), (size_t)nsteps * 4, cudaMemcpyHostToDevice), "upload schedule");
    CUDA_TRY(cudaMemset(L->d_recs, 0, (size_t)nsteps * sizeof(StepRec)), "clear records");
    // fresh step sums (M, B and the sweep counter carry on)
    CUDA_TRY(cudaMemset(&L->st->n_meas, 0, offsetof(FilmState, red) - offsetof(FilmState, n_meas)), "clear sums");
    L->nsteps = nsteps;
    L->k = 0;
    L->pos = 0;
    g_err.clear();
    return ISF_OK;
}

// Rows [part[g], part[g+1]) of each of the G CTAs of the row-slab kernel: contiguous, 1..cap
// rows each, cut where the running count of occupied words (all colours) is closest to an even
// share.  Returns the most rows of any CTA.
static int slab_partition(const Layout& lay, const std::vector<int32_t>& roff, int G, int cap,
                          std::vector<int32_t>& part) {
    const int Rh = lay.Rh;
    std::vector<int64_t> pre((size_t)Rh + 1, 0);
    for (int j = 0; j < Rh; ++j) {
        int64_t w = 0;
        for (int cz = 0; cz < 4 * lay.L; ++cz) {
            const int32_t* ro = roff.data() + (size_t)cz * (Rh + 1);
            w += ro[j + 1] - ro[j];
        }
        pre[j + 1] = pre[j] + w;
    }
    part.assign((size_t)G + 1, 0);
    int nrm = 0;
    for (int g = 0; g < G; ++g) {
        const int left = G - g - 1;                     // CTAs after this one
        const int lo = std::max(part[g] + 1, Rh - left * cap);
        const int hi = std::min(part[g] + cap, Rh - left);
        const double target = (double)pre[Rh] * (g + 1) / G;
        int best = lo;
        for (int e = lo; e <= hi; ++e)
            if (std::fabs((double)pre[e] - target) < std::fabs((double)pre[best] - target)) best = e;
        part[g + 1] = best;
        nrm = std::max(nrm, best - part[g]);
    }
    return nrm;
}

// Sweeps of a packed whole film by the row-slab kernel, in launches of at most kSeriesChunk
// sweeps, each followed by the fold of its per-sweep series.  *fits = false (and nothing
// launched) when the film or the requested shape does not fit the kernel.
static int run_slabs(isf_lattice* L, int64_t nsweeps, cudaStream_t s, bool* fits) {
    *fits = false;
    const Layout& lay = L->lay;
    if (!lay.packed || L->f.slab || !L->f.items || !L->f.ivq || L->roff_h.empty() || lay.L > kSlabMaxLayers)
        return ISF_OK;
    const int threads = L->threads ? L->threads : 512;
    if (threads % 32 || threads < 64 || threads > 512) return ISF_OK;
    int dev = 0, sms = 1, optin = 0;
    CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
    CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "device attribute");
    const int G = L->ctas > 0 ? L->ctas : std::min(sms, lay.slab_gmax);
    if (G < 1 || G > lay.slab_gmax) return ISF_OK;
    const uint32_t per_row = slab_smem_bytes(L->f, 1) - slab_smem_bytes(L->f, 0);
    const int64_t cap = ((int64_t)optin - kSlabStaticSmem - (int64_t)slab_smem_bytes(L->f, 0)) / per_row;
    if (cap < 1 || cap * G < lay.Rh) return ISF_OK;
    if (G != L->part_G) {
        // a new partition: the film's earlier launches (which read the old one) must be done
        int rc = sync_film(L);
        if (rc) return rc;
        L->part_nrm = slab_partition(lay, L->roff_h, G, (int)std::min<int64_t>(cap, lay.Rh), L->part_h);
        CUDA_TRY(cudaMemcpy(L->dev + lay.part_off, L->part_h.data(), L->part_h.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice), "copy row partition");
        L->part_G = G;
    }
    const uint32_t smem = slab_smem_bytes(L->f, L->part_nrm);
    int units = 0;
    int e = slab_units(threads, smem, &units);
    if (e) return cuda_fail((cudaError_t)e, "row-slab occupancy query");
    if (units < G) return ISF_OK;
    *fits = true;
    SlabArgs A{};
    A.part = reinterpret_cast<const int32_t*>(L->dev + lay.part_off);
    A.roff = reinterpret_cast<const int32_t*>(L->dev + lay.roff_off);
    A.xbuf = reinterpret_cast<uint32_t*>(L->dev + lay.xbuf_off);
    A.done = reinterpret_cast<unsigned*>(L->dev + lay.done_off);
    A.series = reinterpret_cast<unsigned long long*>(L->dev + lay.series_off);
    A.nrm = L->part_nrm;
    for (int64_t done = 0; done < nsweeps;) {
        const int64_t n = std::min<int64_t>(nsweeps - done, kSeriesChunk);
        A.s = sweep_args(L, n);
        e = launch_slabs(A, G, threads, smem, s);
        if (e) return cuda_fail((cudaError_t)e, "row-slab sweep kernel launch");
        e = launch_fold_series(A.s, A.series, s);
        if (e) return cuda_fail((cudaError_t)e, "series fold launch");
        advance_cursor(L, n);
        done += n;
    }
    L->last_path = ISF_PATH_SLABS; L->last_ctas = G; L->last_threads = threads; L->last_sites = 32;
    L->last = s;
    return ISF_OK;
}

// Automatic choice for packed whole films: the row-slab kernel when a colour pass has more words
// than one CTA of the word kernel takes (512) and at most eight CTAs' worth; else the word kernel
// on global memory.  Measured on fractal films of 6 layers (bench.py --sizes): with one word per
// thread the word kernel's sweep is its four grid barriers and one round of words, 13.5 to
// 13.7 us from 256^2 to 1536^2; the slab kernel's is 13.1 us at 256^2, equal at 384^2 and
// 15 to 27 us from 512^2 up, so it is kept only where the word kernel runs on a handful of CTAs.
static bool slabs_preferred(const isf_lattice* L) {
    if (!L->lay.packed || L->f.slab || !L->f.items || L->roff_h.empty() || L->lay.L > kSlabMaxLayers) return false;
    const int64_t words = sweep_items_per_pass(L->f);
    return words > 512 && words <= 8 * 512;
}

int isf_run_sweeps(isf_lattice* L, int64_t nsweeps, void* cuda_stream) {
    const isf::TraceRange trace("isf_run_sweeps");
    if (!L) return fail(ISF_ERR_ARG, "lattice is NULL");
    if (!L->nsteps) return fail(ISF_ERR_STATE, "no schedule set");
    if (L->f.slab) return fail(ISF_ERR_STATE, "a slab film advances by isf_run_pass, with halo exchanges between passes");
    const int64_t remaining = sweeps_remaining(L);
    if (nsweeps == -1) nsweeps = remaining;
    if (nsweeps < 0) return fail(ISF_ERR_ARG, "nsweeps must be >= 0 or -1");
    if (nsweeps > remaining) return fail(ISF_ERR_SCHEDULE, "past the end of the schedule");
    if (nsweeps == 0) return ISF_OK;
    CUDA_TRY(cudaSetDevice(L->device), "cudaSetDevice");
    const SweepArgs a = sweep_args(L, nsweeps);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (L->path == ISF_PATH_SLABS || (L->path == ISF_PATH_AUTO && slabs_preferred(L))) {
        bool fits = false;
        int rc = run_slabs(L, nsweeps, s, &fits);
        if (rc) return rc;
        if (fits) return ISF_OK;
        if (L->path == ISF_PATH_SLABS)
            return fail(ISF_ERR_ARG, "the row-slab path needs a packed whole film with word lists whose rows fit the CTAs' shared memory with this launch shape");
    }
    bool launched = false;
    if (L->path != ISF_PATH_GLOBAL && !L->lay.packed) {
        ResPlan plan;
        const bool forced = L->path == ISF_PATH_RESIDENT;
        if (resident_plan(L->f, L->ctas, L->threads, L->item_sites, &plan) == 0) {
            int e = launch_resident(a, plan, s);
            if (e) return cuda_fail((cudaError_t)e, "resident sweep kernel launch");
            launched = true;
            L->last_path = ISF_PATH_RESIDENT; L->last_ctas = plan.K; L->last_threads = plan.threads;
            L->last_sites = plan.item_sites;
        } else {
            cudaGetLastError();
            if (forced) return fail(ISF_ERR_ARG, "film does not fit one cluster's shared memory with this launch shape");
        }
    }
    if (!launched) {
        const bool listed = L->f.packed && L->f.items;
        int threads = L->threads ? std::min(L->threads, 512) : (listed ? 512 : 256);
        int maxc = 0;
        int e = sweep_max_ctas_for(L->f, threads, &maxc);
        if (e) return cuda_fail((cudaError_t)e, "occupancy query");
        if (maxc < 1) return fail(ISF_ERR_CUDA, "sweep kernel cannot be resident with this block size");
        int ctas = L->ctas;
        const int64_t items = sweep_items_per_pass(L->f);
        if (ctas <= 0 && listed) {
            // a whole number of CTAs per SM, the fewest that reach the smallest count of words
            // per thread (every thread then takes that count or one less)
            int dev = 0, sms = 1;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const int64_t one_each = (items + threads - 1) / threads;
            if (one_each <= sms) {
                ctas = (int)std::max<int64_t>(1, one_each);     // small film: one word per thread
            } else {
                int64_t best_k = -1;
                for (int g = sms; g <= maxc; g += sms) {
                    const int64_t k = (items + (int64_t)g * threads - 1) / ((int64_t)g * threads);
                    if (best_k < 0 || k < best_k) { best_k = k; ctas = g; }
                }
                if (ctas <= 0) ctas = maxc;
            }
        } else if (ctas <= 0) {
            int64_t want = (items + threads - 1) / threads;   // about one work item per thread
            ctas = (int)(want < 1 ? 1 : want);
        }
        if (ctas > maxc) ctas = maxc;
        e = launch_sweeps(a, ctas, threads, s);
        if (e) return cuda_fail((cudaError_t)e, "sweep kernel launch");
        L->last_path = ISF_PATH_GLOBAL; L->last_ctas = ctas; L->last_threads = threads;
        L->last_sites = L->lay.packed ? 32 : 16;
    }
    L->last = s;
    advance_cursor(L, nsweeps);
    return ISF_OK;
}

int isf_read_observables(isf_lattice* L, isf_step_obs* out, int32_t max, int32_t* n_out) {
    if (!L || !n_out || (max > 0 && !out)) return fail(ISF_ERR_ARG, "bad arguments");
    int rc = sync_film(L);
    if (rc) return rc;
    const int32_t n = std::min<int32_t>(L->k, std::max<int32_t>(max, 0));
    std::vector<StepRec> recs(n);
    if (n) CUDA_TRY(cudaMemcpy(recs.data(), L->d_recs, (size_t)n * sizeof(StepRec), cudaMemcpyDeviceToHost), "read records");
    for (int32_t k = 0; k < n; ++k) {
        const StepRec& r = recs[k];
        isf_step_obs& o = out[k];
        o.T = L->T[k]; o.h = L->h[k];
        o.M_last = r.M_last; o.B_last = r.B_last; o.n_meas = r.n_meas;
        o.sumM = r.sumM; o.sumAbsM = r.sumAbsM; o.sumB = r.sumB;
        for (int w = 0; w < 2; ++w) { o.sumM2[w] = r.sumM2[w]; o.sumB2[w] = r.sumB2[w]; o.sumMB[w] = r.sumMB[w]; }
        double d[6];
        derive_record(r, L->T[k], L->h[k], L->J, L->n_occ, d);
        o.m = d[0]; o.abs_m = d[1]; o.e = d[2]; o.chi = d[3]; o.chi_abs = d[4]; o.C = d[5];
    }
    *n_out = n;
    g_err.clear();
    return ISF_OK;
}

int isf_read_spins(isf_lattice* L, int8_t* host_out) {
    if (!L || !host_out) return fail(ISF_ERR_ARG, "bad arguments");
    int rc = sync_film(L);
    if (rc) return rc;
    const size_t n = (size_t)L->lay.R * L->lay.C * L->lay.L;
    int8_t* d = nullptr;
    CUDA_TRY(cudaMalloc(&d, n), "cudaMalloc read buffer");
    int e = launch_unpack(L->f, d, L->last);
    cudaError_t ce = (cudaError_t)e;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(host_out, d, n, cudaMemcpyDeviceToHost, L->last);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(L->last);
    cudaFree(d);
    if (ce != cudaSuccess) return cuda_fail(ce, "read spins");
    return ISF_OK;
}

int isf_read_surface_image(isf_lattice* L, uint8_t* host_out, int64_t* n_up) {
    if (!L || !host_out) return fail(ISF_ERR_ARG, "bad arguments");
    int rc = sync_film(L);
    if (rc) return rc;
    const size_t n = (size_t)L->lay.R * L->lay.C;
    uint8_t* d = nullptr;
    CUDA_TRY(cudaMalloc(&d, n + 256), "cudaMalloc image buffer");
    unsigned long long* up = reinterpret_cast<unsigned long long*>(d + ((n + 7) & ~size_t(7)));
    cudaError_t ce = cudaMemsetAsync(up, 0, sizeof(unsigned long long), L->last);
    if (ce == cudaSuccess) ce = (cudaError_t)launch_surface(L->f, d, up, L->last);
    unsigned long long nup = 0;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(host_out, d, n, cudaMemcpyDeviceToHost, L->last);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&nup, up, sizeof nup, cudaMemcpyDeviceToHost, L->last);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(L->last);
    cudaFree(d);
    if (ce != cudaSuccess) return cuda_fail(ce, "surface image");
    if (n_up) *n_up = (int64_t)nup;
    return ISF_OK;
}

int isf_surface_domains(isf_lattice* L, int64_t* out4) {
    if (!L || !out4) return fail(ISF_ERR_ARG, "bad arguments");
    if (L->lay.R * (int64_t)L->lay.C > 0x7FFFFFFFLL) return fail(ISF_ERR_ARG, "image too large for 32-bit labels");
    int rc = sync_film(L);
    if (rc) return rc;
    const size_t n = (size_t)L->lay.R * L->lay.C;
    const size_t img_bytes = (n + 255) & ~size_t(255);
    uint8_t* d = nullptr;
    CUDA_TRY(cudaMalloc(&d, img_bytes + 2 * n * sizeof(int) + 64), "cudaMalloc domain buffers");
    int* scratch = reinterpret_cast<int*>(d + img_bytes);
    unsigned long long* out = reinterpret_cast<unsigned long long*>(d + img_bytes + 2 * n * sizeof(int));
    int* bad = reinterpret_cast<int*>(out + 4);
    unsigned long long* up = out + 6;     // the image kernel's white count (unused here)
    unsigned long long h[4] = {0, 0, 0, 0};
    int hbad = 0;
    cudaError_t ce = cudaMemsetAsync(up, 0, sizeof(unsigned long long), L->last);
    if (ce == cudaSuccess) ce = (cudaError_t)launch_surface(L->f, d, up, L->last);
    if (ce == cudaSuccess) ce = (cudaError_t)launch_surface_domains(L->f, d, scratch, out, bad, L->last);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h, out, sizeof h, cudaMemcpyDeviceToHost, L->last);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hbad, bad, sizeof hbad, cudaMemcpyDeviceToHost, L->last);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(L->last);
    cudaFree(d);
    if (ce != cudaSuccess) return cuda_fail(ce, "surface domains");
    if (hbad) return fail(ISF_ERR_TIMEOUT, "domain labelling: a bounded union retry ran out");
    for (int i = 0; i < 4; ++i) out4[i] = (int64_t)h[i];
    return ISF_OK;
}

int isf_lattice_stats(isf_lattice* L, double* p, double* zbar, double* p_c) {
    if (!L) return fail(ISF_ERR_ARG, "lattice is NULL");
    const double sites = (double)L->lay.R * L->lay.C * L->lay.L;
    const double z = L->n_occ ? 2.0 * (double)L->n_bonds / (double)L->n_occ : 0.0;
    if (p) *p = (double)L->n_occ / sites;
    if (zbar) *zbar = z;
    if (p_c) *p_c = z > 0 ? 2.0 / z : INFINITY;
    return ISF_OK;
}

int isf_estimate_tc(const isf_step_obs* recs, int32_t n, double* T_c, int32_t* index) {
    if (!recs || n < 1 || !T_c) return fail(ISF_ERR_ARG, "bad arguments");
    // chi' = (<M^2> - <|M|>^2) / (N T) per step; N is the same for every step of a film, so the
    // largest (n sumM2 - sumAbsM^2) / (n^2 T), formed from the exact integer sums, marks it
    int best = -1;
    double best_score = 0.0;
    for (int32_t k = 0; k < n; ++k) {
        const isf_step_obs& r = recs[k];
        if (r.n_meas <= 0 || !(r.T > 0.0) || !std::isfinite(r.T)) continue;
        const __int128 nm = r.n_meas, sa = r.sumAbsM;
        const __int128 s2 = (__int128)(((unsigned __int128)r.sumM2[1] << 64) | r.sumM2[0]);
        const double nd = (double)r.n_meas;
        const double score = (double)(nm * s2 - sa * sa) / (nd * nd) / r.T;
        if (best < 0 || score > best_score) {
            best = k;
            best_score = score;
        }
    }
    if (best < 0) return fail(ISF_ERR_STATE, "no step with measured sweeps at a finite, positive temperature");
    *T_c = recs[best].T;
    if (index) *index = best;
    return set_last_error(ISF_OK, "");
}

int isf_write_spins(isf_lattice* L, const int8_t* host_in, int64_t sweep) {
    if (!L || !host_in || sweep < 0) return fail(ISF_ERR_ARG, "bad arguments");
    if (L->f.slab) return fail(ISF_ERR_STATE, "a slab film's spins come from its seed and the halo exchanges");
    const int R = L->lay.R, C = L->lay.C, Lz = L->lay.L;
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < R; ++y)
            for (int x = 0; x < C; ++x) {
                const int8_t v = host_in[((size_t)z * R + y) * C + x];
                const bool occ = z < L->heights[(size_t)y * C + x];
                if (occ ? (v != 1 && v != -1) : (v != 0)) return fail(ISF_ERR_ARG, "spins must be +-1 on occupied sites and 0 elsewhere");
            }
    int rc = sync_film(L);
    if (rc) return rc;
    const size_t n = (size_t)R * C * Lz;
    int8_t* d = nullptr;
    CUDA_TRY(cudaMalloc(&d, n), "cudaMalloc write buffer");
    cudaError_t ce = cudaMemcpyAsync(d, host_in, n, cudaMemcpyHostToDevice, L->last);
    if (ce == cudaSuccess) ce = (cudaError_t)launch_pack(L->f, d, L->last);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(L->last);
    cudaFree(d);
    if (ce != cudaSuccess) return cuda_fail(ce, "write spins");
    long long red[4];
    rc = recompute(L, L->last, red);
    if (rc) return rc;
    long long mb[2] = {red[0], red[1] / 2};
    CUDA_TRY(cudaMemcpy(&L->st->M, mb, sizeof(mb), cudaMemcpyHostToDevice), "write state");
    L->sweep = sweep;
    return ISF_OK;
}

int isf_lattice_info(isf_lattice* L, int64_t* n_occ, int64_t* n_bonds, double* zbar, int64_t* sweep) {
    if (!L) return fail(ISF_ERR_ARG, "lattice is NULL");
    if (n_occ) *n_occ = L->n_occ;
    if (n_bonds) *n_bonds = L->n_bonds;
    if (zbar) *zbar = L->n_occ ? 2.0 * (double)L->n_bonds / (double)L->n_occ : 0.0;
    if (sweep) *sweep = L->sweep;
    return ISF_OK;
}

int isf_read_state(isf_lattice* L, int64_t* M, int64_t* B, int32_t recompute_too, int64_t* M_full, int64_t* B_full) {
    if (!L) return fail(ISF_ERR_ARG, "lattice is NULL");
    int rc = sync_film(L);
    if (rc) return rc;
    long long mb[2];
    CUDA_TRY(cudaMemcpy(mb, &L->st->M, sizeof(mb), cudaMemcpyDeviceToHost), "read state");
    if (M) *M = mb[0];
    if (B) *B = mb[1];
    if (recompute_too) {
        long long red[4];
        rc = recompute(L, L->last, red);
        if (rc) return rc;
        if (M_full) *M_full = red[0];
        if (B_full) *B_full = red[1] / 2;
    }
    return ISF_OK;
}

int isf_enable_trace(isf_lattice* L, int64_t max_sweeps) {
    if (!L || max_sweeps < 0) return fail(ISF_ERR_ARG, "bad arguments");
    int rc = sync_film(L);
    if (rc) return rc;
    if (L->d_trace) cudaFree(L->d_trace);
    L->d_trace = nullptr;
    L->trace_cap = 0;
    L->trace_n = 0;
    if (max_sweeps == 0) return ISF_OK;
    cudaError_t e = cudaMalloc(&L->d_trace, (size_t)max_sweeps * 2 * sizeof(long long));
    if (e != cudaSuccess) { cudaGetLastError(); L->d_trace = nullptr; return fail(ISF_ERR_OOM, "cudaMalloc trace"); }
    L->trace_cap = max_sweeps;
    return ISF_OK;
}

int isf_read_trace(isf_lattice* L, int64_t* host_out, int64_t max_pairs, int64_t* n_out) {
    if (!L || !n_out || (max_pairs > 0 && !host_out)) return fail(ISF_ERR_ARG, "bad arguments");
    int rc = sync_film(L);
    if (rc) return rc;
    const int64_t n = std::min<int64_t>(L->trace_n, std::max<int64_t>(max_pairs, 0));
    if (n) CUDA_TRY(cudaMemcpy(host_out, L->d_trace, (size_t)n * 2 * sizeof(long long), cudaMemcpyDeviceToHost), "read trace");
    *n_out = n;
    return ISF_OK;
}

int isf_set_launch(isf_lattice* L, int32_t ctas, int32_t threads) {
    if (!L || ctas < 0) return fail(ISF_ERR_ARG, "bad arguments");
    if (threads != 0 && (threads % 32 || threads < 32 || threads > 1024))
        return fail(ISF_ERR_ARG, "threads must be 0 or a multiple of 32 in 32..1024");
    L->ctas = ctas;
    L->threads = threads;
    return ISF_OK;
}

int isf_set_item_sites(isf_lattice* L, int32_t sites) {
    if (!L) return fail(ISF_ERR_ARG, "lattice is NULL");
    if (sites != 0 && sites != 8 && sites != 16) return fail(ISF_ERR_ARG, "sites per work item must be 0, 8 or 16");
    L->item_sites = sites;
    return ISF_OK;
}

int isf_launch_item_sites(isf_lattice* L, int32_t* sites) {
    if (!L || !sites) return fail(ISF_ERR_ARG, "bad arguments");
    *sites = L->last_sites;
    return ISF_OK;
}

int isf_debug_item_lists(const uint8_t* heights, int32_t rows, int32_t cols, int32_t layers, uint32_t flags,
                         int32_t* n_out, uint32_t* out, int64_t cap, int32_t* bits_out) {
    if (!heights || !n_out || !out || !bits_out) return fail(ISF_ERR_ARG, "a pointer argument is NULL");
    Layout lay;
    const char* why = "";
    int rc = make_layout(rows, cols, layers, flags, &lay, &why);
    if (rc) return fail(rc, why);
    rc = check_colouring(lay, &why);
    if (rc) return fail(rc, why);
    if (lay.items_cap == 0) return fail(ISF_ERR_ARG, "this film has no item lists (periodic int8)");
    if (!lists_fit_32_bits(lay))
        return fail(ISF_ERR_ARG, "this film keeps no lists: its neighbour offsets do not fit 32 bits");
    if (cap < lay.items_cap) return fail(ISF_ERR_ARG, "cap is smaller than layers x colour rows x items per row");
    std::vector<uint32_t> items;
    int32_t n[4], wb = 0, jb = 0;
    if (!build_word_items(lay, heights, items, n, &wb, &jb, 0, lay.Rh))
        return fail(ISF_ERR_ARG, "the list entries' fields do not fit 32 bits");
    for (int c = 0; c < 4; ++c) {
        n_out[c] = n[c];
        std::memcpy(out + (size_t)c * cap, items.data() + (size_t)c * lay.items_cap, (size_t)n[c] * sizeof(uint32_t));
    }
    bits_out[0] = wb;
    bits_out[1] = jb;
    g_err.clear();
    return ISF_OK;
}

int isf_debug_slab_partition(const uint8_t* heights, int32_t rows, int32_t cols, int32_t layers, int32_t bands,
                             int32_t max_rows, int32_t* part_out) {
    if (!heights || !part_out) return fail(ISF_ERR_ARG, "a pointer argument is NULL");
    Layout lay;
    const char* why = "";
    int rc = make_layout(rows, cols, layers, ISF_PACKED, &lay, &why);
    if (rc) return fail(rc, why);
    if (!lists_fit_32_bits(lay))
        return fail(ISF_ERR_ARG, "the row-slab path needs word lists: this film's neighbour offsets do not fit 32 bits");
    if (bands < 1 || bands > lay.Rh || max_rows < 1 || (int64_t)max_rows * bands < lay.Rh)
        return fail(ISF_ERR_ARG, "need 1 <= bands <= colour rows and bands x max_rows >= colour rows");
    std::vector<uint32_t> items;
    std::vector<int32_t> roff, part;
    int32_t n[4], wb = 0, jb = 0;
    if (!build_word_items(lay, heights, items, n, &wb, &jb, 0, lay.Rh, &roff))
        return fail(ISF_ERR_ARG, "the list entries' fields do not fit 32 bits");
    slab_partition(lay, roff, bands, std::min(max_rows, lay.Rh), part);
    std::memcpy(part_out, part.data(), part.size() * sizeof(int32_t));
    g_err.clear();
    return ISF_OK;
}

int isf_debug_checks(uint64_t* out4) {
    if (!out4) return fail(ISF_ERR_ARG, "out is NULL");
    unsigned long long v[4];
    int e = read_checks(v);
    if (e) return cuda_fail((cudaError_t)e, "read checks");
    for (int i = 0; i < 4; ++i) out4[i] = v[i];
    return ISF_OK;
}

int isf_launch_info(isf_lattice* L, int32_t* path, int32_t* ctas, int32_t* threads) {
    if (!L) return fail(ISF_ERR_ARG, "lattice is NULL");
    if (path) *path = L->last_path;
    if (ctas) *ctas = L->last_ctas;
    if (threads) *threads = L->last_threads;
    return ISF_OK;
}

int isf_set_path(isf_lattice* L, int32_t path) {
    if (!L || path < ISF_PATH_AUTO || path > ISF_PATH_SLABS) return fail(ISF_ERR_ARG, "bad arguments");
    if (path == ISF_PATH_RESIDENT && L->lay.packed) return fail(ISF_ERR_ARG, "the resident path holds int8 films only");
    if (path == ISF_PATH_SLABS && (!L->lay.packed || L->f.slab || !L->f.items || L->lay.L > kSlabMaxLayers))
        return fail(ISF_ERR_ARG, "the row-slab path holds packed whole films of at most 16 layers with word lists only");
    L->path = path;
    return ISF_OK;
}

int isf_save(isf_lattice* L, const char* path) {
    if (!L || !path) return fail(ISF_ERR_ARG, "bad arguments");
    if (L->f.slab) return fail(ISF_ERR_STATE, "slab films are saved as the whole film they belong to");
    const size_t n = (size_t)L->lay.R * L->lay.C * L->lay.L;
    std::vector<int8_t> spins(n);
    int rc = isf_read_spins(L, spins.data());
    if (rc) return rc;
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(ISF_ERR_ARG, std::string("cannot open ") + path);
    const char magic[8] = {'I', 'S', 'F', 'I', 'L', 'M', '0', '1'};
    int32_t hdr[5] = {L->lay.R, L->lay.C, L->lay.L, (int32_t)L->lay.flags, L->init};
    int64_t tail[2] = {(int64_t)L->seed, L->sweep};
    bool ok = std::fwrite(magic, 1, 8, fp) == 8 && std::fwrite(hdr, 4, 5, fp) == 5 &&
              std::fwrite(tail, 8, 2, fp) == 2 &&
              std::fwrite(L->heights.data(), 1, L->heights.size(), fp) == L->heights.size() &&
              std::fwrite(spins.data(), 1, n, fp) == n;
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) return fail(ISF_ERR_ARG, "write failed");
    return ISF_OK;
}

int isf_load(const char* path, void* cuda_stream, isf_lattice** out) {
    if (!path || !out) return fail(ISF_ERR_ARG, "bad arguments");
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(ISF_ERR_ARG, std::string("cannot open ") + path);
    char magic[8];
    int32_t hdr[5];
    int64_t tail[2];
    bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, "ISFILM01", 8) == 0 &&
              std::fread(hdr, 4, 5, fp) == 5 && std::fread(tail, 8, 2, fp) == 2;
    if (!ok || hdr[0] < 1 || hdr[1] < 1 || hdr[2] < 1 || hdr[0] > 65536 || hdr[1] > 65536 || hdr[2] > 255) {
        std::fclose(fp);
        return fail(ISF_ERR_ARG, "not a film file");
    }
    const size_t npx = (size_t)hdr[0] * hdr[1], n = npx * hdr[2];
    std::vector<uint8_t> H(npx);
    std::vector<int8_t> S(n);
    ok = std::fread(H.data(), 1, npx, fp) == npx && std::fread(S.data(), 1, n, fp) == n;
    std::fclose(fp);
    if (!ok) return fail(ISF_ERR_ARG, "truncated film file");
    isf_lattice* L = nullptr;
    int rc = isf_lattice_create(H.data(), hdr[0], hdr[1], hdr[2], (uint32_t)hdr[3], (uint64_t)tail[0], hdr[4],
                                cuda_stream, &L);
    if (rc) return rc;
    rc = isf_write_spins(L, S.data(), tail[1]);
    if (rc) { isf_lattice_destroy(L); return rc; }
    *out = L;
    return ISF_OK;
}

int isf_debug_wait_timeout(int32_t ctas, int32_t* status_out, int32_t* where_out) {
    if (ctas < 2 || !status_out || !where_out) return fail(ISF_ERR_ARG, "bad arguments");
    int status = 0, where = 0;
    const cudaError_t e = (cudaError_t)wait_probe(ctas, &status, &where);
    if (e == cudaErrorInvalidValue) return fail(ISF_ERR_ARG, "more CTAs than can be co-resident");
    if (e != cudaSuccess) return cuda_fail(e, "wait probe");
    *status_out = status;
    *where_out = where;
    return ISF_OK;
}

int isf_philox_blocks(uint64_t seed, uint32_t stream, uint64_t sweep, uint32_t q0, int64_t nblocks,
                      uint32_t* host_out) {
    if (nblocks < 0 || (nblocks > 0 && !host_out)) return fail(ISF_ERR_ARG, "bad arguments");
    if (nblocks == 0) return ISF_OK;
    uint32_t* d = nullptr;
    CUDA_TRY(cudaMalloc(&d, (size_t)nblocks * 16), "cudaMalloc");
    cudaError_t e = (cudaError_t)launch_philox_blocks(seed, stream, sweep, q0, nblocks, d, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(host_out, d, (size_t)nblocks * 16, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "philox blocks");
    return ISF_OK;
}

}  // extern "C"
