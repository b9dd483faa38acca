// kernels_sweep.cu — the hot path: Metropolis colour passes (Eq. 8, items 1-3 of Sec. 5; the
// Eq. 9 gate of items 4-5 when a switching field is set) over the four conflict-free colours
// of the "checkerboard decomposition" (Sec. 3, Fig. 1), stepped through the temperature /
// field schedule with the state kept on the device.
//
// One persistent launch runs any number of sweeps.  Its CTAs split every colour pass between
// them and meet at a grid barrier between passes (cooperative launch, bounded spin: on
// expiry the kernel records ISF_ERR_TIMEOUT and returns).  Every attempt's random word is
// Philox(seed; site block, sweep, stream), so the result does not depend on the launch shape.
//
// Per accepted flip of spin s with neighbour sum n: dM = -2s, dB = -2 s n (B = sum over bonds
// of S S').  Threads accumulate, CTAs reduce, one atomic per CTA per sweep; after the sweep's
// last barrier CTA 0 folds the deltas into M and B and into the step's exact sums.
#include <cuda_runtime.h>

#include <algorithm>

#include "grid_sync.cuh"

namespace isf {

namespace {

enum { MODE_INT8 = 0, MODE_GENERIC = 1, MODE_PACKED = 2 };
constexpr int kBlock = 512;      // largest CTA of the global kernel (<= 128 registers per thread)
// ---- int8 layout, open boundaries: one thread per 16-site chunk of a colour row ------------
// The chunk at byte offset `base` of colour c (layer parity zp), Philox counter q0.
template <bool GATE>
__device__ __forceinline__ void chunk_int8_at(const DevFilm& f, int c, int zp, int64_t base, uint32_t q0,
                                              unsigned long long sweep, const uint32_t* tab, uint32_t gthr, int& dM,
                                              int& dB, bool neg) {
    const NbrClass& nc = f.nb[c][zp];
    uint8_t* own = f.s8 + base;
    const uint8_t* nbp[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) nbp[k] = own + nc.off[k];
    update_chunk16<GATE>(own, nbp, nc.sgn, q0, sweep, tab, gthr, f.key0, f.key1, 0, f.Ch, dM, dB, neg);
}
template <bool GATE>
__device__ __forceinline__ void chunk_int8(const DevFilm& f, int c, int z, int j, int ck,
                                           unsigned long long sweep, const uint32_t* tab,
                                           uint32_t gthr, int& dM, int& dB, bool neg) {
    chunk_int8_at<GATE>(f, c, z & 1, addr8(f, c, z, j, 16 * ck), block_counter(f, c, z, j, 16 * ck), sweep, tab, gthr,
                        dM, dB, neg);
}

// ---- int8 layout, any boundary (periodic wraps): one thread per 4-site Philox block --------
template <bool GATE>
__device__ __forceinline__ void block_generic(const DevFilm& f, int c, int z, int j, int blk,
                                              unsigned long long sweep, const uint32_t* tab,
                                              uint32_t gthr, int& dM, int& dB) {
    const int zp = z & 1, px = (c & 1) ^ zp, py = ((c >> 1) & 1) ^ zp;
    const int y = 2 * j + py;
    if (y >= f.R) return;
    uint32_t thr[4], idx[4];
    int64_t ad[4];
    bool need = false;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int i = 4 * blk + b, x = 2 * i + px;
        thr[b] = 0;
        idx[b] = 0;
        ad[b] = 0;
        if (i >= f.Ch || x >= f.C) continue;
        ad[b] = addr8(f, c, z, j, i);
        const uint32_t sb = f.s8[ad[b]];
        if (sb == 1u) continue;
        int n = 0;
        for (int k = 0; k < 12; ++k) {
            int xa, ya, za;
            if (neighbour_of(f, x, y, z, k, xa, ya, za)) n += site_spin(f, xa, ya, za);
        }
        idx[b] = (sb << 5) | (uint32_t)(n + 12);
        thr[b] = tab[idx[b]];
        need |= needs_word(thr[b]);
    }
    const uint32_t q = block_counter(f, c, z, j, 4 * blk);
    uint4 u = make_uint4(0, 0, 0, 0);
    if (need) u = philox10(make_uint4(q, (uint32_t)sweep, (uint32_t)(sweep >> 32), 0u), f.key0, f.key1);
    uint32_t lanes = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
        if (metropolis_accept(word_of(u, b), thr[b])) lanes |= 1u << b;
    if (GATE) lanes = gate_block(lanes, gthr, q, sweep, f.key0, f.key1);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        if (!(lanes & (1u << b))) continue;
        const int s = (idx[b] & 64u) ? 1 : -1;
        const int n = (int)(idx[b] & 31u) - 12;
        dM -= 2 * s;
        dB -= 2 * s * n;
        f.s8[ad[b]] = (uint8_t)(2 - (int)(idx[b] >> 5));
    }
}

// The bit-sliced count of vacant neighbours from the 12 neighbour occupancy words (for words
// that have no precomputed entry).
template <bool NARROW>
__device__ __forceinline__ void packed_vacancies(const DevFilm& f, const NbrClass& nc, int64_t base, uint32_t V[4]) {
    const uint32_t* opb = f.op + base;
    auto off = [&](int k) -> int64_t { return NARROW ? (int64_t)(int32_t)nc.off[k] : nc.off[k]; };
    uint32_t vac[12];
#pragma unroll
    for (int k = 0; k < 9; ++k) vac[k] = ~opb[off(k)];
    if (nc.sgn < 0) {
#pragma unroll
        for (int k = 9; k < 12; ++k) vac[k] = ~__funnelshift_l(opb[off(k) - 1], opb[off(k)], 1);
    } else {
#pragma unroll
        for (int k = 9; k < 12; ++k) vac[k] = ~__funnelshift_r(opb[off(k)], opb[off(k) + 1], 1);
    }
    popcount12(vac, V[0], V[1], V[2], V[3]);
}

// One packed word at word index `base` of colour c (layer parity zp), Philox counter q0.  vq: its
// precomputed vacant-neighbour count (VQ), else counted from the occupancy words.  sflags: the
// step's table flags (kFlagAlwaysDraw, kFlagNoNever).
template <bool GATE, bool NARROW, bool VQ>
__device__ __forceinline__ void word_packed_at(const DevFilm& f, int c, int zp, int64_t base, uint32_t q0,
                                               const uint4* vq, unsigned long long sweep, const uint32_t* tab,
                                               uint32_t gthr, uint32_t sflags, int& dM, int& dB,
                                               const uint4 (&pre)[4], bool use_pre) {
    const bool always_draw = (sflags & kFlagAlwaysDraw) != 0;
    const NbrClass& nc = f.nb[c][zp];
    uint32_t S, O, up[12], V[4];
    packed_loads<NARROW>(f, nc, base, S, O, up);
    if (VQ) {
        const uint4 v = *vq;
        V[0] = v.x;
        V[1] = v.y;
        V[2] = v.z;
        V[3] = v.w;
    } else {
        packed_vacancies<NARROW>(f, nc, base, V);
    }
    // the first half's four Philox blocks do not depend on the loads: drawn while they are in
    // flight (every pass starts all warps together, so nothing else would fill that wait)
    uint4 u_first[4];
    if (use_pre) {
#pragma unroll
        for (int v = 0; v < 4; ++v) u_first[v] = pre[v];
    } else {
        philox10_xn<4>(q0, (uint32_t)sweep, (uint32_t)(sweep >> 32), 0u, f.key0, f.key1, u_first);
    }
    if (!O) return;             // no occupied site in the word (tested after the loads are issued)
    const uint32_t F =
        (!GATE && (sflags & kFlagNoNever))
            ? packed_decide<false, true>(S, O, up, V, q0, sweep, tab, gthr, always_draw, f.key0, f.key1, u_first, dM, dB)
            : packed_decide<GATE>(S, O, up, V, q0, sweep, tab, gthr, always_draw, f.key0, f.key1, u_first, dM, dB);
    if (F) f.sp[base] = S ^ F;
}

template <bool GATE, bool NARROW>
__device__ __forceinline__ void word_packed(const DevFilm& f, int c, int z, int j, int w,
                                            unsigned long long sweep, const uint32_t* tab,
                                            uint32_t gthr, uint32_t sflags, int& dM, int& dB, const uint4 (&pre)[4],
                                            bool use_pre) {
    word_packed_at<GATE, NARROW, false>(f, c, z & 1, addrw(f, c, z, j, w), block_counter(f, c, z, j, 32 * w), nullptr,
                                        sweep, tab, gthr, sflags, dM, dB, pre, use_pre);
}

template <int MODE, bool GATE>
__device__ __forceinline__ void colour_pass(const DevFilm& f, int c, unsigned long long sweep,
                                            const uint32_t* tab, uint32_t gthr, int items,
                                            ItemWalk w, unsigned G, unsigned cta, uint32_t sflags, int& dM, int& dB,
                                            const uint4 (&pre)[4], bool have_pre) {
    const int stride = (int)G * blockDim.x;
    if (MODE == MODE_PACKED && f.ient) {
        // the colour's occupied words only, thread t taking entries t, t + stride, ...: each
        // entry's word index (layer parity in bit 31), Philox counter and vacant-neighbour count
        // are precomputed; the first one's first four Philox blocks may have been drawn before
        // the pass (pre)
        const uint2* ent = reinterpret_cast<const uint2*>(f.ient) + (int64_t)c * f.item_cap;
        const uint4* vq = reinterpret_cast<const uint4*>(f.ivq) + (int64_t)c * f.item_cap;
        const int n = f.nitems[c];
        const int it0 = first_item(G, cta);
        for (int it = it0; it < n; it += stride) {
            const uint2 pq = ent[it];
            word_packed_at<GATE, true, true>(f, c, (int)(pq.x >> 31), (int64_t)(pq.x & 0x7FFFFFFFu), pq.y, vq + it, sweep,
                                             tab, gthr, sflags, dM, dB, pre, have_pre && it == it0);
        }
        return;
    }
    if (MODE == MODE_INT8 && f.ient) {
        // the colour's chunks holding an occupied site, each with its precomputed byte offset
        // (layer parity in bit 31) and Philox counter
        const uint2* ent = reinterpret_cast<const uint2*>(f.ient) + (int64_t)c * f.item_cap;
        const int n = f.nitems[c];
        for (int it = first_item(G, cta); it < n; it += stride) {
            const uint2 pq = ent[it];
            chunk_int8_at<GATE>(f, c, (int)(pq.x >> 31), (int64_t)(pq.x & 0x7FFFFFFFu), pq.y, sweep, tab, gthr, dM, dB,
                                (sflags & kFlagNoNever) != 0u);
        }
        return;
    }
    const int j0 = f.slab ? f.jlo : 0;
    for (int it = first_item(G, cta); it < items; it += stride, w.next()) {
        if (MODE == MODE_INT8) chunk_int8<GATE>(f, c, w.z, j0 + w.jr, w.ck, sweep, tab, gthr, dM, dB,
                                                (sflags & kFlagNoNever) != 0u);
        else if (MODE == MODE_GENERIC) block_generic<GATE>(f, c, w.z, j0 + w.jr, w.ck, sweep, tab, gthr, dM, dB);
        else word_packed<GATE, false>(f, c, w.z, j0 + w.jr, w.ck, sweep, tab, gthr, sflags, dM, dB, pre, false);
    }
}

// Barrier between colour passes: over a cooperative grid (counter in the film's state), or
// over the CTAs of one thread-block cluster (hardware barrier).
enum { BAR_GRID = 0, BAR_CLUSTER = 1 };

// The launch's sweeps of one film by G CTAs (this one is number cta), the film in global
// memory; G = 1 needs no barrier beyond __syncthreads.
template <int MODE, int BAR = BAR_GRID>
__device__ __forceinline__ void sweep_body(const SweepArgs& a, unsigned G, unsigned cta) {
    __shared__ uint32_t tab[128];
    __shared__ uint32_t gate_s[2];      // gate threshold, step flags
    __shared__ long long red[64];
    __shared__ int ok_s;
    const DevFilm& f = a.f;
    FilmState* st = a.st;
    unsigned target = 0;
    const int per_row = MODE == MODE_INT8 ? f.nck : (MODE == MODE_GENERIC ? f.Qw : f.nw);
    const int nrows = f.slab ? f.jhi - f.jlo : f.Rh;        // rows this film updates
    const int items = f.L * nrows * per_row;
    ItemWalk walk0;
    walk0.init(first_item(G, cta), (int)G * blockDim.x, per_row, nrows > 0 ? nrows : 1);
    // colours of this launch: all four, or one colour pass of one sweep
    const int c_begin = a.pass_plus1 ? a.pass_plus1 - 1 : 0, c_end = a.pass_plus1 ? a.pass_plus1 : 4;
    // packed films with word lists on the grid path: the barrier is split (see grid_arrive)
    const bool PREFETCH = MODE == MODE_PACKED && BAR == BAR_GRID && G > 1 && f.ient != nullptr && !a.pass_plus1;
    uint4 pf[4];
    bool have_pf = false;
    int k = a.k0, pos = a.pos0;
    const bool folder = cta == 0 && threadIdx.x == 0;
    __shared__ RunState rs;     // touched by the folding thread only
    int k_eq = 0, k_tot = 0;
    if (folder) {
        load_run_state(st, rs);
        k_eq = a.step_eq[k];
        k_tot = a.step_total[k];
    }
    stage_table<MODE == MODE_PACKED, MODE == MODE_INT8>(a.tables, k, tab, gate_s);
    for (long long t = 0; t < a.nsweeps; ++t) {
        if (pos == a.step_total[k]) {
            ++k;
            pos = 0;
            stage_table<MODE == MODE_PACKED, MODE == MODE_INT8>(a.tables, k, tab, gate_s);
            if (folder) { k_eq = a.step_eq[k]; k_tot = a.step_total[k]; }
        }
        const unsigned long long sweep = (unsigned long long)(a.sweep0 + t + 1);
        const uint32_t gthr = gate_s[0];
        const uint32_t sflags = gate_s[1];
        int dM = 0, dB = 0;
        for (int c = c_begin; c < c_end; ++c) {
            if (a.use_gate) colour_pass<MODE, true>(f, c, sweep, tab, gthr, items, walk0, G, cta, sflags, dM, dB, pf, have_pf);
            else colour_pass<MODE, false>(f, c, sweep, tab, gthr, items, walk0, G, cta, sflags, dM, dB, pf, have_pf);
            if (c == c_end - 1) {
                long long sM = dM, sB = dB;
                block_sum2(sM, sB, red);
                if (threadIdx.x == 0 && (sM | sB)) {
                    unsigned long long* acc = reinterpret_cast<unsigned long long*>(&st->acc[sweep & 1][0]);
                    atomicAdd(acc, (unsigned long long)sM);
                    atomicAdd(acc + 1, (unsigned long long)sB);
                }
            }
            if (BAR == BAR_CLUSTER) {
                if (G > 1) cluster_barrier();
                else __syncthreads();
            } else if (PREFETCH) {
                grid_arrive(st, G, target);
                // the first word of the next pass (the lists do not change): its first four
                // Philox blocks while thread 0 waits for the other CTAs
                have_pf = false;
                const int cn = (c + 1) & 3;
                const long long tn = c == 3 ? t + 1 : t;
                const int it0 = first_item(G, cta);
                if (tn < a.nsweeps && it0 < f.nitems[cn]) {
                    const uint32_t qn = f.ient[2 * ((int64_t)cn * f.item_cap + it0) + 1];
                    const unsigned long long sn = (unsigned long long)(a.sweep0 + tn + 1);
                    philox10_xn<4>(qn, (uint32_t)sn, (uint32_t)(sn >> 32), 0u, f.key0, f.key1, pf);
                    have_pf = true;
                }
                if (!grid_wait(st, G, target, &ok_s)) return;
            } else if (!grid_barrier(st, G, target, &ok_s)) {
                return;
            }
        }
        if (folder && c_end == 4) {
            unsigned long long* acc = reinterpret_cast<unsigned long long*>(&st->acc[sweep & 1][0]);
            const long long sM = (long long)atomicExch(acc, 0ull);
            const long long sB = (long long)atomicExch(acc + 1, 0ull);
            fold_sweep(a, rs, k, pos, k_eq, k_tot, sM, sB, t);
        }
        ++pos;
    }
    if (folder) store_run_state(st, rs);
}

template <int MODE>
__global__ void __launch_bounds__(kBlock) k_sweep(const __grid_constant__ SweepArgs a) {
    sweep_body<MODE>(a, gridDim.x, blockIdx.x);
}

__device__ __forceinline__ int mode_of_film(const DevFilm& f);

// The next film of a global-memory queue kernel: its own queue first; once that is empty, the
// not yet started films of a resident queue (`steal`, the films of the resident kernel of the
// same size class), which it runs in global memory with the same trajectory.  Returns the film's
// index in its queue, own (>= 0) or stolen (-2 - index), or -1 when both are empty.
__device__ __forceinline__ int take_film(unsigned* next, int nfilms, const StealQueue& steal, bool& own_done) {
    if (!own_done) {
        const int idx = (int)atomicAdd(next, 1u);
        if (idx < nfilms) return idx;
        own_done = true;
    }
    if (steal.n > 0) {
        const int idx = (int)atomicAdd(steal.next, 1u);
        if (idx < steal.n) {
            atomicAdd(steal.taken, 1u);
            return -2 - idx;
        }
    }
    return -1;
}

// Batched films one thread-block cluster of K CTAs each, with their state in global memory:
// every cluster takes the next film of the queue and runs its sweeps, colour passes separated
// by the cluster barrier; then films of the resident cluster queue that have not started yet.
template <int K>
__global__ void __launch_bounds__(kBlock) k_batch_cluster_global(const SweepArgs* films, int nfilms,
                                                                 unsigned* next, StealQueue steal) {
    __shared__ int film_s;
    const unsigned rank = cluster_ctarank();
    bool own_done = false;
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            const int idx = take_film(next, nfilms, steal, own_done);
            for (unsigned r = 0; r < (unsigned)K; ++r) {
                uint64_t p;
                asm volatile("mapa.u64 %0, %1, %2;" : "=l"(p) : "l"(reinterpret_cast<uint64_t>(&film_s)), "r"(r));
                *reinterpret_cast<int*>(p) = idx;
            }
        }
        cluster_barrier();
        const int idx = film_s;
        cluster_barrier();      // every CTA has the index before CTA 0 writes the next one
        if (idx == -1 || idx >= nfilms || (idx < -1 && -2 - idx >= steal.n)) break;
        const SweepArgs& a = idx >= 0 ? films[idx] : steal.films[-2 - idx].s;
        switch (mode_of_film(a.f)) {
            case MODE_INT8: sweep_body<MODE_INT8, BAR_CLUSTER>(a, (unsigned)K, rank); break;
            case MODE_GENERIC: sweep_body<MODE_GENERIC, BAR_CLUSTER>(a, (unsigned)K, rank); break;
            default: sweep_body<MODE_PACKED, BAR_CLUSTER>(a, (unsigned)K, rank); break;
        }
    }
}

__device__ __forceinline__ int mode_of_film(const DevFilm& f) {
    return f.packed ? MODE_PACKED : ((f.flags & 7u) ? MODE_GENERIC : MODE_INT8);
}

// Batched films one CTA each, with their state in global memory: every CTA takes the next film
// of the queue (a device counter), runs its sweeps (colour passes separated by __syncthreads
// only) and takes another until the queue is empty; then films of the resident single-CTA
// queue that have not started yet.  Films are independent chains.
__global__ void __launch_bounds__(kBlock) k_batch_global(const SweepArgs* films, int nfilms, unsigned* next,
                                                         StealQueue steal) {
    __shared__ int film_s;
    bool own_done = false;
    for (;;) {
        if (threadIdx.x == 0) film_s = take_film(next, nfilms, steal, own_done);
        __syncthreads();
        const int idx = film_s;
        __syncthreads();        // every thread has the index before thread 0 takes the next one
        if (idx == -1 || idx >= nfilms || (idx < -1 && -2 - idx >= steal.n)) break;
        const SweepArgs& a = idx >= 0 ? films[idx] : steal.films[-2 - idx].s;
        switch (mode_of_film(a.f)) {
            case MODE_INT8: sweep_body<MODE_INT8>(a, 1u, 0u); break;
            case MODE_GENERIC: sweep_body<MODE_GENERIC>(a, 1u, 0u); break;
            default: sweep_body<MODE_PACKED>(a, 1u, 0u); break;
        }
    }
}

// k_words runs packed whole films with word lists over several CTAs (grid barrier, whole sweeps).
inline bool words_path(const DevFilm& f) { return f.packed && f.ient != nullptr && !f.slab; }

template <int MODE>
int launch_mode(const SweepArgs& a, int ctas, int threads, cudaStream_t s) {
    if (threads % 32 || threads < 32 || threads > kBlock) return (int)cudaErrorInvalidValue;   // whole warps
    if (ctas <= 1) {
        k_sweep<MODE><<<1, threads, 0, s>>>(a);
        return (int)cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(&a.st->bar_count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return (int)e;
    if (MODE == MODE_PACKED && words_path(a.f) && !a.pass_plus1) return launch_words(a, ctas, threads, s);
    void* args[] = {const_cast<SweepArgs*>(&a)};
    return (int)cudaLaunchCooperativeKernel((const void*)k_sweep<MODE>, dim3(ctas), dim3(threads), args, 0, s);
}

template <int MODE>
int max_ctas_mode(const DevFilm& f, int threads, int* out) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (MODE == MODE_PACKED && words_path(f)) {
        if (e == cudaSuccess) return words_max_ctas(threads, out);
    } else if (e == cudaSuccess) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep<MODE>, threads, 0);
    }
    *out = sms * per;
    return (int)e;
}

}  // namespace

static int mode_of(const DevFilm& f) {
    if (f.packed) return MODE_PACKED;
    return (f.flags & 7u) ? MODE_GENERIC : MODE_INT8;
}

int launch_sweeps(const SweepArgs& a, int ctas, int threads, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (mode_of(a.f)) {
        case MODE_INT8: return launch_mode<MODE_INT8>(a, ctas, threads, s);
        case MODE_GENERIC: return launch_mode<MODE_GENERIC>(a, ctas, threads, s);
        default: return launch_mode<MODE_PACKED>(a, ctas, threads, s);
    }
}

int sweep_max_ctas_for(const DevFilm& f, int threads, int* max_ctas) {
    switch (mode_of(f)) {
        case MODE_INT8: return max_ctas_mode<MODE_INT8>(f, threads, max_ctas);
        case MODE_GENERIC: return max_ctas_mode<MODE_GENERIC>(f, threads, max_ctas);
        default: return max_ctas_mode<MODE_PACKED>(f, threads, max_ctas);
    }
}

int batch_global_units(int threads, int* units) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_global, threads, 0);
    *units = sms * per;
    return (int)e;
}

int launch_batch_global(const SweepArgs* films, int n, unsigned* next, int threads, int units, void* stream,
                        StealQueue steal) {
    if (threads % 32 || threads < 32 || threads > kBlock || units < 1) return (int)cudaErrorInvalidValue;
    k_batch_global<<<units, threads, 0, static_cast<cudaStream_t>(stream)>>>(films, n, next, steal);
    return (int)cudaGetLastError();
}

namespace {
template <int K>
cudaLaunchConfig_t cluster_global_config(int threads, int units, cudaStream_t s, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(units * K);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}
template <int K>
int cluster_global_units_k(int threads, int* units) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_global_config<K>(threads, 1, nullptr, attr);
    return (int)cudaOccupancyMaxActiveClusters(units, k_batch_cluster_global<K>, &cfg);
}
template <int K>
int launch_cluster_global_k(const SweepArgs* films, int n, unsigned* next, int threads, int units, cudaStream_t s,
                            StealQueue steal) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_global_config<K>(threads, units, s, attr);
    return (int)cudaLaunchKernelEx(&cfg, k_batch_cluster_global<K>, films, n, next, steal);
}
}  // namespace

int batch_cluster_global_units(int K, int threads, int* units) {
    switch (K) {
        case 2: return cluster_global_units_k<2>(threads, units);
        case 4: return cluster_global_units_k<4>(threads, units);
        case 8: return cluster_global_units_k<8>(threads, units);
        default: return (int)cudaErrorInvalidValue;
    }
}

int launch_batch_cluster_global(const SweepArgs* films, int n, unsigned* next, int K, int threads, int units,
                                void* stream, StealQueue steal) {
    if (threads % 32 || threads < 32 || threads > kBlock || units < 1) return (int)cudaErrorInvalidValue;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (K) {
        case 2: return launch_cluster_global_k<2>(films, n, next, threads, units, s, steal);
        case 4: return launch_cluster_global_k<4>(films, n, next, threads, units, s, steal);
        case 8: return launch_cluster_global_k<8>(films, n, next, threads, units, s, steal);
        default: return (int)cudaErrorInvalidValue;
    }
}

int sweep_items_per_pass(const DevFilm& f) {
    if (f.items) return std::max(std::max(f.nitems[0], f.nitems[1]), std::max(f.nitems[2], f.nitems[3]));
    const int per_row = f.packed ? f.nw : ((f.flags & 7u) ? f.Qw : f.nck);
    return f.L * f.Rh * per_row;
}

namespace {

// Test of the grid barrier's bounded wait: every CTA arrives once, then waits, with the kernels'
// own wait, for one arrival more than there are CTAs, which nothing makes; the wait gives up,
// records ISF_ERR_TIMEOUT in the status word and the kernel returns.
__global__ void k_wait_probe(FilmState* st) {
    __shared__ int ok_s;
    unsigned target = 0;
    grid_arrive(st, gridDim.x, target);
    grid_wait(st, gridDim.x, target + 1u, &ok_s);
}

}  // namespace

int wait_probe(int ctas, int* status, int* where) {
    if (ctas < 2) return (int)cudaErrorInvalidValue;
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_wait_probe, 32, 0);
    if (e != cudaSuccess) return (int)e;
    if (ctas > sms * per) return (int)cudaErrorInvalidValue;       // all CTAs must be co-resident
    FilmState* st = nullptr;
    e = cudaMalloc(&st, sizeof(FilmState));
    if (e != cudaSuccess) return (int)e;
    e = cudaMemset(st, 0, sizeof(FilmState));
    void* args[] = {&st};
    if (e == cudaSuccess) e = cudaLaunchCooperativeKernel((const void*)k_wait_probe, dim3(ctas), dim3(32), args, 0, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    FilmState h{};
    if (e == cudaSuccess) e = cudaMemcpy(&h, st, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(st);
    if (e != cudaSuccess) return (int)e;
    *status = h.error;
    *where = h.error_where;
    return 0;
}

}  // namespace isf
