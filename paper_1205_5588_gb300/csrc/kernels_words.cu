// kernels_words.cu — the colour passes of a bit-packed film with occupied-word lists on the
// whole grid (Eq. 8, items 1-3 of Sec. 5; the Eq. 9 gate of items 4-5 when a switching field is
// set), the film's four conflict-free colours (Sec. 3, Fig. 1) stepped through the temperature /
// field schedule in one persistent cooperative launch.  Same decisions, random words and
// bookkeeping as k_sweep: only the order of the work differs (the path's hot kernel).
#include <cuda_runtime.h>

#include "grid_sync.cuh"

namespace isf {

namespace {

constexpr int kBlock = 512;      // CTA of the words kernel (<= 128 registers per thread)

// ---- packed films with occupied-word lists on the whole grid: random words drawn ahead -----
// A colour pass of a packed film is half Philox arithmetic (8 blocks per 32-site word), and
// the counters of a pass's words are known before the pass: they depend on the word and the
// sweep, not on the spins.  So once a warp has decided its words of pass c it arrives at the
// grid barrier (through a per-CTA counter, without waiting for the CTA's other warps) and draws
// the Philox blocks of its first word of pass c + 1 into shared memory (the first four blocks,
// and the last four too when the step's table says nearly every word needs them); a thread's
// second word of a pass gets its blocks drawn while its first word's loads are in flight.  The
// decisions themselves only load, count, look up and compare.  The threads with fewer words in a
// pass thus fill the time the others need for their extra word, and everyone fills the barrier's
// latency.  A thread keeps kAheadSlots words this way; further words of a pass (small grids)
// draw in the pass.
constexpr int kAheadSlots = 2;

// Bytes of dynamic shared memory of k_words with this block size: the random words drawn ahead
// ([slot][block][thread] uint4) and the thread's list entries of every colour ([colour][slot]
// [thread] uint2; a thread takes the same words in every sweep, so they are read once a launch).
constexpr size_t ahead_bytes(int threads) {
    return (size_t)kAheadSlots * 8 * (size_t)threads * sizeof(uint4) + (size_t)4 * kAheadSlots * threads * sizeof(uint2);
}

// The Philox blocks of this thread's words s0 .. s1-1 of colour c at `sweep` into its slots of
// `ahead`; the second four blocks only when `both`.  ents: the entries cached in shared memory.
__device__ __forceinline__ void draw_ahead(const DevFilm& f, int c, unsigned long long sweep, bool both, int it0,
                                           int stride, uint4* ahead, const uint2* ents, const uint32_t (&rk)[20],
                                           int s0 = 0, int s1 = kAheadSlots) {
    const SweepConst sc = sweep_const(sweep, rk);
    const int n = f.nitems[c];
    const int bd = blockDim.x, tid = threadIdx.x;
    int it = it0 + s0 * stride;
#pragma unroll 1
    for (int slot = s0; slot < s1 && it < n; ++slot, it += stride) {
        const uint32_t q = ents[(c * kAheadSlots + slot) * bd + tid].y;
        uint4 u[4];
        philox10_sc<4>(q, 0u, sc, rk, u);
#pragma unroll
        for (int v = 0; v < 4; ++v) ahead[(slot * 8 + v) * bd + tid] = u[v];
        if (both) {
            philox10_sc<4>(q + 4, 0u, sc, rk, u);
#pragma unroll
            for (int v = 0; v < 4; ++v) ahead[(slot * 8 + 4 + v) * bd + tid] = u[v];
        }
    }
}

// One colour pass over this thread's listed words it0, it0 + stride, ... (their random words
// in `ahead` for the first kAheadSlots: the first word's drawn before the pass, the second's
// here while the first word's loads are in flight; `both`: the second four blocks too).
template <bool GATE>
__device__ __forceinline__ void pass_words(const DevFilm& f, int c, unsigned long long sweep, const uint32_t* tab,
                                           uint32_t gthr, bool always_draw, bool both, bool no_never, int it0,
                                           int stride, uint4* ahead, const uint2* ents, int& dM, int& dB,
                                           const uint32_t (&rk)[20]) {
    const uint2* ent = reinterpret_cast<const uint2*>(f.ient) + (int64_t)c * f.item_cap;
    const uint4* vq = reinterpret_cast<const uint4*>(f.ivq) + (int64_t)c * f.item_cap;
    const int n = f.nitems[c];
    const int bd = blockDim.x, tid = threadIdx.x;
    int slot = 0;
#pragma unroll 1
    for (int it = it0; it < n; it += stride, ++slot) {
        // the entry from shared memory, so the word's loads leave at once
        const uint2 pq = slot < kAheadSlots ? ents[(c * kAheadSlots + slot) * bd + tid] : ent[it];
        const int64_t base = (int64_t)(pq.x & 0x7FFFFFFFu);
        const NbrClass& nc = f.nb[c][pq.x >> 31];
        uint32_t S, O, up[12], V[4];
        packed_loads<true>(f, nc, base, S, O, up);
        const uint4 v4 = vq[it];
        // the second word's random blocks while the first word's loads are in flight (the barrier
        // wait before the pass drew only the first word's, so every thread draws one word there)
        if (slot == 0) draw_ahead(f, c, sweep, both, it0, stride, ahead, ents, rk, 1, 2);
        V[0] = v4.x; V[1] = v4.y; V[2] = v4.z; V[3] = v4.w;
        uint4 uf[4], us[4];
        const bool drawn = slot < kAheadSlots;
        if (drawn) {
#pragma unroll
            for (int v = 0; v < 4; ++v) uf[v] = ahead[(slot * 8 + v) * bd + tid];
            if (both) {
#pragma unroll
                for (int v = 0; v < 4; ++v) us[v] = ahead[(slot * 8 + 4 + v) * bd + tid];
            }
        } else {
            philox10_xn<4>(pq.y, (uint32_t)sweep, (uint32_t)(sweep >> 32), 0u, f.key0, f.key1, uf);
        }
        const uint4* u2 = (drawn && both) ? us : nullptr;
        const uint32_t F =
            (!GATE && no_never)
                ? packed_decide<false, true>(S, O, up, V, pq.y, sweep, tab, gthr, always_draw, f.key0, f.key1, uf,
                                             dM, dB, u2)
                : packed_decide<GATE>(S, O, up, V, pq.y, sweep, tab, gthr, always_draw, f.key0, f.key1, uf, dM, dB,
                                      u2);
        if (F) f.sp[base] = S ^ F;
    }
}

template <bool GATE>
__global__ void __launch_bounds__(kBlock) k_words(const __grid_constant__ SweepArgs a) {
    extern __shared__ uint4 ahead[];                 // [kAheadSlots][8][blockDim], then the entries
    __shared__ uint32_t tab[128];
    __shared__ uint32_t gate_s[2];
    __shared__ int ok_s;
    __shared__ RunState rs;                          // touched by the folding thread only
    __shared__ unsigned warps_in;                    // warps that finished a pass (grows through the launch)
    __shared__ long long acc_s[2];                   // the CTA's dM, dB of the current sweep
    const DevFilm& f = a.f;
    FilmState* st = a.st;
    const unsigned G = gridDim.x, cta = blockIdx.x;
    const unsigned nwarps = blockDim.x >> 5;
    unsigned pass_no = 0;
    if (threadIdx.x == 0) {         // published by stage_table's barrier below
        warps_in = 0;
        acc_s[0] = 0;
        acc_s[1] = 0;
    }
    unsigned target = 0;
    int k = a.k0, pos = a.pos0;
    const bool folder = cta == 0 && threadIdx.x == 0;
    int k_eq = 0, k_tot = 0;
    if (folder) {
        load_run_state(st, rs);
        k_eq = a.step_eq[k];
        k_tot = a.step_total[k];
    }
    const int it0 = first_item(G, cta);
    const int stride = (int)G * blockDim.x;
    uint32_t rk[20];
    round_keys(f.key0, f.key1, rk);
    uint2* ents = reinterpret_cast<uint2*>(ahead + (size_t)kAheadSlots * 8 * blockDim.x);
    for (int c = 0; c < 4; ++c) {
        const uint2* ent = reinterpret_cast<const uint2*>(f.ient) + (int64_t)c * f.item_cap;
        for (int slot = 0; slot < kAheadSlots; ++slot) {
            const int it = it0 + slot * stride;
            ents[(c * kAheadSlots + slot) * blockDim.x + threadIdx.x] = it < f.nitems[c] ? ent[it] : make_uint2(0u, 0u);
        }
    }
    auto step_draws_all = [&](int kk) {
        return (a.tables[(size_t)kk * kTableStride + kFlagSlot] & kFlagAlwaysDraw) != 0u;
    };
    // the first pass's random words
    {
        const int kf = a.pos0 == a.step_total[a.k0] ? a.k0 + 1 : a.k0;
        if (a.nsweeps > 0)
            draw_ahead(f, 0, (unsigned long long)(a.sweep0 + 1), step_draws_all(kf), it0, stride, ahead, ents, rk, 0, 1);
    }
    stage_table<true>(a.tables, k, tab, gate_s);
    for (long long t = 0; t < a.nsweeps; ++t) {
        if (pos == a.step_total[k]) {
            ++k;
            pos = 0;
            stage_table<true>(a.tables, k, tab, gate_s);
            if (folder) { k_eq = a.step_eq[k]; k_tot = a.step_total[k]; }
        }
        const unsigned long long sweep = (unsigned long long)(a.sweep0 + t + 1);
        const uint32_t gthr = gate_s[0];
        const bool always_draw = (gate_s[1] & kFlagAlwaysDraw) != 0;
        // the step of the next sweep (for the random words of its first pass)
        const int k_next = pos + 1 == a.step_total[k] ? k + 1 : k;
        int dM = 0, dB = 0;
        for (int c = 0; c < 4; ++c) {
            pass_words<GATE>(f, c, sweep, tab, gthr, always_draw, always_draw, (gate_s[1] & kFlagNoNever) != 0, it0,
                             stride, ahead, ents, dM, dB, rk);
            // each warp arrives as soon as its own words are done: the CTA's last warp to finish
            // (release / acquire on a shared counter orders every warp's stores before it) adds
            // the CTA's (dM, dB) of the sweep and arrives at the grid barrier with release semantics
            const int lane = threadIdx.x & 31;
            if (c == 3) {
                const long long wM = warp_sum((long long)dM), wB = warp_sum((long long)dB);
                if (lane == 0 && (wM | wB)) {
                    atomicAdd(reinterpret_cast<unsigned long long*>(&acc_s[0]), (unsigned long long)wM);
                    atomicAdd(reinterpret_cast<unsigned long long*>(&acc_s[1]), (unsigned long long)wB);
                }
            }
            __syncwarp();
            ++pass_no;
            if (lane == 0) {
                unsigned old;
                asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], 1;"
                             : "=r"(old) : "r"((unsigned)__cvta_generic_to_shared(&warps_in)) : "memory");
                if (old == pass_no * nwarps - 1u) {
                    if (c == 3) {
                        const long long sM = acc_s[0], sB = acc_s[1];
                        acc_s[0] = 0;
                        acc_s[1] = 0;
                        if (sM | sB) {
                            unsigned long long* acc = reinterpret_cast<unsigned long long*>(&st->acc[sweep & 1][0]);
                            atomicAdd(acc, (unsigned long long)sM);
                            atomicAdd(acc + 1, (unsigned long long)sB);
                        }
                    }
                    if (G > 1) red_release_add_u32(&st->bar_count, 1u);
                }
            }
            target += G;
            // while the other warps and CTAs finish this pass: the random words of the next one
            if (c < 3) {
                draw_ahead(f, c + 1, sweep, always_draw, it0, stride, ahead, ents, rk, 0, 1);
            } else if (t + 1 < a.nsweeps) {
                draw_ahead(f, 0, sweep + 1, step_draws_all(k_next), it0, stride, ahead, ents, rk, 0, 1);
            }
            if (!grid_wait(st, G, target, &ok_s)) return;
        }
        if (folder) {
            unsigned long long* acc = reinterpret_cast<unsigned long long*>(&st->acc[sweep & 1][0]);
            const long long sM = (long long)atomicExch(acc, 0ull);
            const long long sB = (long long)atomicExch(acc + 1, 0ull);
            fold_sweep(a, rs, k, pos, k_eq, k_tot, sM, sB, t);
        }
        ++pos;
    }
    if (folder) store_run_state(st, rs);
}

template <bool GATE>
cudaError_t words_smem_attr(int threads) {
    return cudaFuncSetAttribute(k_words<GATE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ahead_bytes(threads));
}

}  // namespace

int words_smem_bytes(int threads) { return (int)ahead_bytes(threads); }

int launch_words(const SweepArgs& a, int ctas, int threads, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (threads % 32 || threads < 32 || threads > kBlock || ctas < 2) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(&a.st->bar_count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return (int)e;
    void* args[] = {const_cast<SweepArgs*>(&a)};
    const size_t smem = ahead_bytes(threads);
    const void* fn = a.use_gate ? (const void*)k_words<true> : (const void*)k_words<false>;
    e = a.use_gate ? words_smem_attr<true>(threads) : words_smem_attr<false>(threads);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(threads), args, smem, s);
}

int words_max_ctas(int threads, int* out) {
    int dev = 0, sms = 0, per = 0, per_g = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the gate and no-gate kernels have the same shared memory; take the smaller residency
    if (e == cudaSuccess) e = words_smem_attr<false>(threads);
    if (e == cudaSuccess) e = words_smem_attr<true>(threads);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_words<false>, threads, ahead_bytes(threads));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_g, k_words<true>, threads, ahead_bytes(threads));
    *out = sms * (per < per_g ? per : per_g);
    return (int)e;
}

}  // namespace isf
