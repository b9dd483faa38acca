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

#include "../../include/isingfilm.h"
#include "device_common.cuh"

namespace isf {

namespace {

enum { MODE_INT8 = 0, MODE_GENERIC = 1, MODE_PACKED = 2 };
constexpr int kBlock = 256;
constexpr unsigned kSpinLimit = 1u << 22;   // ~ seconds of waiting, then give up

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// Barrier over the G co-resident CTAs.  Thread 0 of each CTA arrives on a counter; the last one
// resets it and publishes a new generation; the others wait for it with a bounded spin.
__device__ bool grid_barrier(FilmState* st, unsigned G, unsigned& gen, int* ok_s) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (G > 1) {
            __threadfence();
            const unsigned arrived = atomicAdd(&st->bar_count, 1u) + 1u;
            if (arrived == G) {
                atomicExch(&st->bar_count, 0u);
                __threadfence();
                st_release_u32(&st->bar_gen, gen + 1u);
            } else {
                unsigned spins = 0;
                while (ld_acquire_u32(&st->bar_gen) == gen) {
                    if (ld_volatile_i32(&st->error)) { ok = 0; break; }
                    if (++spins > kSpinLimit) {
                        atomicCAS(&st->error, 0, (int)ISF_ERR_TIMEOUT);
                        st->error_where = 1;
                        ok = 0;
                        break;
                    }
                    if (spins > 32) __nanosleep(40);
                }
            }
            gen += 1u;
            __threadfence();
        }
        if (ld_volatile_i32(&st->error)) ok = 0;
        *ok_s = ok;
    }
    __syncthreads();
    return *ok_s != 0;
}

// Table of the current step in shared memory, indexed by the per-site byte the pass forms:
//   int8 / generic: (stored byte << 5) | (n + 12), stored byte 0 = down, 1 = vacancy, 2 = up
//   packed        : (occupied << 6) | (up << 5) | (n + 12)
// Vacancies map to 0 ("never"), so they never flip and never draw a random word.
template <int MODE>
__device__ void load_table(const SweepArgs& a, int k, uint32_t* tab, uint32_t* gate) {
    const uint32_t* src = a.tables + (size_t)k * kTableStride;
    for (int t = threadIdx.x; t < 128; t += blockDim.x) {
        uint32_t v = 0;
        const int X = t & 31;
        if (X <= 24) {
            if (MODE == MODE_PACKED) {
                if (t >> 6) v = src[X * 2 + ((t >> 5) & 1)];
            } else {
                const int sb = t >> 5;
                if (sb == 0) v = src[X * 2 + 0];
                else if (sb == 2) v = src[X * 2 + 1];
            }
        }
        tab[t] = v;
    }
    if (threadIdx.x == 0) *gate = src[kGateSlot];
    __syncthreads();
}

// accept iff u < thr, or thr == always (min keeps u = 2^32-1 below always)
__device__ __forceinline__ bool metropolis_accept(uint32_t u, uint32_t thr) {
    return min(u, 0xFFFFFFFEu) < thr;
}
// a random word decides the site only when thr is neither 0 ("never") nor always
__device__ __forceinline__ bool needs_word(uint32_t thr) { return (thr - 1u) < 0xFFFFFFFEu; }

__device__ __forceinline__ uint4 ld16(const uint8_t* p) { return *reinterpret_cast<const uint4*>(p); }
__device__ __forceinline__ uint32_t ld4(const uint8_t* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ void add4(uint4& a, const uint4& b) {
    a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
}

// Eq. 9 gate for the accepted lanes of one 4-site block (stream 1): clears the lanes that fail.
__device__ __forceinline__ uint32_t gate_block(uint32_t acc_lanes, uint32_t gthr, uint32_t q,
                                               unsigned long long sweep, const DevFilm& f) {
    if (!acc_lanes || gthr == kAlways) return acc_lanes;
    if (gthr == 0u) return 0u;
    const uint4 g = philox10(make_uint4(q, (uint32_t)sweep, (uint32_t)(sweep >> 32), 1u), f.key0, f.key1);
    uint32_t keep = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
        if (metropolis_accept(word_of(g, b), gthr)) keep |= 1u << b;
    return acc_lanes & keep;
}

// ---- int8 layout, open boundaries: one thread per 16-site chunk of a colour row ------------
template <bool GATE>
__device__ __forceinline__ void chunk_int8(const DevFilm& f, int c, int z, int j, int ck,
                                           unsigned long long sweep, const uint32_t* tab,
                                           uint32_t gthr, long long& dM, long long& dB) {
    const NbrClass& nc = f.nb[c][z & 1];
    uint8_t* own = f.s8 + addr8(f, c, z, j, 16 * ck);
    const uint4 S = ld16(own);
    // n + 12 per byte: sum of the 12 neighbour bytes (S + 1, vacancy 1), no carries (<= 24)
    uint4 acc = ld16(own + nc.off[0]);
#pragma unroll
    for (int k = 1; k < 9; ++k) add4(acc, ld16(own + nc.off[k]));
    if (nc.sgn < 0) {
#pragma unroll
        for (int k = 9; k < 12; ++k) {
            const uint8_t* p = own + nc.off[k];
            const uint4 v = ld16(p);
            const uint32_t e = ld4(p - 4);
            add4(acc, make_uint4(__funnelshift_l(e, v.x, 8), __funnelshift_l(v.x, v.y, 8),
                                 __funnelshift_l(v.y, v.z, 8), __funnelshift_l(v.z, v.w, 8)));
        }
    } else {
#pragma unroll
        for (int k = 9; k < 12; ++k) {
            const uint8_t* p = own + nc.off[k];
            const uint4 v = ld16(p);
            const uint32_t e = ld4(p + 16);
            add4(acc, make_uint4(__funnelshift_r(v.x, v.y, 8), __funnelshift_r(v.y, v.z, 8),
                                 __funnelshift_r(v.z, v.w, 8), __funnelshift_r(v.w, e, 8)));
        }
    }
    const uint32_t q0 = block_counter(f, c, z, j, 16 * ck);
    const uint32_t Sw[4] = {S.x, S.y, S.z, S.w};
    const uint32_t Aw[4] = {acc.x, acc.y, acc.z, acc.w};
    uint32_t out[4];
    uint32_t any = 0;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const uint32_t iw = (Sw[v] << 5) + Aw[v];
        uint32_t thr[4];
        bool need = false;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            thr[b] = tab[(iw >> (8 * b)) & 0xFFu];
            need |= needs_word(thr[b]);
        }
        uint4 u = make_uint4(0, 0, 0, 0);
        if (need) u = philox10(make_uint4(q0 + v, (uint32_t)sweep, (uint32_t)(sweep >> 32), 0u), f.key0, f.key1);
        uint32_t lanes = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (metropolis_accept(word_of(u, b), thr[b])) lanes |= 1u << b;
        if (GATE) lanes = gate_block(lanes, gthr, q0 + v, sweep, f);
        uint32_t flip = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            if (lanes & (1u << b)) {
                const uint32_t byte = (iw >> (8 * b)) & 0xFFu;
                const int s = (byte & 64u) ? 1 : -1;
                const int n = (int)(byte & 31u) - 12;
                dM -= 2 * s;
                dB -= 2 * s * n;
                flip |= 2u << (8 * b);   // 0 <-> 2
            }
        }
        out[v] = Sw[v] ^ flip;
        any |= flip;
    }
    if (any) *reinterpret_cast<uint4*>(own) = make_uint4(out[0], out[1], out[2], out[3]);
}

// ---- int8 layout, any boundary (periodic wraps): one thread per 4-site Philox block --------
template <bool GATE>
__device__ __forceinline__ void block_generic(const DevFilm& f, int c, int z, int j, int blk,
                                              unsigned long long sweep, const uint32_t* tab,
                                              uint32_t gthr, long long& dM, long long& dB) {
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
    if (GATE) lanes = gate_block(lanes, gthr, q, sweep, f);
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

// ---- packed layout: one thread per 32-site word --------------------------------------------
__device__ __forceinline__ void full_add(uint32_t a, uint32_t b, uint32_t c, uint32_t& s, uint32_t& cy) {
    s = a ^ b ^ c;
    cy = (a & b) | (c & (a ^ b));
}
// bit-sliced population count of 12 one-bit inputs per lane -> 4 bit-planes
__device__ __forceinline__ void popcount12(const uint32_t* x, uint32_t& b0, uint32_t& b1, uint32_t& b2, uint32_t& b3) {
    uint32_t s0, c0, s1, c1, s2, c2, s3, c3;
    full_add(x[0], x[1], x[2], s0, c0);
    full_add(x[3], x[4], x[5], s1, c1);
    full_add(x[6], x[7], x[8], s2, c2);
    full_add(x[9], x[10], x[11], s3, c3);
    uint32_t t0, d0;
    full_add(s0, s1, s2, t0, d0);
    b0 = t0 ^ s3;
    const uint32_t d1 = t0 & s3;
    uint32_t e0, f0, e1, f1;
    full_add(c0, c1, c2, e0, f0);
    full_add(c3, d0, d1, e1, f1);
    b1 = e0 ^ e1;
    const uint32_t f2 = e0 & e1;
    full_add(f0, f1, f2, b2, b3);
}

template <bool GATE>
__device__ __forceinline__ void word_packed(const DevFilm& f, int c, int z, int j, int w,
                                            unsigned long long sweep, const uint32_t* tab,
                                            uint32_t gthr, long long& dM, long long& dB) {
    const NbrClass& nc = f.nb[c][z & 1];
    const int64_t base = addrw(f, c, z, j, w);
    const uint32_t* sp = f.sp;
    const uint32_t* op = f.op;
    const uint32_t S = sp[base], O = op[base];
    uint32_t up[12], vac[12];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        up[k] = sp[base + nc.off[k]];
        vac[k] = ~op[base + nc.off[k]];
    }
    if (nc.sgn < 0) {
#pragma unroll
        for (int k = 9; k < 12; ++k) {
            const int64_t a = base + nc.off[k];
            up[k] = __funnelshift_l(sp[a - 1], sp[a], 1);
            vac[k] = ~__funnelshift_l(op[a - 1], op[a], 1);
        }
    } else {
#pragma unroll
        for (int k = 9; k < 12; ++k) {
            const int64_t a = base + nc.off[k];
            up[k] = __funnelshift_r(sp[a], sp[a + 1], 1);
            vac[k] = ~__funnelshift_r(op[a], op[a + 1], 1);
        }
    }
    // X = n + 12 = 2 * (#up) + (#vacant) over the 12 neighbours, 5 bit-planes
    uint32_t U0, U1, U2, U3, V0, V1, V2, V3;
    popcount12(up, U0, U1, U2, U3);
    popcount12(vac, V0, V1, V2, V3);
    uint32_t X[5], k2, k3;
    X[0] = V0;
    X[1] = U0 ^ V1;
    const uint32_t k1 = U0 & V1;
    full_add(U1, V2, k1, X[2], k2);
    full_add(U2, V3, k2, X[3], k3);
    X[4] = U3 ^ k3;
    // transpose the 8 planes {X0..X4, S, O, 0}: byte k of P[r] = table index of lane 8k + r
    uint32_t P[8] = {X[0], X[1], X[2], X[3], X[4], S, O, 0u};
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const uint32_t t = ((P[p] >> 4) ^ P[p + 4]) & 0x0F0F0F0Fu;
        P[p + 4] ^= t;
        P[p] ^= t << 4;
    }
#pragma unroll
    for (int p = 0; p < 8; p += (p & 1) ? 3 : 1) {   // p = 0, 1, 4, 5
        const uint32_t t = ((P[p] >> 2) ^ P[p + 2]) & 0x33333333u;
        P[p + 2] ^= t;
        P[p] ^= t << 2;
    }
#pragma unroll
    for (int p = 0; p < 8; p += 2) {
        const uint32_t t = ((P[p] >> 1) ^ P[p + 1]) & 0x55555555u;
        P[p + 1] ^= t;
        P[p] ^= t << 1;
    }
    const uint32_t q0 = block_counter(f, c, z, j, 32 * w);
    uint32_t F = 0;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        uint32_t thr[4];
        bool need = false;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            thr[b] = tab[(P[4 * (v & 1) + b] >> (8 * (v >> 1))) & 0x7Fu];
            need |= needs_word(thr[b]);
        }
        uint4 u = make_uint4(0, 0, 0, 0);
        if (need) u = philox10(make_uint4(q0 + v, (uint32_t)sweep, (uint32_t)(sweep >> 32), 0u), f.key0, f.key1);
        uint32_t lanes = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (metropolis_accept(word_of(u, b), thr[b])) lanes |= 1u << b;
        if (GATE) lanes = gate_block(lanes, gthr, q0 + v, sweep, f);
        F |= lanes << (4 * v);
    }
    if (F) {
        f.sp[base] = S ^ F;
        const uint32_t Fu = F & S, Fd = F & ~S;        // flipped up -> down, down -> up
        const int nu = __popc(Fu), nd = __popc(Fd);
        int xu = 0, xd = 0;
#pragma unroll
        for (int p = 0; p < 5; ++p) {
            xu += __popc(X[p] & Fu) << p;
            xd += __popc(X[p] & Fd) << p;
        }
        dM += -2LL * (nu - nd);
        dB += -2LL * ((xu - 12 * nu) - (xd - 12 * nd));
    }
}

__device__ void fold_sweep(const SweepArgs& a, int k, int pos, unsigned long long sweep, long long t) {
    FilmState* st = a.st;
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(&st->acc[sweep & 1][0]);
    const long long dM = (long long)atomicExch(acc, 0ull);
    const long long dB = (long long)atomicExch(acc + 1, 0ull);
    const long long M = st->M + dM, B = st->B + dB;
    st->M = M;
    st->B = B;
    if (pos >= a.step_eq[k]) {
        st->n_meas += 1;
        st->sumM += M;
        st->sumAbsM += M < 0 ? -M : M;
        st->sumB += B;
        typedef unsigned __int128 u128;
        u128 m2 = ((u128)st->sumM2[1] << 64 | st->sumM2[0]) + (u128)((__int128)M * M);
        u128 b2 = ((u128)st->sumB2[1] << 64 | st->sumB2[0]) + (u128)((__int128)B * B);
        u128 mb = ((u128)st->sumMB[1] << 64 | st->sumMB[0]) + (u128)((__int128)M * B);
        st->sumM2[0] = (unsigned long long)m2; st->sumM2[1] = (unsigned long long)(m2 >> 64);
        st->sumB2[0] = (unsigned long long)b2; st->sumB2[1] = (unsigned long long)(b2 >> 64);
        st->sumMB[0] = (unsigned long long)mb; st->sumMB[1] = (unsigned long long)(mb >> 64);
    }
    if (pos + 1 == a.step_total[k]) {
        StepRec r;
        r.M_last = M; r.B_last = B; r.n_meas = st->n_meas;
        r.sumM = st->sumM; r.sumAbsM = st->sumAbsM; r.sumB = st->sumB;
        r.sumM2[0] = st->sumM2[0]; r.sumM2[1] = st->sumM2[1];
        r.sumB2[0] = st->sumB2[0]; r.sumB2[1] = st->sumB2[1];
        r.sumMB[0] = st->sumMB[0]; r.sumMB[1] = st->sumMB[1];
        a.recs[k] = r;
        st->n_meas = 0; st->sumM = 0; st->sumAbsM = 0; st->sumB = 0;
        st->sumM2[0] = st->sumM2[1] = 0; st->sumB2[0] = st->sumB2[1] = 0; st->sumMB[0] = st->sumMB[1] = 0;
    }
    if (a.trace && a.trace_begin + t < a.trace_cap) {
        a.trace[2 * (a.trace_begin + t)] = M;
        a.trace[2 * (a.trace_begin + t) + 1] = B;
    }
}

template <int MODE, bool GATE>
__device__ __forceinline__ void colour_pass(const DevFilm& f, int c, unsigned long long sweep,
                                            const uint32_t* tab, uint32_t gthr, int per_row,
                                            int items, long long& dM, long long& dB) {
    const int stride = gridDim.x * blockDim.x;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += stride) {
        const int row = it / per_row;
        const int w = it - row * per_row;
        const int z = row / f.Rh;
        const int j = row - z * f.Rh;
        if (MODE == MODE_INT8) chunk_int8<GATE>(f, c, z, j, w, sweep, tab, gthr, dM, dB);
        else if (MODE == MODE_GENERIC) block_generic<GATE>(f, c, z, j, w, sweep, tab, gthr, dM, dB);
        else word_packed<GATE>(f, c, z, j, w, sweep, tab, gthr, dM, dB);
    }
}

template <int MODE>
__global__ void __launch_bounds__(kBlock) k_sweep(const __grid_constant__ SweepArgs a) {
    __shared__ uint32_t tab[128];
    __shared__ uint32_t gate_s;
    __shared__ long long red[2][32];
    __shared__ int ok_s;
    const DevFilm& f = a.f;
    FilmState* st = a.st;
    const unsigned G = gridDim.x;
    unsigned gen = 0;
    if (threadIdx.x == 0 && G > 1) gen = *reinterpret_cast<const volatile unsigned*>(&st->bar_gen);
    const int per_row = MODE == MODE_INT8 ? f.nck : (MODE == MODE_GENERIC ? f.Qw : f.nw);
    const int items = f.L * f.Rh * per_row;
    int k = a.k0, pos = a.pos0;
    load_table<MODE>(a, k, tab, &gate_s);
    for (long long t = 0; t < a.nsweeps; ++t) {
        if (pos == a.step_total[k]) {
            ++k;
            pos = 0;
            load_table<MODE>(a, k, tab, &gate_s);
        }
        const unsigned long long sweep = (unsigned long long)(a.sweep0 + t + 1);
        const uint32_t gthr = gate_s;
        long long dM = 0, dB = 0;
        for (int c = 0; c < 4; ++c) {
            if (a.use_gate) colour_pass<MODE, true>(f, c, sweep, tab, gthr, per_row, items, dM, dB);
            else colour_pass<MODE, false>(f, c, sweep, tab, gthr, per_row, items, dM, dB);
            if (c == 3) {
                dM = warp_sum(dM);
                dB = warp_sum(dB);
                const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
                if (lane == 0) { red[0][wid] = dM; red[1][wid] = dB; }
                __syncthreads();
                if (wid == 0) {
                    const int nw = blockDim.x >> 5;
                    dM = lane < nw ? red[0][lane] : 0;
                    dB = lane < nw ? red[1][lane] : 0;
                    dM = warp_sum(dM);
                    dB = warp_sum(dB);
                    if (lane == 0 && (dM | dB)) {
                        unsigned long long* acc = reinterpret_cast<unsigned long long*>(&st->acc[sweep & 1][0]);
                        atomicAdd(acc, (unsigned long long)dM);
                        atomicAdd(acc + 1, (unsigned long long)dB);
                    }
                }
            }
            if (!grid_barrier(st, G, gen, &ok_s)) return;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) fold_sweep(a, k, pos, sweep, t);
        ++pos;
    }
}

template <int MODE>
int launch_mode(const SweepArgs& a, int ctas, int threads, cudaStream_t s) {
    if (ctas <= 1) {
        k_sweep<MODE><<<1, threads, 0, s>>>(a);
        return (int)cudaGetLastError();
    }
    void* args[] = {const_cast<SweepArgs*>(&a)};
    return (int)cudaLaunchCooperativeKernel((const void*)k_sweep<MODE>, dim3(ctas), dim3(threads), args, 0, s);
}

template <int MODE>
int max_ctas_mode(int threads, int* out) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep<MODE>, threads, 0);
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
        case MODE_INT8: return max_ctas_mode<MODE_INT8>(threads, max_ctas);
        case MODE_GENERIC: return max_ctas_mode<MODE_GENERIC>(threads, max_ctas);
        default: return max_ctas_mode<MODE_PACKED>(threads, max_ctas);
    }
}

int sweep_items_per_pass(const DevFilm& f) {
    const int per_row = f.packed ? f.nw : ((f.flags & 7u) ? f.Qw : f.nck);
    return f.L * f.Rh * per_row;
}

}  // namespace isf
