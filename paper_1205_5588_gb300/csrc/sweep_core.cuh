// sweep_core.cuh — the per-site Metropolis update (Eq. 8; the Eq. 9 gate of items 4-5 of
// Sec. 5), shared by the global-memory and the cluster-resident sweep kernels, plus the
// step-table staging and the per-sweep fold of M, B into the step's exact sums.
#pragma once
#include <cuda_runtime.h>

#include "../../include/isingfilm.h"
#include "device_common.cuh"

namespace isf {

// Table of the current step in shared memory, indexed by the per-site byte a pass forms:
//   int8   : (stored byte << 5) | (n + 12), stored byte 0 = down, 1 = vacancy, 2 = up;
//            vacancies map to 0 ("never"), so they never flip and never draw a random word
//   packed : (up << 5) | (n + 12); the packed kernel masks vacant sites out of the flips itself.
//            Entries 64..127 hold the same thresholds negated, 2^32 - thr ("always": 0), for
//            the carry form of the comparison (kFlagNoNever).
// INT8_NEG (int8 kernels that take the carry form): on steps with kFlagNoNever the int8 entries
// are negated the same way (vacancies stay 0; the kernel masks them out of the flips).
__device__ __forceinline__ uint32_t neg_threshold(uint32_t thr) { return thr == kAlways ? 0u : 0u - thr; }
template <bool PACKED, bool INT8_NEG = false>
__device__ __forceinline__ void stage_table(const uint32_t* tables, int k, uint32_t* tab, uint32_t* gate) {
    const uint32_t* src = tables + (size_t)k * kTableStride;
    const bool neg8 = INT8_NEG && (src[kFlagSlot] & kFlagNoNever);
    for (int t = threadIdx.x; t < 128; t += blockDim.x) {
        uint32_t v = 0;
        const int X = t & 31;
        if (X <= 24) {
            if (PACKED) {
                const uint32_t thr = src[X * 2 + ((t >> 5) & 1)];
                v = t < 64 ? thr : neg_threshold(thr);
            } else {
                const int sb = t >> 5;
                if (sb == 0) v = src[X * 2 + 0];
                else if (sb == 2) v = src[X * 2 + 1];
                if (neg8 && (sb == 0 || sb == 2)) v = neg_threshold(v);
            }
        }
        tab[t] = v;
    }
    if (threadIdx.x == 0) {
        gate[0] = src[kGateSlot];
        gate[1] = src[kFlagSlot];
    }
    __syncthreads();
}

// accept iff u < thr, or thr == always (min keeps u = 2^32-1 below always)
__device__ __forceinline__ bool metropolis_accept(uint32_t u, uint32_t thr) { return min(u, 0xFFFFFFFEu) < thr; }
// a random word decides the site only when thr is neither 0 ("never") nor always
__device__ __forceinline__ bool needs_word(uint32_t thr) { return (thr - 1u) < 0xFFFFFFFEu; }

__device__ __forceinline__ uint4 ld16(const uint8_t* p) { return *reinterpret_cast<const uint4*>(p); }
__device__ __forceinline__ uint32_t ld4(const uint8_t* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ void add4(uint4& a, const uint4& b) {
    a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
}

// Eq. 9 gate for the accepted lanes of one 4-site block (stream 1): clears the lanes that fail.
__device__ __forceinline__ uint32_t gate_block(uint32_t lanes, uint32_t gthr, uint32_t q,
                                               unsigned long long sweep, uint32_t key0, uint32_t key1) {
    if (!lanes || gthr == kAlways) return lanes;
    if (gthr == 0u) return 0u;
    const uint4 g = philox10(make_uint4(q, (uint32_t)sweep, (uint32_t)(sweep >> 32), 1u), key0, key1);
    uint32_t keep = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
        if (metropolis_accept(word_of(g, b), gthr)) keep |= 1u << b;
    return lanes & keep;
}

// Rejected-lane bits of the carry form of the comparison: with neg = 2^32 - thr (0 for
// "always"), u + neg carries out exactly when u >= thr, i.e. when the flip is rejected; the carry
// is shifted in below R (R = 2R + carry).
__device__ __forceinline__ uint32_t shift_in_reject(uint32_t R, uint32_t u, uint32_t neg) {
    uint32_t out;
    asm("{\n\t.reg .u32 t;\n\tadd.cc.u32 t, %1, %2;\n\taddc.u32 %0, %3, %3;\n\t}"
        : "=r"(out) : "r"(u), "r"(neg), "r"(R));
    return out;
}

// NW Philox4x32-10 blocks at consecutive counters, interleaved so that their dependency chains
// overlap (same rounds as philox10).
template <int NW>
__device__ __forceinline__ void philox10_xn(uint32_t q0, uint32_t s_lo, uint32_t s_hi, uint32_t stream,
                                            uint32_t k0, uint32_t k1, uint4 out[NW]) {
    uint32_t c0[NW], c1[NW], c2[NW], c3[NW];
#pragma unroll
    for (int v = 0; v < NW; ++v) { c0[v] = q0 + v; c1[v] = s_lo; c2[v] = s_hi; c3[v] = stream; }
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#pragma unroll
        for (int v = 0; v < NW; ++v) {
            uint32_t lo0, hi0, lo1, hi1;
            mul_wide(0xD2511F53u, c0[v], lo0, hi0);
            mul_wide(0xCD9E8D57u, c2[v], lo1, hi1);
            c0[v] = hi1 ^ c1[v] ^ k0;
            c1[v] = lo1;
            c2[v] = hi0 ^ c3[v] ^ k1;
            c3[v] = lo0;
        }
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
#pragma unroll
    for (int v = 0; v < NW; ++v) out[v] = make_uint4(c0[v], c1[v], c2[v], c3[v]);
}

// Philox4x32-10 with its round keys precomputed (rk[2r], rk[2r+1]: the key of round r) and the
// parts of rounds 1 and 2 that depend on the sweep only (the counter's words 1 and 2 are the
// sweep, word 0 varies), computed once per sweep: the same blocks as philox10_xn.
struct SweepConst {
    uint32_t A, B;      // counter words 0 and 1 after round 1
    uint32_t C, D;      // high and low words of M0 * A (round 2)
};
__device__ __forceinline__ void round_keys(uint32_t k0, uint32_t k1, uint32_t (&rk)[20]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
        rk[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
}
__device__ __forceinline__ SweepConst sweep_const(unsigned long long sweep, const uint32_t (&rk)[20]) {
    SweepConst sc;
    uint32_t lo, hi;
    mul_wide(0xCD9E8D57u, (uint32_t)(sweep >> 32), lo, hi);
    sc.A = hi ^ (uint32_t)sweep ^ rk[0];
    sc.B = lo;
    mul_wide(0xD2511F53u, sc.A, sc.D, sc.C);
    return sc;
}
template <int NW>
__device__ __forceinline__ void philox10_sc(uint32_t q0, uint32_t stream, const SweepConst& sc,
                                            const uint32_t (&rk)[20], uint4 out[NW]) {
    uint32_t c0[NW], c1[NW], c2[NW], c3[NW];
#pragma unroll
    for (int v = 0; v < NW; ++v) {
        uint32_t lo0, hi0, lo1, hi1;
        mul_wide(0xD2511F53u, q0 + v, lo0, hi0);          // round 1; its other half is sc.A, sc.B
        mul_wide(0xCD9E8D57u, hi0 ^ stream ^ rk[1], lo1, hi1);   // round 2; M0 * sc.A = sc.C:sc.D
        c0[v] = hi1 ^ sc.B ^ rk[2];
        c1[v] = lo1;
        c2[v] = sc.C ^ lo0 ^ rk[3];
        c3[v] = sc.D;
    }
#pragma unroll
    for (int r = 2; r < 10; ++r) {
#pragma unroll
        for (int v = 0; v < NW; ++v) {
            uint32_t lo0, hi0, lo1, hi1;
            mul_wide(0xD2511F53u, c0[v], lo0, hi0);
            mul_wide(0xCD9E8D57u, c2[v], lo1, hi1);
            c0[v] = hi1 ^ c1[v] ^ rk[2 * r];
            c1[v] = lo1;
            c2[v] = hi0 ^ c3[v] ^ rk[2 * r + 1];
            c3[v] = lo0;
        }
    }
#pragma unroll
    for (int v = 0; v < NW; ++v) out[v] = make_uint4(c0[v], c1[v], c2[v], c3[v]);
}

// The Metropolis decisions of one 4*NW-site chunk (NW words) of an int8 colour row (Eq. 8; Eq. 9
// gate).
// Sw: the chunk's 4 words of stored bytes (S + 1: 0 down, 1 vacancy, 2 up); Aw: per byte the
// sum of the 12 neighbour bytes, n + 12.  All 16 table lookups first; then, if any lane's
// threshold is neither 0 nor "always", the chunk's NW Philox blocks at once (a real word
// decides a 0 / "always" lane exactly as no word does, so computing it never changes a
// result).  The flips come back as a byte mask per word (0 <-> 2 is XOR 2).  PX: lanes past the
// row end (column Ch on) are masked.  Returns the OR of the four masks.
// U_IN: the chunk's NW Philox blocks are already in u_in (drawn before the neighbour sum was
// available, to fill the wait for its loads); else they are drawn here only if a lane needs one.
// neg (steps with kFlagNoNever, tables staged with INT8_NEG; not with PX): the table holds
// 2^32 - thr and each lane's rejection is the carry of u + that (shift_in_reject), vacant lanes
// masked out afterwards.
// dM, dB: a signed byte per lane (+1 for a flip from down, -1 from up) dotted with all-ones and
// with Aw gives #down - #up flips and the same sum of n + 12; dM = 2 (#down - #up),
// dB = 2 [sum over down-flips of n - sum over up-flips of n].
template <bool GATE, bool PX, int NW = 4, bool U_IN = false>
__device__ __forceinline__ uint32_t decide16(const uint32_t Sw[NW], const uint32_t Aw[NW], uint32_t q0,
                                             unsigned long long sweep, const uint32_t* tab, uint32_t gthr,
                                             uint32_t key0, uint32_t key1, int i0, int Ch, uint32_t fm[NW],
                                             int& dM, int& dB, const uint4* u_in = nullptr, bool neg = false) {
    uint32_t thr[4 * NW];
    bool need = false;
#pragma unroll
    for (int v = 0; v < NW; ++v) {
        const uint32_t iw = (Sw[v] << 5) + Aw[v];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            uint32_t t = tab[__byte_perm(iw, 0u, 0x4440u + b)];
            if (PX && i0 + 4 * v + b >= Ch) t = 0u;
            thr[4 * v + b] = t;
            // negated entries: 0 is "always" (or a vacancy), and no lane is "never"
            if (!U_IN) need |= neg ? t != 0u : needs_word(t);
        }
    }
    uint4 u[NW];
    if (U_IN) {
#pragma unroll
        for (int v = 0; v < NW; ++v) u[v] = u_in[v];
    } else {
#pragma unroll
        for (int v = 0; v < NW; ++v) u[v] = make_uint4(0, 0, 0, 0);
        if (need) philox10_xn<NW>(q0, (uint32_t)sweep, (uint32_t)(sweep >> 32), 0u, key0, key1, u);
    }
    uint32_t any = 0;
    int dn = 0, dx = 0;     // #down - #up flips; sum of n + 12 over down-flips minus over up-flips
#pragma unroll
    for (int v = 0; v < NW; ++v) {
        uint32_t m;
        if (!PX && neg) {
            // rejection bits, lane 3 shifted in first (bit b = lane b); bit b -> bit 8b + 1 by one
            // multiply (the partial products do not overlap); accepted lanes of occupied sites
            // (stored byte 1 has bit 1 set once shifted) become bytes 2
            uint32_t R = shift_in_reject(0u, u[v].w, thr[4 * v + 3]);
            R = shift_in_reject(R, u[v].z, thr[4 * v + 2]);
            R = shift_in_reject(R, u[v].y, thr[4 * v + 1]);
            R = shift_in_reject(R, u[v].x, thr[4 * v + 0]);
            m = ~(R * 0x00408102u) & ~(Sw[v] << 1) & 0x02020202u;
        } else {
            m = (metropolis_accept(u[v].x, thr[4 * v + 0]) ? 0x00000002u : 0u) |
                (metropolis_accept(u[v].y, thr[4 * v + 1]) ? 0x00000200u : 0u) |
                (metropolis_accept(u[v].z, thr[4 * v + 2]) ? 0x00020000u : 0u) |
                (metropolis_accept(u[v].w, thr[4 * v + 3]) ? 0x02000000u : 0u);
        }
        if (GATE && m) {
            uint32_t lanes = ((m >> 1) & 1u) | ((m >> 8) & 2u) | ((m >> 15) & 4u) | ((m >> 22) & 8u);
            lanes = gate_block(lanes, gthr, q0 + v, sweep, key0, key1);
            m = ((lanes & 1u) << 1) | ((lanes & 2u) << 8) | ((lanes & 4u) << 15) | ((lanes & 8u) << 22);
        }
        // byte of sg: 1 where a down spin flips, 0xFF (-1) where an up spin flips (bytes of up are
        // 0 or 2, so up * 0x7F stays within each byte)
        const uint32_t up = m & Sw[v];
        const uint32_t sg = (m >> 1) ^ (up * 0x7Fu);
        dn = __dp4a((int)sg, 0x01010101, dn);
        dx = __dp4a((int)sg, (int)Aw[v], dx);
        fm[v] = m;
        any |= m;
    }
    dM += 2 * dn;
    dB += 2 * dx - 24 * dn;
    return any;
}

// One 16-site chunk, neighbours through generic pointers (global-memory kernel).
template <bool GATE>
__device__ __forceinline__ void update_chunk16(uint8_t* own, const uint8_t* const* nb, int sgn, uint32_t q0,
                                               unsigned long long sweep, const uint32_t* tab, uint32_t gthr,
                                               uint32_t key0, uint32_t key1, int i0, int Ch,
                                               int& dM, int& dB, bool neg) {
    const uint4 S = ld16(own);
    // the 15 neighbour loads first, then the chunk's four Philox blocks while they are in flight
    uint4 v[12];
    uint32_t e[3];
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = ld16(nb[k]);
#pragma unroll
    for (int k = 9; k < 12; ++k) e[k - 9] = ld4(sgn < 0 ? nb[k] - 4 : nb[k] + 16);
    uint4 u[4];
    philox10_xn<4>(q0, (uint32_t)sweep, (uint32_t)(sweep >> 32), 0u, key0, key1, u);
    uint4 acc = v[0];
#pragma unroll
    for (int k = 1; k < 9; ++k) add4(acc, v[k]);
    if (sgn < 0) {
#pragma unroll
        for (int k = 9; k < 12; ++k)
            add4(acc, make_uint4(__funnelshift_l(e[k - 9], v[k].x, 8), __funnelshift_l(v[k].x, v[k].y, 8),
                                 __funnelshift_l(v[k].y, v[k].z, 8), __funnelshift_l(v[k].z, v[k].w, 8)));
    } else {
#pragma unroll
        for (int k = 9; k < 12; ++k)
            add4(acc, make_uint4(__funnelshift_r(v[k].x, v[k].y, 8), __funnelshift_r(v[k].y, v[k].z, 8),
                                 __funnelshift_r(v[k].z, v[k].w, 8), __funnelshift_r(v[k].w, e[k - 9], 8)));
    }
    const uint32_t Sw[4] = {S.x, S.y, S.z, S.w};
    const uint32_t Aw[4] = {acc.x, acc.y, acc.z, acc.w};
    uint32_t fm[4];
    if (decide16<GATE, false, 4, true>(Sw, Aw, q0, sweep, tab, gthr, key0, key1, i0, Ch, fm, dM, dB, u, neg))
        *reinterpret_cast<uint4*>(own) = make_uint4(Sw[0] ^ fm[0], Sw[1] ^ fm[1], Sw[2] ^ fm[2], Sw[3] ^ fm[3]);
}

// ---- packed layout: one 32-site word ----------------------------------------------------
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

// The Metropolis decisions of one 32-site word of the packed layout (Eq. 8; the Eq. 9 gate):
// S, O: the word's spin and occupancy bits; up: the 12 neighbours' up bits per lane; V: the
// bit-sliced count of vacant neighbours.  X = n + 12 = 2 (#up) + (#vacant) as 5 bit-planes; an
// 8x32 bit-plane transpose gives each lane its table entry's byte offset; u_first: the word's
// first four Philox blocks (lanes 0-15), drawn by the caller; u_second (may be null): the last
// four (lanes 16-31) when the caller drew them too, else they are drawn here when a lane needs
// them.  CARRY (steps without a "never" threshold, no gate): each lane's decision is the carry of
// u + (2^32 - thr), shifted into a rejection mask (two instructions a lane instead of a minimum,
// a compare, a select and an or), in four independent 8-lane chains (highest lane first, so that
// chain j ends with lane 8j + i in bit i) joined at the end.  Returns the flip mask (vacant
// lanes cleared) and adds the flips' dM, dB.
template <bool GATE, bool CARRY = false>
__device__ __forceinline__ uint32_t packed_decide(uint32_t S, uint32_t O, const uint32_t up[12], const uint32_t V[4],
                                                  uint32_t q0, unsigned long long sweep, const uint32_t* tab,
                                                  uint32_t gthr, bool always_draw, uint32_t key0, uint32_t key1,
                                                  const uint4 (&u_first)[4], int& dM, int& dB,
                                                  const uint4* u_second = nullptr) {
    // X = n + 12 = 2 * (#up) + (#vacant) over the 12 neighbours, 5 bit-planes
    uint32_t U0, U1, U2, U3;
    popcount12(up, U0, U1, U2, U3);
    const uint32_t V0 = V[0], V1 = V[1], V2 = V[2], V3 = V[3];
    uint32_t X[5], k2, k3;
    X[0] = V0;
    X[1] = U0 ^ V1;
    const uint32_t k1 = U0 & V1;
    full_add(U1, V2, k1, X[2], k2);
    full_add(U2, V3, k2, X[3], k3);
    X[4] = U3 ^ k3;
    // transpose the 8 planes {0, 0, X0..X4, S}: byte k of P[r] = 4 x the table index
    // (up << 5) | X of lane 8k + r, i.e. its byte offset in the table
    uint32_t P[8] = {0u, 0u, X[0], X[1], X[2], X[3], X[4], S};
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
    static_assert(!(GATE && CARRY), "the gate needs the accepted lanes of each block");
    uint32_t F = 0;
    uint32_t R[4] = {0u, 0u, 0u, 0u};       // CARRY: rejected lanes 8j..8j+7 of chain j
    const uint8_t* tabb = reinterpret_cast<const uint8_t*>(tab) + (CARRY ? 256 : 0);
    // two halves of 16 lanes (4 Philox blocks each): all 16 lookups first, then the half's four
    // blocks interleaved when any of its lanes needs a word
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        uint32_t thr[16];
        bool need = false;
#pragma unroll
        for (int vv = 0; vv < 4; ++vv) {
            const int v = 4 * g + vv;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                // byte v >> 1 of the transposed word, zero-extended (one byte permute)
                const uint32_t t = *reinterpret_cast<const uint32_t*>(
                    tabb + __byte_perm(P[4 * (v & 1) + b], 0u, 0x4440u + (uint32_t)(v >> 1)));
                thr[4 * vv + b] = t;
            }
        }
        // the second half draws its words only if a lane needs one (unless the step's table
        // says nearly every group does, or the caller drew them)
        if (g) {
            if (always_draw || u_second) {
                need = true;
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) need |= CARRY ? thr[i] != 0u : needs_word(thr[i]);
            }
        }
        uint4 u[4];
        if (g == 0) {
#pragma unroll
            for (int vv = 0; vv < 4; ++vv) u[vv] = u_first[vv];
        } else if (u_second) {
#pragma unroll
            for (int vv = 0; vv < 4; ++vv) u[vv] = u_second[vv];
        } else {
#pragma unroll
            for (int vv = 0; vv < 4; ++vv) u[vv] = make_uint4(0, 0, 0, 0);
            if (need) philox10_xn<4>(q0 + 4, (uint32_t)sweep, (uint32_t)(sweep >> 32), 0u, key0, key1, u);
        }
        if (CARRY) {
            // lanes 16g + 4vv + b; chain 2g + (vv >> 1) takes its 8 lanes from the highest down
#pragma unroll
            for (int i = 7; i >= 0; --i) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int vv = 2 * h + (i >> 2), b = i & 3;
                    R[2 * g + h] = shift_in_reject(R[2 * g + h], word_of(u[vv], b), thr[4 * vv + b]);
                }
            }
        } else {
#pragma unroll
            for (int vv = 0; vv < 4; ++vv) {
                uint32_t lanes = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (metropolis_accept(word_of(u[vv], b), thr[4 * vv + b])) lanes |= 1u << b;
                if (GATE) lanes = gate_block(lanes, gthr, q0 + 4 * g + vv, sweep, key0, key1);
                F |= lanes << (4 * (4 * g + vv));
            }
        }
    }
    if (CARRY) F = ~(R[0] | (R[1] << 8) | (R[2] << 16) | (R[3] << 24));
    F &= O;                     // vacant sites never flip
    if (F) {
        const uint32_t Fu = F & S, Fd = F & ~S;        // flipped up -> down, down -> up
        const int nu = __popc(Fu), nd = __popc(Fd);
        int xu = 0, xd = 0;
#pragma unroll
        for (int p = 0; p < 5; ++p) {
            xu += __popc(X[p] & Fu) << p;
            xd += __popc(X[p] & Fd) << p;
        }
        dM += -2 * (nu - nd);
        dB += -2 * ((xu - 12 * nu) - (xd - 12 * nd));
    }
    return F;
}

// ---- packed layout: the loads of one 32-site word -------------------------------------------
// Loads of one packed word position: the own spin and occupancy words, the 12 neighbour spin
// words (three of them shifted by one column, completed from the word before or after) as the
// neighbours' up bits, and the position's precomputed bit-sliced count V of vacant neighbours.
// NARROW: every offset fits 32 bits, so each address is one 32-bit offset from the own word's
// pointer.
template <bool NARROW>
__device__ __forceinline__ void packed_loads(const DevFilm& f, const NbrClass& nc, int64_t base, uint32_t& S,
                                             uint32_t& O, uint32_t up[12]) {
    const uint32_t* spb = f.sp + base;
    auto off = [&](int k) -> int64_t { return NARROW ? (int64_t)(int32_t)nc.off[k] : nc.off[k]; };
    S = spb[0];
    O = f.op[base];
#pragma unroll
    for (int k = 0; k < 9; ++k) up[k] = spb[off(k)];
    if (nc.sgn < 0) {
#pragma unroll
        for (int k = 9; k < 12; ++k) up[k] = __funnelshift_l(spb[off(k) - 1], spb[off(k)], 1);
    } else {
#pragma unroll
        for (int k = 9; k < 12; ++k) up[k] = __funnelshift_r(spb[off(k)], spb[off(k) + 1], 1);
    }
}

// Walks a thread's work items it, it + T, it + 2T, ... of a pass laid out as (z, row, chunk)
// with nc chunks per row and nr rows per layer, by carries instead of divisions.
struct ItemWalk {
    int ck, jr, z;              // current item
    int dck, djr, dz;           // the stride T split the same way
    int nc, nr;
    __device__ __forceinline__ void init(int it, int T, int nc_, int nr_) {
        nc = nc_; nr = nr_;
        ck = it % nc; const int rz = it / nc; jr = rz % nr; z = rz / nr;
        dck = T % nc; const int drz = T / nc; djr = drz % nr; dz = drz / nr;
    }
    __device__ __forceinline__ void next() {
        ck += dck;
        int carry = 0;
        if (ck >= nc) { ck -= nc; carry = 1; }
        jr += djr + carry;
        z += dz;
        if (jr >= nr) { jr -= nr; z += 1; }
    }
};

// Running film state kept in shared memory by the one folding thread for a whole launch;
// loaded from and stored to the FilmState at the launch's start and end, so a sweep's fold
// costs no device-memory round trip.
struct RunState {
    long long M, B, n_meas, sumM, sumAbsM, sumB;
    unsigned __int128 sumM2, sumB2, sumMB;
};

__device__ __forceinline__ void load_run_state(const FilmState* st, RunState& r) {
    r.M = st->M; r.B = st->B; r.n_meas = st->n_meas;
    r.sumM = st->sumM; r.sumAbsM = st->sumAbsM; r.sumB = st->sumB;
    r.sumM2 = (unsigned __int128)st->sumM2[1] << 64 | st->sumM2[0];
    r.sumB2 = (unsigned __int128)st->sumB2[1] << 64 | st->sumB2[0];
    r.sumMB = (unsigned __int128)st->sumMB[1] << 64 | st->sumMB[0];
}

__device__ __forceinline__ void store_run_state(FilmState* st, const RunState& r) {
    st->M = r.M; st->B = r.B; st->n_meas = r.n_meas;
    st->sumM = r.sumM; st->sumAbsM = r.sumAbsM; st->sumB = r.sumB;
    st->sumM2[0] = (unsigned long long)r.sumM2; st->sumM2[1] = (unsigned long long)(r.sumM2 >> 64);
    st->sumB2[0] = (unsigned long long)r.sumB2; st->sumB2[1] = (unsigned long long)(r.sumB2 >> 64);
    st->sumMB[0] = (unsigned long long)r.sumMB; st->sumMB[1] = (unsigned long long)(r.sumMB >> 64);
}

// Fold one sweep's (dM, dB) into M, B and the current step's exact sums; write the step's
// record after its last sweep; keep the trace.  Single thread, stores only.
__device__ __forceinline__ void fold_sweep(const SweepArgs& a, RunState& r, int k, int pos, int step_eq,
                                           int step_total, long long dM, long long dB, long long t) {
    r.M += dM;
    r.B += dB;
    const long long M = r.M, B = r.B;
    if (pos >= step_eq) {
        r.n_meas += 1;
        r.sumM += M;
        r.sumAbsM += M < 0 ? -M : M;
        r.sumB += B;
        r.sumM2 += (unsigned __int128)((__int128)M * M);
        r.sumB2 += (unsigned __int128)((__int128)B * B);
        r.sumMB += (unsigned __int128)((__int128)M * B);
    }
    if (pos + 1 == step_total) {
        StepRec rec;
        rec.M_last = M; rec.B_last = B; rec.n_meas = r.n_meas;
        rec.sumM = r.sumM; rec.sumAbsM = r.sumAbsM; rec.sumB = r.sumB;
        rec.sumM2[0] = (unsigned long long)r.sumM2; rec.sumM2[1] = (unsigned long long)(r.sumM2 >> 64);
        rec.sumB2[0] = (unsigned long long)r.sumB2; rec.sumB2[1] = (unsigned long long)(r.sumB2 >> 64);
        rec.sumMB[0] = (unsigned long long)r.sumMB; rec.sumMB[1] = (unsigned long long)(r.sumMB >> 64);
        a.recs[k] = rec;
        r.n_meas = 0; r.sumM = 0; r.sumAbsM = 0; r.sumB = 0;
        r.sumM2 = 0; r.sumB2 = 0; r.sumMB = 0;
    }
    if (a.trace && a.trace_begin + t < a.trace_cap) {
        a.trace[2 * (a.trace_begin + t)] = M;
        a.trace[2 * (a.trace_begin + t) + 1] = B;
    }
}

// Block-wide sum of (dM, dB); the result is valid in thread 0.  red: 64 long longs of smem.
__device__ __forceinline__ void block_sum2(long long& dM, long long& dB, long long* red) {
    dM = warp_sum(dM);
    dB = warp_sum(dB);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[wid] = dM; red[32 + wid] = dB; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        dM = lane < nw ? red[lane] : 0;
        dB = lane < nw ? red[32 + lane] : 0;
        dM = warp_sum(dM);
        dB = warp_sum(dB);
    }
}

}  // namespace isf
