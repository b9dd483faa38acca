// device_common.cuh — device helpers shared by the library's kernels: Philox4x32-10, layout
// addressing, the z = 12 stencil with periodic wrap, and small integer utilities.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "isf_internal.h"

namespace isf {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each multiplies counter words
// 0 and 2 by the round constants, swaps the halves, XORs in the key, and the key advances by
// the Weyl increments.  The key is uniform across the grid, so its schedule stays in uniform
// registers.
// One 32x32 -> 64-bit product as a single wide multiply (its low and high words).
__device__ __forceinline__ void mul_wide(uint32_t a, uint32_t b, uint32_t& lo, uint32_t& hi) {
    unsigned long long p;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
    lo = (uint32_t)p;
    hi = (uint32_t)(p >> 32);
}

__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0, hi0, lo1, hi1;
        mul_wide(0xD2511F53u, c.x, lo0, hi0);
        mul_wide(0xCD9E8D57u, c.z, lo1, hi1);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t word_of(const uint4& v, int b) {
    return b == 0 ? v.x : (b == 1 ? v.y : (b == 2 ? v.z : v.w));
}

// Philox counter word of the 4-site block holding column i of row (c, z, j).
__device__ __forceinline__ uint32_t block_counter(const DevFilm& f, int c, int z, int j, int i) {
    if (f.slab) {               // a slab's rows carry the whole film's counters
        int jg = (j + f.cj0) % f.cRh;
        if (jg < 0) jg += f.cRh;
        return (uint32_t)((((int64_t)c * f.L + z) * f.cRh + jg) * f.Qw + (i >> 2));
    }
    return (uint32_t)((((int64_t)c * f.L + z) * f.Rh + j) * f.Qw + (i >> 2));
}

__device__ __forceinline__ int colour_of(int x, int y, int z) {
    return ((x + z) & 1) | (((y + z) & 1) << 1);
}

// Byte address (int8 layout) / word index (packed layout) of column i, row j, layer z, colour c.
__device__ __forceinline__ int64_t addr8(const DevFilm& f, int c, int z, int j, int i) {
    return (int64_t)c * f.cs8 + (int64_t)(z + 1) * f.ls8 + (int64_t)(j + 1) * f.P + 16 + i;
}
__device__ __forceinline__ int64_t addrw(const DevFilm& f, int c, int z, int j, int w) {
    return (int64_t)c * f.csw + (int64_t)(z + 1) * f.lsw + (int64_t)(j + 1) * f.Wp + 1 + w;
}

__device__ __forceinline__ bool site_occupied(const DevFilm& f, int x, int y, int z) {
    return z < (int)f.heights[(int64_t)y * f.C + x];
}

// Spin S in {-1, 0 (vacancy), +1} of an in-range site, read from the film's layout.
__device__ __forceinline__ int site_spin(const DevFilm& f, int x, int y, int z) {
    const int c = colour_of(x, y, z), i = x >> 1, j = y >> 1;
    if (!f.packed) return (int)f.s8[addr8(f, c, z, j, i)] - 1;
    const int64_t a = addrw(f, c, z, j, i >> 5);
    const uint32_t bit = 1u << (i & 31);
    if (!(f.op[a] & bit)) return 0;
    return (f.sp[a] & bit) ? 1 : -1;
}

// Neighbour k of (x, y, z) with periodic wrap where flagged; false outside an open boundary.
__device__ __forceinline__ bool neighbour_of(const DevFilm& f, int x, int y, int z, int k,
                                             int& a, int& b, int& c) {
    // (+-1,0,0), (0,+-1,0), +-(1,-1,0); up (0,0,1), (0,-1,1), (-1,0,1); down (0,0,-1), (0,1,-1), (1,0,-1)
    const int dx[12] = {1, -1, 0, 0, 1, -1, 0, 0, -1, 0, 0, 1};
    const int dy[12] = {0, 0, 1, -1, -1, 1, 0, -1, 0, 0, 1, 0};
    const int dz[12] = {0, 0, 0, 0, 0, 0, 1, 1, 1, -1, -1, -1};
    a = x + dx[k];
    b = y + dy[k];
    c = z + dz[k];
    if (a < 0 || a >= f.C) {
        if (!(f.flags & 1u)) return false;
        a = (a + f.C) % f.C;
    }
    if (b < 0 || b >= f.R) {
        if (!(f.flags & 2u)) return false;
        b = (b + f.R) % f.R;
    }
    if (c < 0 || c >= f.L) {
        if (!(f.flags & 4u)) return false;
        c = (c + f.L) % f.L;
    }
    return true;
}

// Thread-block cluster: this CTA's rank, and a barrier over every thread of the cluster whose
// release / acquire orders all earlier memory operations (shared, distributed shared and
// global) before everything after it in the other CTAs.
__device__ __forceinline__ unsigned cluster_ctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    return v;
}

}  // namespace isf
