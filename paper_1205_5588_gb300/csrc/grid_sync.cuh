// grid_sync.cuh — the grid barrier of the cooperative sweep kernels and the work-item
// numbering they share (kernels_sweep.cu, kernels_words.cu).
#pragma once
#include <cuda_runtime.h>

#include "sweep_core.cuh"

namespace isf {

constexpr unsigned kSpinLimit = 1u << 22;   // ~ seconds of waiting, then give up

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// Barrier over the G co-resident CTAs of a cooperative launch.  The arrival counter only grows
// during a launch (the host zeroes it before each launch): barrier b is passed once it reaches
// b * G.  Thread 0 of each CTA adds 1 with release semantics and polls with acquire loads; the
// wait is bounded, and on expiry the kernel records ISF_ERR_TIMEOUT and every CTA returns.
__device__ __forceinline__ bool grid_barrier(FilmState* st, unsigned G, unsigned& target, int* ok_s) {
    __syncthreads();
    if (G > 1) {
        if (threadIdx.x == 0) {
            int ok = 1;
            target += G;
            red_release_add_u32(&st->bar_count, 1u);
            unsigned spins = 0;
            while ((int)(ld_acquire_u32(&st->bar_count) - target) < 0) {
                ++spins;
                if ((spins & 15u) == 0 && ld_volatile_i32(&st->error)) { ok = 0; break; }
                if (spins > kSpinLimit) {
                    atomicCAS(&st->error, 0, (int)ISF_ERR_TIMEOUT);
                    st->error_where = 1;
                    ok = 0;
                    break;
                }
                if (spins > 64) __nanosleep(32);
            }
            *ok_s = ok;
        }
        __syncthreads();
        return *ok_s != 0;
    }
    return true;
}

// The barrier in two halves, so that work needing no other CTA's writes of the pass (the next
// pass's first random words) can run while thread 0 waits.
__device__ __forceinline__ void grid_arrive(FilmState* st, unsigned G, unsigned& target) {
    __syncthreads();
    if (G > 1 && threadIdx.x == 0) {
        target += G;
        red_release_add_u32(&st->bar_count, 1u);
    }
}
__device__ __forceinline__ bool grid_wait(FilmState* st, unsigned G, unsigned target, int* ok_s) {
    if (G > 1) {
        if (threadIdx.x == 0) {
            int ok = 1;
            unsigned spins = 0;
            while ((int)(ld_acquire_u32(&st->bar_count) - target) < 0) {
                ++spins;
                if ((spins & 15u) == 0 && ld_volatile_i32(&st->error)) { ok = 0; break; }
                if (spins > kSpinLimit) {
                    atomicCAS(&st->error, 0, (int)ISF_ERR_TIMEOUT);
                    st->error_where = 1;
                    ok = 0;
                    break;
                }
                if (spins > 64) __nanosleep(32);
            }
            *ok_s = ok;
        }
        __syncthreads();
        return *ok_s != 0;
    }
    return true;
}

// First work item of this thread in a pass.  Warps are numbered across CTAs first (warp w of
// CTA b is warp w * G + b), so when a pass has fewer items than two per thread, the threads
// that take one more item are spread evenly over all CTAs (and SMs); lanes stay consecutive,
// so a warp still reads consecutive words.
__device__ __forceinline__ int first_item(unsigned G, unsigned cta) {
    return (((int)(threadIdx.x >> 5) * (int)G + (int)cta) << 5) + (int)(threadIdx.x & 31);
}

}  // namespace isf
