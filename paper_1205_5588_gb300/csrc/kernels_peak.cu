// kernels_peak.cu — integer-issue ceilings of the GPU, measured for the roofline of the sweep
// kernels.  The Metropolis path (Eq. 8) has no contraction, and with the film L2-resident its
// kernels are bound by integer issue; these probes measure that bound on this device, in the
// units the sweep kernels are reported in, with no loads of a film and no barriers:
//   LOP3    independent chains of three-input logic ops: the plain lane-op issue rate;
//   MIX     the integer mix of the sweep kernels' random-number work, one op per instruction:
//           32x32 -> 64-bit multiplies, three-input XOR / majority, 32-bit adds;
//   PHILOX  Philox4x32-10 blocks, four interleaved per thread (the same code the sweeps use);
//   ATTEMPT the whole arithmetic of a bit-packed 32-site word with every random word drawn,
//           in the form the packed sweep uses (8 Philox blocks with precomputed round keys and
//           sweep parts; packed_decide: the bit-sliced neighbour count, the transpose to table
//           offsets, 32 table lookups and carry comparisons, the flip mask, dM and dB).
// Every chain feeds a final value that is stored only when it equals a host-chosen word, so
// nothing is dead code and nothing but that one conditional store touches memory.
#include <cuda_runtime.h>

#include <cstdio>

#include "sweep_core.cuh"
#include "../../include/isingfilm_tuning.h"

namespace isf {
int set_last_error(int code, const char* msg);   // capi.cpp
}

using namespace isf;

namespace {

__device__ uint32_t g_peak_sink[4];

__device__ __forceinline__ uint32_t lop3_xor(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t lop3_maj(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

template <int MODE>
constexpr int max_threads() { return MODE == ISF_PEAK_ATTEMPT ? 512 : 1024; }

template <int MODE>
__global__ void __launch_bounds__(max_threads<MODE>()) k_peak(long long iters, uint32_t seed, uint32_t magic) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t out = 0;
    if (MODE == ISF_PEAK_LOP3) {
        // 8 chains, 32 ops per iteration; each op reads three different chains, so no two ops
        // can be merged into one three-input op
        uint32_t a[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) a[v] = tid * (2u * v + 1u) + seed;
        for (long long i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    a[v] = (v & 1) ? lop3_maj(a[v], a[(v + 1) & 7], a[(v + 3) & 7])
                                   : lop3_xor(a[v], a[(v + 1) & 7], a[(v + 3) & 7]);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < 8; ++v) out ^= a[v];
    } else if (MODE == ISF_PEAK_MIX) {
        // 8 chains of (wide multiply, XOR3, majority, add) = 32 ops per iteration; every result
        // feeds an op of another kind, so each stays one instruction
        uint32_t a[8], b[8], c[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            a[v] = tid * (2u * v + 1u) + seed;
            b[v] = a[v] ^ 0x5bd1e995u;
            c[v] = a[v] + 0x9E3779B9u;
        }
        for (long long i = 0; i < iters; ++i) {
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                uint32_t lo, hi;
                mul_wide(0xD2511F53u, a[v], lo, hi);
                a[v] = lop3_xor(hi, b[v], c[v]);
                c[v] = lop3_maj(lo, c[v], a[v]);
                b[v] = b[v] + lo;
            }
        }
#pragma unroll
        for (int v = 0; v < 8; ++v) out ^= a[v] ^ b[v] ^ c[v];
    } else if (MODE == ISF_PEAK_PHILOX) {
        const uint32_t k0 = seed, k1 = seed ^ 0xA5A5A5A5u;
        uint32_t q = tid * 4u;
        for (long long i = 0; i < iters; ++i) {
            uint4 u[4];
            philox10_xn<4>(q, (uint32_t)i, 0u, 0u, k0, k1, u);
#pragma unroll
            for (int v = 0; v < 4; ++v) out ^= lop3_xor(u[v].x, u[v].y, lop3_xor(u[v].z, u[v].w, 0u));
            q += 0x10000u;
        }
    } else {
        // the packed word update of the sweep kernels, on words made from its own random draws
        __shared__ uint32_t tab[128];
        __shared__ uint32_t gate_s[2];
        // thresholds in 0..63, their negations (the carry form) in 64..127, as the sweeps stage them
        for (int t = threadIdx.x; t < 128; t += blockDim.x) {
            const uint32_t thr = 0x40000000u + (uint32_t)(t & 63) * 0x01000193u;
            tab[t] = t < 64 ? thr : 0u - thr;
        }
        if (threadIdx.x == 0) { gate_s[0] = kAlways; gate_s[1] = kFlagAlwaysDraw | kFlagNoNever; }
        __syncthreads();
        uint32_t rk[20];
        round_keys(seed, seed ^ 0xA5A5A5A5u, rk);
        uint32_t q0 = tid * 8u, S = tid ^ seed;
        int dM = 0, dB = 0;
        for (long long i = 0; i < iters; ++i) {
            // a word's 8 blocks as the packed sweep draws them (sweep-only parts once per sweep)
            const unsigned long long sweep = (unsigned long long)i + 1ull;
            const SweepConst sc = sweep_const(sweep, rk);
            uint4 uf[4], us[4];
            philox10_sc<4>(q0, 0u, sc, rk, uf);
            philox10_sc<4>(q0 + 4, 0u, sc, rk, us);
            const uint32_t up[12] = {uf[0].x, uf[0].y, uf[0].z, uf[0].w, uf[1].x, uf[1].y,
                                     uf[1].z, uf[1].w, uf[2].x, uf[2].y, uf[2].z, uf[2].w};
            const uint32_t V[4] = {uf[3].x, uf[3].y, uf[3].z, uf[3].w & 0x0F0F0F0Fu};
            const uint32_t F = packed_decide<false, true>(S, 0xFFFFFFFFu, up, V, q0, sweep, tab, gate_s[0],
                                                          (gate_s[1] & kFlagAlwaysDraw) != 0, rk[0], rk[1], uf, dM, dB,
                                                          us);
            S ^= F;
            q0 += 0x20000u;
        }
        out = S ^ (uint32_t)dM ^ ((uint32_t)dB << 7);
    }
    if (out == magic) g_peak_sink[tid & 3] = out;
}

template <int MODE>
int launch_peak(int ctas, int threads, long long iters, cudaStream_t s, double* units) {
    if (threads == 0) threads = 256;
    if (threads < 32 || threads > max_threads<MODE>() || threads % 32) return ISF_ERR_ARG;
    if (ctas <= 0) {
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_peak<MODE>, threads, 0);
        if (e != cudaSuccess) return set_last_error(ISF_ERR_CUDA, cudaGetErrorString(e));
        if (per < 1) return set_last_error(ISF_ERR_CUDA, "probe kernel cannot be resident with these threads");
        ctas = sms * per;
    }
    k_peak<MODE><<<ctas, threads, 0, s>>>(iters, 0x2545F491u, 0x0u);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_last_error(ISF_ERR_CUDA, cudaGetErrorString(e));
    const double per_iter = MODE == ISF_PEAK_LOP3 || MODE == ISF_PEAK_MIX ? 32.0 : (MODE == ISF_PEAK_PHILOX ? 4.0 : 32.0);
    *units = (double)ctas * (double)threads * (double)iters * per_iter;
    return ISF_OK;
}

}  // namespace

extern "C" int isf_peak_probe(int32_t mode, int32_t ctas, int32_t threads, int64_t iters, void* cuda_stream,
                              double* units_out) {
    if (!units_out) return set_last_error(ISF_ERR_ARG, "isf_peak_probe: units_out is NULL");
    if (iters < 1 || iters > (int64_t)1 << 40) return set_last_error(ISF_ERR_ARG, "isf_peak_probe: iters out of range");
    if (ctas < 0) return set_last_error(ISF_ERR_ARG, "isf_peak_probe: ctas must be >= 0");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int rc;
    switch (mode) {
        case ISF_PEAK_LOP3: rc = launch_peak<ISF_PEAK_LOP3>(ctas, threads, iters, s, units_out); break;
        case ISF_PEAK_MIX: rc = launch_peak<ISF_PEAK_MIX>(ctas, threads, iters, s, units_out); break;
        case ISF_PEAK_PHILOX: rc = launch_peak<ISF_PEAK_PHILOX>(ctas, threads, iters, s, units_out); break;
        case ISF_PEAK_ATTEMPT: rc = launch_peak<ISF_PEAK_ATTEMPT>(ctas, threads, iters, s, units_out); break;
        default: return set_last_error(ISF_ERR_ARG, "isf_peak_probe: unknown mode");
    }
    if (rc == ISF_ERR_ARG) return set_last_error(ISF_ERR_ARG, "isf_peak_probe: threads must be a multiple of 32 "
                                                              "in 32..1024 (32..512 for ISF_PEAK_ATTEMPT)");
    if (rc) return rc;
    return set_last_error(ISF_OK, "");
}
