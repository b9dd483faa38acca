// kernels_slabs.cu — Metropolis sweeps (Eq. 8; the Eq. 9 gate of items 4-5 of Sec. 5) of a
// packed film split by rows over the CTAs of one cooperative launch, each CTA holding its band
// of rows in shared memory: the paper's decomposition of the image into bands of rows, one per
// process, with the rows next to a neighbour's band exchanged between updates (Sec. 3, list
// items 1-2), here with CTAs as the processes and device memory as the channel.
//
// Shared memory of CTA r (rows [part[r], part[r+1]) of every colour, nr of them): per colour c,
// layer index zz = z + 1 (0 and L + 1 are the vacant layers outside the film), local row jj
// (0: the row below the band, 1..nr: own rows, nr + 1: the row above) and word index ww
// (0 and nw + 1: vacant padding), one uint2 {spin bits, occupancy bits} per 32-site word.  The
// 12 neighbour offsets of each (colour, layer parity) class are the device-memory layout's with
// these strides, so the word update is the global kernel's, reading shared memory; a word's
// vacant-neighbour count comes from its list entry's precomputed record.
//
// Colour pass P (colour c = P mod 4) on CTA r:
//   - the warps take r's occupied words of colour c 32 at a time from a shared counter, the two
//     boundary rows' words first: their new spin words also go to r's xbuf, and after each such
//     chunk its lane 0 adds the chunk's boundary word count to done[r] (release);
//   - warp 0, once the boundary words are handed out, waits until each neighbour's done counter
//     shows all its boundary words of pass P (acquire) and copies its boundary rows of colour c
//     into r's halo row on that side; pass P does not read colour c's halo, so the copy may run
//     while the other warps still update;
//   - a CTA barrier ends the pass.
// Pass P + 1's boundary words read the halo imported in pass P, so a CTA is never more than one
// pass ahead of a neighbour and one xbuf row per colour and side suffices.  There is no grid
// barrier, and a neighbour's boundary rows are ready early in its pass, so the wait is short.
//
// Observables: every CTA adds its (dM, dB) of sweep t to series[t]; launch_fold_series then folds
// the series into M, B and the step sums in sweep order (the same fold as the other kernels).
#include <cuda_runtime.h>

#include "sweep_core.cuh"

namespace isf {

namespace {

constexpr int kSlabBlock = 512;              // threads per CTA (<= 128 registers per thread)
constexpr unsigned kNbrSpinLimit = 1u << 22; // polls of a neighbour's counter (~ seconds)

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_gpu(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct SlabGeom {
    int G, r, jr0, jr1, nr;
    int Wp, nw, L;
    int ls, cs;                 // shared-memory layer and colour strides (words)
    int per;                    // words of one boundary row over all layers (L * nw)
    int xs;                     // xbuf row stride: per rounded up to 4 words (16-byte rows)
};

// The word's own spin and occupancy words and the 12 neighbours' up bits (three of them shifted
// by one column, completed from the word before or after).
__device__ __forceinline__ void slab_loads(const uint2* film, int base, const int* off, int sgn, uint32_t& S,
                                           uint32_t& O, uint32_t up[12]) {
    const uint2 own = film[base];
    S = own.x;
    O = own.y;
#pragma unroll
    for (int k = 0; k < 9; ++k) up[k] = film[base + off[k]].x;
#pragma unroll
    for (int k = 9; k < 12; ++k) {
        const uint32_t a0 = film[base + off[k]].x, a1 = film[base + off[k] + sgn].x;
        up[k] = sgn < 0 ? __funnelshift_l(a1, a0, 1) : __funnelshift_r(a0, a1, 1);
    }
}

// Segment tables of one colour pass of this CTA's rows, in the (z, row, word) word lists:
// boundary segments (row jr0 of layer z at 2z, row jr1 - 1 at 2z + 1) and interior segments
// (rows jr0 + 1 .. jr1 - 2 of layer z at z), each with its first list entry and the running
// count of words before it; unused slots count INT_MAX so that a binary search never picks them.
struct PassSegs {
    int bstart[2 * kSlabMaxLayers], bcum[2 * kSlabMaxLayers];
    int istart[kSlabMaxLayers], icum[kSlabMaxLayers];
    int nB, nI;
};

// Built by warp 0 (lane z handles layer z).
__device__ __forceinline__ void build_segs(PassSegs& t, const int32_t* roff, int c, int L, int Rh, int jr0, int jr1) {
    const int lane = threadIdx.x & 31, nr = jr1 - jr0;
    int lb0 = 0, lb1 = 0, li = 0, s0 = 0, s1 = 0, si = 0;
    if (lane < L) {
        const int32_t* ro = roff + ((int64_t)c * L + lane) * (Rh + 1);
        s0 = ro[jr0];
        lb0 = ro[jr0 + 1] - s0;
        if (nr >= 2) { s1 = ro[jr1 - 1]; lb1 = ro[jr1] - s1; }
        if (nr >= 3) { si = ro[jr0 + 1]; li = ro[jr1 - 1] - si; }
    }
    int bsum = lb0 + lb1, isum = li;       // inclusive scans over the lanes
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int vb = __shfl_up_sync(0xFFFFFFFFu, bsum, d), vi = __shfl_up_sync(0xFFFFFFFFu, isum, d);
        if (lane >= d) { bsum += vb; isum += vi; }
    }
    if (lane < kSlabMaxLayers) {
        const int bex = bsum - lb0 - lb1, iex = isum - li;
        t.bstart[2 * lane] = s0;
        t.bstart[2 * lane + 1] = s1;
        t.bcum[2 * lane] = lane < L ? bex : 0x7FFFFFFF;
        t.bcum[2 * lane + 1] = lane < L ? bex + lb0 : 0x7FFFFFFF;
        t.istart[lane] = si;
        t.icum[lane] = lane < L ? iex : 0x7FFFFFFF;
    }
    const int totb = __shfl_sync(0xFFFFFFFFu, bsum, 31), toti = __shfl_sync(0xFFFFFFFFu, isum, 31);
    if (lane == 0) { t.nB = totb; t.nI = toti; }
}

// Boundary words of colour c of the rows [jr0, jr1) over all layers (the count a neighbour
// publishes per pass of that colour).
__device__ __forceinline__ int boundary_words(const int32_t* roff, int c, int L, int Rh, int jr0, int jr1) {
    int n = 0;
    for (int z = 0; z < L; ++z) {
        const int32_t* ro = roff + ((int64_t)c * L + z) * (Rh + 1);
        n += ro[jr0 + 1] - ro[jr0];
        if (jr1 - jr0 >= 2) n += ro[jr1] - ro[jr1 - 1];
    }
    return n;
}

template <bool GATE>
__global__ void __launch_bounds__(kSlabBlock, 1) k_slabs(const __grid_constant__ SlabArgs A) {
    extern __shared__ __align__(16) uint2 film[];       // [4][L+2][nrm+2][Wp]
    __shared__ uint32_t tab[128];
    __shared__ uint32_t gate_s[2];
    __shared__ long long red[64];
    __shared__ int off_s[4][2][12];
    __shared__ int sgn_s[4][2];
    __shared__ PassSegs segs[2];        // by pass parity
    __shared__ int grab_s[2];           // next unclaimed word of the pass, by pass parity
    __shared__ int nbw_s[2][4];         // words the lower / upper neighbour publishes per pass of colour c
    __shared__ volatile int err_s;
    const SweepArgs& a = A.s;
    const DevFilm& f = a.f;
    SlabGeom g;
    g.G = gridDim.x;
    g.r = blockIdx.x;
    g.jr0 = A.part[g.r];
    g.jr1 = A.part[g.r + 1];
    g.nr = g.jr1 - g.jr0;
    g.Wp = (int)f.Wp;
    g.nw = f.nw;
    g.L = f.L;
    g.ls = (A.nrm + 2) * g.Wp;
    g.cs = (g.L + 2) * g.ls;
    g.per = g.L * g.nw;
    g.xs = (g.per + 3) & ~3;
    uint32_t* spin32 = reinterpret_cast<uint32_t*>(film);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int passes = (int)(4 * a.nsweeps);

    for (int t = threadIdx.x; t < 96; t += blockDim.x) {
        const int c = t / 24, zp = (t / 12) & 1, k = t % 12;
        const NbrClass& nc = f.nb[c][zp];
        off_s[c][zp][k] = (nc.c2[k] - c) * g.cs + nc.dz[k] * g.ls + nc.dj[k] * g.Wp;
        if (k == 0) sgn_s[c][zp] = nc.sgn;
    }
    // the band and its halo rows, every colour and layer (device rows jr0 - 1 .. jr1)
    {
        const int per_cz = (g.nr + 2) * g.Wp;
        const int total = 4 * (g.L + 2) * per_cz;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int cz = t / per_cz, rem = t - cz * per_cz;
            const int c = cz / (g.L + 2), zz = cz - c * (g.L + 2);
            const int64_t gi = (int64_t)c * f.csw + (int64_t)zz * f.lsw + (int64_t)g.jr0 * g.Wp + rem;
            film[c * g.cs + zz * g.ls + rem] = make_uint2(f.sp[gi], f.op[gi]);
        }
    }
    if (warp == 0) build_segs(segs[0], A.roff, 0, g.L, f.Rh, g.jr0, g.jr1);
    if (threadIdx.x < 8) {
        const int side = threadIdx.x >> 2, c = threadIdx.x & 3, nb = side ? g.r + 1 : g.r - 1;
        nbw_s[side][c] = (nb >= 0 && nb < g.G) ? boundary_words(A.roff, c, g.L, f.Rh, A.part[nb], A.part[nb + 1]) : 0;
    }
    if (threadIdx.x == 0) {
        grab_s[0] = 0;
        grab_s[1] = 0;
        err_s = 0;
    }
    __syncthreads();
    // this CTA's boundary rows as its neighbours will first read them, then the first token
    for (int t = threadIdx.x; t < 8 * g.per; t += blockDim.x) {
        const int cs2 = t / g.per, q = t - cs2 * g.per;
        const int c = cs2 >> 1, side = cs2 & 1, z = q / g.nw, w = q - z * g.nw;
        const int jj = side ? g.nr : 1;
        A.xbuf[(int64_t)(g.r * 8 + cs2) * g.xs + q] = spin32[2 * (c * g.cs + (z + 1) * g.ls + jj * g.Wp + w + 1)];
    }
    __syncthreads();
    if (threadIdx.x == 0) red_release_gpu(&A.done[g.r * 32], 1u);

    const int wb = f.item_wbits, jb = f.item_jbits;
    const uint32_t wmask = (1u << wb) - 1u, jmask = (1u << jb) - 1u;
    unsigned want_lo = 1, want_hi = 1;      // warp 0: the neighbours' counters after the pass imported
    int k = a.k0, pos = a.pos0;
    stage_table<true>(a.tables, k, tab, gate_s);
    for (long long t = 0; t < a.nsweeps; ++t) {
        if (pos == a.step_total[k]) {
            ++k;
            pos = 0;
            stage_table<true>(a.tables, k, tab, gate_s);
        }
        const unsigned long long sweep = (unsigned long long)(a.sweep0 + t + 1);
        const uint32_t gthr = gate_s[0];
        const bool always_draw = (gate_s[1] & kFlagAlwaysDraw) != 0;
        const bool carry = !GATE && (gate_s[1] & kFlagNoNever) != 0;
        int dM = 0, dB = 0;
        for (int c = 0; c < 4; ++c) {
            const int P = (int)(4 * t) + c, buf = P & 1;
            const PassSegs& sg = segs[buf];
            const int nB = sg.nB, n = sg.nB + sg.nI;
            const uint32_t* list = f.items + (int64_t)c * f.item_cap;
            if (threadIdx.x == 0) grab_s[buf ^ 1] = 0;        // the next pass's counter
            // warp 0, once the boundary words are handed out: the next pass's segments, then the
            // neighbours' boundary rows of this colour into the halo (read from the next pass on)
            bool imported = warp != 0 || P + 1 >= passes;
            auto import_halo = [&]() {
                build_segs(segs[buf ^ 1], A.roff, (c + 1) & 3, g.L, f.Rh, g.jr0, g.jr1);
                want_lo += nbw_s[0][c];
                want_hi += nbw_s[1][c];
                const int nb = lane < 16 ? g.r - 1 : g.r + 1;
                const unsigned want = lane < 16 ? want_lo : want_hi;
                const bool has = nb >= 0 && nb < g.G;
                unsigned spins = 0;
                bool ok = true;
                for (;;) {
                    const bool ready = !has || (int)(ld_acquire_gpu(&A.done[nb * 32]) - want) >= 0;
                    if (__all_sync(0xFFFFFFFFu, ready)) break;
                    ++spins;
                    if ((spins & 15u) == 0 && *reinterpret_cast<const volatile int*>(&a.st->error)) { ok = false; break; }
                    if (spins > kNbrSpinLimit) {
                        if (lane == 0) {
                            atomicCAS(&a.st->error, 0, (int)ISF_ERR_TIMEOUT);
                            a.st->error_where = 3;
                        }
                        ok = false;
                        break;
                    }
                    if (spins > 64) __nanosleep(32);
                }
                if (!ok) {
                    if (lane == 0) err_s = 1;
                    return;
                }
                // 16-byte loads, four per lane in flight at a time
                const int nv = g.xs >> 2;
                for (int q0 = lane; q0 < 2 * nv; q0 += 128) {
                    uint4 v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int q = q0 + 32 * u, side = q >= nv, nb2 = side ? g.r + 1 : g.r - 1;
                        v[u] = make_uint4(0, 0, 0, 0);
                        if (q < 2 * nv && nb2 >= 0 && nb2 < g.G)
                            v[u] = __ldcg(reinterpret_cast<const uint4*>(A.xbuf + (int64_t)(nb2 * 8 + c * 2 + (side ? 0 : 1)) * g.xs) +
                                          (q - side * nv));
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int q = q0 + 32 * u, side = q >= nv, nb2 = side ? g.r + 1 : g.r - 1;
                        if (q >= 2 * nv || nb2 < 0 || nb2 >= g.G) continue;
                        const uint32_t vv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int wq = 4 * (q - side * nv) + e;     // word of the row: z * nw + w
                            if (wq >= g.per) break;
                            const int z = wq / g.nw, w = wq - z * g.nw;
                            spin32[2 * (c * g.cs + (z + 1) * g.ls + (side ? g.nr + 1 : 0) * g.Wp + w + 1)] = vv[e];
                        }
                    }
                }
            };
            for (;;) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&grab_s[buf], 32);
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
                if (!imported && base >= nB) {
                    import_halo();
                    imported = true;
                }
                if (base >= n) break;
                const int kk = base + lane;
                if (kk < n) {
                    int idx;
                    if (kk < nB) {
                        int s2 = 0;
#pragma unroll
                        for (int st = kSlabMaxLayers; st >= 1; st >>= 1)
                            if (s2 + st < 2 * kSlabMaxLayers && sg.bcum[s2 + st] <= kk) s2 += st;
                        idx = sg.bstart[s2] + (kk - sg.bcum[s2]);
                    } else {
                        const int ki = kk - nB;
                        int s2 = 0;
#pragma unroll
                        for (int st = kSlabMaxLayers / 2; st >= 1; st >>= 1)
                            if (s2 + st < kSlabMaxLayers && sg.icum[s2 + st] <= ki) s2 += st;
                        idx = sg.istart[s2] + (ki - sg.icum[s2]);
                    }
                    const uint32_t e = list[idx];
                    const int z = (int)(e >> (jb + wb)), j = (int)((e >> wb) & jmask), w = (int)(e & wmask);
                    const int jj = j - g.jr0 + 1;
                    const int at = c * g.cs + (z + 1) * g.ls + jj * g.Wp + w + 1;
                    uint32_t S, O, up[12], V[4];
                    const uint4 v = reinterpret_cast<const uint4*>(f.ivq)[(int64_t)c * f.item_cap + idx];
                    V[0] = v.x;
                    V[1] = v.y;
                    V[2] = v.z;
                    V[3] = v.w;
                    slab_loads(film, at, off_s[c][z & 1], sgn_s[c][z & 1], S, O, up);
                    const uint32_t q0 = block_counter(f, c, z, j, 32 * w);
                    uint4 u_first[4];
                    philox10_xn<4>(q0, (uint32_t)sweep, (uint32_t)(sweep >> 32), 0u, f.key0, f.key1, u_first);
                    const uint32_t F =
                        carry ? packed_decide<false, true>(S, O, up, V, q0, sweep, tab, gthr, always_draw, f.key0, f.key1,
                                                           u_first, dM, dB)
                              : packed_decide<GATE>(S, O, up, V, q0, sweep, tab, gthr, always_draw, f.key0, f.key1,
                                                    u_first, dM, dB);
                    if (F) {
                        const uint32_t Sn = S ^ F;
                        spin32[2 * at] = Sn;
                        const int64_t xq = (int64_t)z * g.nw + w;
                        if (jj == 1) A.xbuf[(int64_t)(g.r * 8 + c * 2 + 0) * g.xs + xq] = Sn;
                        if (jj == g.nr) A.xbuf[(int64_t)(g.r * 8 + c * 2 + 1) * g.xs + xq] = Sn;
                    }
                }
                if (base < nB) {
                    // this chunk's boundary words are in xbuf: publish them
                    __syncwarp();
                    if (lane == 0) red_release_gpu(&A.done[g.r * 32], (unsigned)min(32, nB - base));
                }
            }
            if (!imported) {
                import_halo();
                imported = true;
            }
            if (c == 3) {
                long long sM = dM, sB = dB;
                block_sum2(sM, sB, red);
                if (threadIdx.x == 0 && (sM | sB)) {
                    atomicAdd(&A.series[2 * t], (unsigned long long)sM);
                    atomicAdd(&A.series[2 * t + 1], (unsigned long long)sB);
                }
            }
            __syncthreads();
            if (err_s) return;
        }
        ++pos;
    }
    // own rows back to device memory (the occupancy does not change)
    const int per_c = g.L * g.nr * g.nw;
    for (int t = threadIdx.x; t < 4 * per_c; t += blockDim.x) {
        const int c = t / per_c, rem = t - c * per_c;
        const int z = rem / (g.nr * g.nw), rem2 = rem - z * (g.nr * g.nw);
        const int jj = 1 + rem2 / g.nw, w = rem2 % g.nw;
        const int64_t gi = (int64_t)c * f.csw + (int64_t)(z + 1) * f.lsw + (int64_t)(g.jr0 + jj) * g.Wp + w + 1;
        f.sp[gi] = spin32[2 * (c * g.cs + (z + 1) * g.ls + jj * g.Wp + w + 1)];
    }
}

__global__ void k_fold_series(const __grid_constant__ SweepArgs a, const unsigned long long* series) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    RunState rs;
    load_run_state(a.st, rs);
    int k = a.k0, pos = a.pos0;
    for (long long t = 0; t < a.nsweeps; ++t) {
        if (pos == a.step_total[k]) {
            ++k;
            pos = 0;
        }
        fold_sweep(a, rs, k, pos, a.step_eq[k], a.step_total[k], (long long)series[2 * t], (long long)series[2 * t + 1],
                   t);
        ++pos;
    }
    store_run_state(a.st, rs);
}


}  // namespace

uint32_t slab_smem_bytes(const DevFilm& f, int nrm) {
    return (uint32_t)((size_t)4 * (size_t)(f.L + 2) * (size_t)(nrm + 2) * (size_t)f.Wp * sizeof(uint2));
}

int slab_units(int threads, uint32_t smem, int* units) {
    *units = 0;
    int dev = 0, sms = 0, optin = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return (int)e;
    if (smem + kSlabStaticSmem > (uint32_t)optin) return 0;
    for (const void* k : {(const void*)k_slabs<false>, (const void*)k_slabs<true>}) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_slabs<false>, threads, smem);
    if (e != cudaSuccess) return (int)e;
    *units = sms * per;
    return 0;
}

int launch_slabs(const SlabArgs& a, int G, int threads, uint32_t smem, void* stream) {
    if (threads % 32 || threads < 64 || threads > kSlabBlock || G < 1 || G > kMaxSlabCTAs) return (int)cudaErrorInvalidValue;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(a.done, 0, (size_t)G * 32 * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.series, 0, (size_t)a.s.nsweeps * 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return (int)e;
    const void* fn = a.s.use_gate ? (const void*)k_slabs<true> : (const void*)k_slabs<false>;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    void* args[] = {const_cast<SlabArgs*>(&a)};
    return (int)cudaLaunchCooperativeKernel(fn, dim3(G), dim3(threads), args, smem, s);
}

int launch_fold_series(const SweepArgs& a, const unsigned long long* series, void* stream) {
    k_fold_series<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(a, series);
    return (int)cudaGetLastError();
}

}  // namespace isf
