// kernels_resident.cu — Metropolis sweeps (Eq. 8; Eq. 9 gate) with the whole film held in the
// shared memory of one thread-block cluster.
//
// The film's int8 layout is cut into row slabs: CTA r of a K-CTA cluster keeps rows
// [r*Jb, (r+1)*Jb) of every (colour, layer) in its shared memory for the whole launch.  A
// neighbour row that belongs to another CTA is read through distributed shared memory; rows
// outside an open boundary point at a shared row of vacancies; periodic rows and layers wrap in
// the row-pointer table, and periodic columns through two wrap bytes per row (column -1 and
// column Ch mirror Ch-1 and 0).  Colour passes are separated by the hardware cluster barrier
// (release / acquire), so one sweep costs four on-chip barriers and no L2 round trip.  This is
// the paper's row decomposition (Sec. 3, list items 1-2: rows per process plus the neighbouring
// processes' boundary rows) with CTAs of one cluster as the processes and DSMEM as the halo.
//
// The state is copied in from the global layout at the start of a launch and written back at
// the end, so launches of this kernel and of the global-memory kernel interleave freely; the
// random words are the same Philox words, so the trajectory is the same.
#include <cuda_runtime.h>

#include "sweep_core.cuh"

namespace isf {

// The resident and batch kernels check every address they compute from a film's descriptor
// before using it: an out-of-range access is recorded here (first one: code, two values) and
// skipped instead of made; the host reports it on its next read of the film.
__device__ unsigned long long g_isf_check[4];
#define ISF_CHECK(cond, code, v1, v2)                                                        \
    ((cond) ? true : (atomicCAS(&g_isf_check[0], 0ull, (unsigned long long)(code)) == 0ull     \
                          ? (g_isf_check[1] = (unsigned long long)(v1),                        \
                             g_isf_check[2] = (unsigned long long)(v2), false)                 \
                          : false))

namespace {

constexpr int kMaxK = 16;
constexpr int kMaxResThreads = 512;     // up to 128 registers per thread (16-site items)
constexpr int kMaxResThreads8 = 768;    // up to 80 registers per thread (8-site items)
template <int NW>
constexpr int max_threads_for() { return NW == 2 ? kMaxResThreads8 : kMaxResThreads; }
// per-CTA bookkeeping after the film and the row table: the step table (128 words), the gate
// threshold (16 bytes), the sweep's dM, dB accumulator (2 x 8 bytes, used in CTA 0) and every
// rank's slab address (kMaxK words)
constexpr uint32_t kMiscBytes = 128 * 4 + 16 + 2 * 8 + kMaxK * 4;


__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned dyn_smem_bytes() {
    unsigned n;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(n));
    return n;
}
__device__ __forceinline__ unsigned cluster_size() {
    unsigned n;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
    return n;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// generic address of the same shared-memory location in CTA `rank` of this cluster
__device__ __forceinline__ uint8_t* map_rank(uint8_t* p, unsigned rank) {
    uint64_t out;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(reinterpret_cast<uint64_t>(p)), "r"(rank));
    return reinterpret_cast<uint8_t*>(out);
}

__device__ __forceinline__ int64_t film_bytes_or(const DevFilm& f) { return 4 * f.cs8; }

// 32-bit shared-window address of a shared-memory pointer, and the same location in CTA `rank`
// of the cluster (a shared::cluster address; a CTA's own shared::cta addresses are valid there).
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t map_rank_addr(uint32_t a, unsigned rank) {
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(a), "r"(rank));
    return out;
}
template <bool CLUSTER>
__device__ __forceinline__ uint4 lds16(uint32_t a) {
    uint4 v;
    if (CLUSTER)
        asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a) : "memory");
    else
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a) : "memory");
    return v;
}
template <bool CLUSTER>
__device__ __forceinline__ uint32_t lds4(uint32_t a) {
    uint32_t v;
    if (CLUSTER) asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    else asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

template <bool CLUSTER>
__device__ __forceinline__ uint2 lds8(uint32_t a) {
    uint2 v;
    if (CLUSTER)
        asm volatile("ld.shared::cluster.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a) : "memory");
    else
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a) : "memory");
    return v;
}

// Neighbour sum of an 8-site half chunk from shared::cluster addresses.
template <bool CLUSTER>
__device__ __forceinline__ uint2 neighbour_sum8_sc(const uint32_t* nb, int sgn) {
    uint2 acc = lds8<CLUSTER>(nb[0]);
#pragma unroll
    for (int k = 1; k < 9; ++k) {
        const uint2 v = lds8<CLUSTER>(nb[k]);
        acc.x += v.x;
        acc.y += v.y;
    }
    if (sgn < 0) {
#pragma unroll
        for (int k = 9; k < 12; ++k) {
            const uint2 v = lds8<CLUSTER>(nb[k]);
            const uint32_t e = lds4<CLUSTER>(nb[k] - 4);
            acc.x += __funnelshift_l(e, v.x, 8);
            acc.y += __funnelshift_l(v.x, v.y, 8);
        }
    } else {
#pragma unroll
        for (int k = 9; k < 12; ++k) {
            const uint2 v = lds8<CLUSTER>(nb[k]);
            const uint32_t e = lds4<CLUSTER>(nb[k] + 8);
            acc.x += __funnelshift_r(v.x, v.y, 8);
            acc.y += __funnelshift_r(v.y, e, 8);
        }
    }
    return acc;
}

// The 15 loads of a 16-site chunk's neighbour sum (12 rows, and the next or previous word of the
// three shifted ones), issued together; neighbour_sum16_from adds them up.
template <bool CLUSTER>
__device__ __forceinline__ void neighbour_loads16(const uint32_t* nb, int sgn, uint4 v[12], uint32_t e[3]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = lds16<CLUSTER>(nb[k]);
#pragma unroll
    for (int k = 9; k < 12; ++k) e[k - 9] = lds4<CLUSTER>(sgn < 0 ? nb[k] - 4 : nb[k] + 16);
}
__device__ __forceinline__ uint4 neighbour_sum16_from(const uint4 v[12], const uint32_t e[3], int sgn) {
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
    return acc;
}

// Add v to the 64-bit word at a shared::cluster address (another CTA's shared memory, or this
// CTA's own when CLUSTER is false).
template <bool CLUSTER>
__device__ __forceinline__ void red_add64(uint32_t a, long long v) {
    if (CLUSTER)
        asm volatile("red.relaxed.cluster.shared::cluster.add.u64 [%0], %1;" :: "r"(a), "l"(v) : "memory");
    else
        asm volatile("red.shared.add.u64 [%0], %1;" :: "r"(a), "l"(v) : "memory");
}

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// The two halves of the cluster barrier, so that work that needs no other CTA's writes (the
// next pass's random words) can run while the slowest CTA finishes.
__device__ __forceinline__ void cluster_arrive() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <bool CLUSTER>
__device__ __forceinline__ void sync_all() {
    if (CLUSTER) cluster_sync_all();
    else __syncthreads();
}

// One film on this CTA (CLUSTER = false) or on this cluster: slab in, the launch's sweeps,
// slab out.  Ends with a barrier over all CTAs that took part.  The last warp of every CTA takes
// no sites: in CTA 0 its first lane folds each sweep's dM, dB into the step sums while the other
// warps run the next colour pass; the other warps add their per-sweep dM, dB into CTA 0's
// accumulator with shared::cluster reductions (no block-wide reduction on the critical path).
// NW = 4: 16-site work items; NW = 2: 8-site items (twice the items per pass, for films whose
// 16-site items would leave the CTA's warps too few to hide the shared-memory latency).
template <bool CLUSTER, bool PX, int NW = 4>
__device__ __forceinline__ void run_film(const ResArgs& a, uint8_t* sm) {
    static_assert(NW == 2 || NW == 4, "work items are 8 or 16 sites");
    constexpr int W = 4 * NW;   // sites (bytes) per item
    const SweepArgs& s = a.s;
    const DevFilm& f = s.f;
    const unsigned K = CLUSTER ? (unsigned)a.K : 1u;
    const unsigned rank = CLUSTER ? cluster_rank() : 0u;
    const int Jb = a.Jb, L = f.L, Rh = f.Rh, nck = f.nck, Ch = f.Ch;
    const int P = (int)f.P;
    const int j0 = (int)rank * Jb;
    const int nown = max(0, min(Jb, Rh - j0));      // trailing CTAs may own no rows
    uint8_t* film = sm + a.film_off;
    uint8_t* vac = sm + a.vac_off;
    uint32_t* ptrs = reinterpret_cast<uint32_t*>(sm + a.ptr_off);
    uint32_t* tab = reinterpret_cast<uint32_t*>(sm + a.misc_off);
    uint32_t* gate = tab + 128;
    unsigned long long* obs = reinterpret_cast<unsigned long long*>(sm + a.misc_off + 128 * 4 + 16);  // CTA 0's: dM, dB of a sweep
    uint32_t* base = reinterpret_cast<uint32_t*>(obs + 2);

    // slab in, vacancy row, every rank's slab address
    const int words = P / 16;
    const uint64_t smem_n = dyn_smem_bytes();
    bool desc_ok = ISF_CHECK(K >= 1 && K <= 16 && Jb >= 1 && (int64_t)Jb * K >= Rh && P % 16 == 0, 1, K, Jb);
    desc_ok = desc_ok && ISF_CHECK(blockDim.x >= 64 && blockDim.x % 32 == 0, 12, blockDim.x, 0);
    desc_ok = desc_ok && ISF_CHECK(a.misc_off + kMiscBytes <= smem_n, 2, a.misc_off, smem_n);
    desc_ok = desc_ok && ISF_CHECK((uint64_t)a.ptr_off + (uint64_t)4 * L * Jb * 48 <= a.misc_off, 3, a.ptr_off, a.misc_off);
    desc_ok = desc_ok && ISF_CHECK(s.k0 >= 0 && s.k0 < s.nsteps && s.nsteps >= 1, 4, s.k0, s.nsteps);
    if (!desc_ok) { sync_all<CLUSTER>(); sync_all<CLUSTER>(); return; }
    for (int t = threadIdx.x; t < 4 * L * nown * words; t += blockDim.x) {
        const int w = t % words;
        const int rr = t / words;
        const int jl = rr % nown, cz = rr / nown;
        const int64_t off = addr8(f, cz / L, cz % L, j0 + jl, -16) + 16 * w;
        const uint64_t dsm = (uint64_t)a.film_off + ((uint64_t)cz * Jb + jl) * P + 16 * w;
        if (!ISF_CHECK(off >= 0 && off + 16 <= film_bytes_or(f), 5, off, film_bytes_or(f))) continue;
        if (!ISF_CHECK(dsm + 16 <= a.vac_off, 6, dsm, a.vac_off)) continue;
        reinterpret_cast<uint4*>(film + ((size_t)cz * Jb + jl) * P)[w] = *reinterpret_cast<const uint4*>(f.s8 + off);
    }
    for (int t = threadIdx.x; t < P / 4; t += blockDim.x) reinterpret_cast<uint32_t*>(vac)[t] = 0x01010101u;
    if (threadIdx.x < K) base[threadIdx.x] = CLUSTER ? map_rank_addr(smem_addr(film), threadIdx.x) : smem_addr(film);
    if (threadIdx.x == 0) { obs[0] = 0; obs[1] = 0; }
    __syncthreads();
    if (PX) {
        for (int rr = threadIdx.x; rr < 4 * L * nown; rr += blockDim.x) {
            uint8_t* row = film + ((size_t)(rr / nown) * Jb + rr % nown) * P;
            row[15] = row[16 + Ch - 1];
            row[16 + Ch] = row[16];
        }
    }
    // neighbour-row table of every own row, in the class order (9 unshifted, 3 shifted)
    for (int t = threadIdx.x; t < 4 * L * nown * 12; t += blockDim.x) {
        const int k = t % 12;
        const int rr = t / 12;
        const int jl = rr % nown, cz = rr / nown;
        const int c = cz / L, z = cz % L;
        const NbrClass& nc = f.nb[c][z & 1];
        int zz = z + nc.dz[k], jj = j0 + jl + nc.dj[k];
        bool inside = true;
        if (zz < 0 || zz >= L) {
            if (f.flags & 4u) zz = (zz + L) % L;
            else inside = false;
        }
        if (jj < 0 || jj >= Rh) {
            if (f.flags & 2u) jj = (jj + Rh) % Rh;
            else inside = false;
        }
        uint32_t p = smem_addr(vac);
        if (inside) {
            const int rk = jj / Jb;
            if (!ISF_CHECK(rk >= 0 && rk < (int)K && nc.c2[k] >= 0 && nc.c2[k] < 4, 7, rk, nc.c2[k])) continue;
            p = base[rk] + (uint32_t)(((nc.c2[k] * L + zz) * Jb + (jj - rk * Jb)) * P);
        }
        ptrs[((size_t)cz * Jb + jl) * 12 + k] = p;
    }
    sync_all<CLUSTER>();    // every slab loaded before anyone reads a neighbour's

    const int nci = NW == 4 ? nck : (Ch + 7) / 8;     // items per row
    const int ithreads = (int)blockDim.x - 32;       // threads that take sites; the last warp folds
    const bool fold_warp = (int)threadIdx.x >= ithreads;
    const int items = fold_warp ? 0 : L * nown * nci;
    ItemWalk walk0;
    walk0.init(threadIdx.x, ithreads, nci, nown > 0 ? nown : 1);
    const uint32_t obs0 = CLUSTER ? map_rank_addr(smem_addr(obs), 0) : smem_addr(obs);
    int k = s.k0, pos = s.pos0;
    const bool folder = rank == 0 && (int)threadIdx.x == ithreads;
    __shared__ RunState rs;     // touched by the folding thread only
    int k_eq = 0, k_tot = 0;
    if (folder) {
        load_run_state(s.st, rs);
        k_eq = s.step_eq[k];
        k_tot = s.step_total[k];
    }
    // In a cluster the barrier after each pass is split: a thread arrives when its sites are
    // done, draws the Philox blocks of its first site chunk of the next pass (they depend only on
    // counters), and waits only then.  The fold of a sweep follows the wait that ends it.
    constexpr bool SPLIT = CLUSTER && NW == 4;
    bool pending = false;                   // arrived, not yet waited
    uint4 pf_u[4];                          // next pass's first chunk: its Philox blocks
    bool pf = false;
    long long fold_t = -1;                  // sweep whose fold waits for the next barrier
    int fold_k = 0, fold_pos = 0, fold_eq = 0, fold_tot = 0;
    auto fold_pending = [&]() {
        if (folder && fold_t >= 0 && ISF_CHECK(fold_k >= 0 && fold_k < s.nsteps, 10, fold_k, s.nsteps)) {
            const long long sM = (long long)obs[0], sB = (long long)obs[1];
            obs[0] = 0;
            obs[1] = 0;
            fold_sweep(s, rs, fold_k, fold_pos, fold_eq, fold_tot, sM, sB, fold_t);
        }
        fold_t = -1;
    };
    stage_table<false, !PX>(s.tables, k, tab, gate);
    for (long long t = 0; t < s.nsweeps; ++t) {
        if (pos == s.step_total[k]) {
            ++k;
            pos = 0;
            // with the split barrier a thread gets here while others may still read the old
            // table in the last pass: everyone first
            if (SPLIT) __syncthreads();
            stage_table<false, !PX>(s.tables, k, tab, gate);
            if (folder) { k_eq = s.step_eq[k]; k_tot = s.step_total[k]; }
        }
        const unsigned long long sweep = (unsigned long long)(s.sweep0 + t + 1);
        const uint32_t gthr = gate[0];
        const bool neg = !PX && (gate[1] & kFlagNoNever);    // table staged negated (carry form)
        int dM = 0, dB = 0;
        for (int c = 0; c < 4; ++c) {
            if (SPLIT && pending) {
                cluster_wait();
                pending = false;
                if (c == 0) fold_pending();
            }
            ItemWalk w = walk0;
            for (int it = threadIdx.x; it < items; it += ithreads, w.next()) {
                const int ck = w.ck, jl = w.jr, z = w.z;
                const size_t r = (size_t)(c * L + z) * Jb + jl;
                if (!ISF_CHECK(z >= 0 && z < L && jl >= 0 && jl < nown && ck >= 0 && ck < nci, 8, it, ((uint64_t)z << 32) | (uint32_t)jl)) continue;
                uint8_t* row = film + r * P;
                uint8_t* own = row + 16 + W * ck;
                uint32_t Sw[NW], Aw[NW];
                if constexpr (NW == 4) {
                    const uint4 S = *reinterpret_cast<const uint4*>(own);
                    Sw[0] = S.x; Sw[1] = S.y; Sw[2] = S.z; Sw[3] = S.w;
                } else {
                    const uint2 S = *reinterpret_cast<const uint2*>(own);
                    Sw[0] = S.x; Sw[1] = S.y;
                }
                uint32_t sites = 0;     // nonzero unless every byte is a vacancy (1)
#pragma unroll
                for (int v = 0; v < NW; ++v) sites |= Sw[v] ^ 0x01010101u;
                if (!sites) continue;   // no site to attempt: no table lookup, no random word
                // the row's 12 neighbour-row addresses (48 bytes, 16-byte aligned)
                const uint4* pr = reinterpret_cast<const uint4*>(ptrs + r * 12);
                const uint4 pa = pr[0], pb = pr[1], pc = pr[2];
                const uint32_t co = 16 + W * ck;
                const uint32_t nbp[12] = {pa.x + co, pa.y + co, pa.z + co, pa.w + co, pb.x + co, pb.y + co,
                                          pb.z + co, pb.w + co, pc.x + co, pc.y + co, pc.z + co, pc.w + co};
                const uint32_t q0 = block_counter(f, c, z, j0 + jl, W * ck);
                const int sgn = f.nb[c][z & 1].sgn;
                uint32_t fm[NW];
                uint32_t any;
                if constexpr (NW == 4) {
                    // loads first, then the chunk's four Philox blocks while they are in flight
                    // (every pass starts all warps at once, so nothing else would fill that wait)
                    uint4 nv[12];
                    uint32_t ne[3];
                    neighbour_loads16<CLUSTER>(nbp, sgn, nv, ne);
                    uint4 u[4];
                    if (SPLIT && pf && it == (int)threadIdx.x) {
#pragma unroll
                        for (int v = 0; v < 4; ++v) u[v] = pf_u[v];
                    } else {
                        philox10_xn<4>(q0, (uint32_t)sweep, (uint32_t)(sweep >> 32), 0u, f.key0, f.key1, u);
                    }
                    const uint4 a4 = neighbour_sum16_from(nv, ne, sgn);
                    Aw[0] = a4.x; Aw[1] = a4.y; Aw[2] = a4.z; Aw[3] = a4.w;
                    any = s.use_gate
                        ? decide16<true, PX, 4, true>(Sw, Aw, q0, sweep, tab, gthr, f.key0, f.key1, W * ck, Ch, fm, dM, dB, u, neg)
                        : decide16<false, PX, 4, true>(Sw, Aw, q0, sweep, tab, gthr, f.key0, f.key1, W * ck, Ch, fm, dM, dB, u, neg);
                } else {
                    const uint2 a2 = neighbour_sum8_sc<CLUSTER>(nbp, sgn);
                    Aw[0] = a2.x; Aw[1] = a2.y;
                    any = s.use_gate
                        ? decide16<true, PX, NW>(Sw, Aw, q0, sweep, tab, gthr, f.key0, f.key1, W * ck, Ch, fm, dM, dB, nullptr, neg)
                        : decide16<false, PX, NW>(Sw, Aw, q0, sweep, tab, gthr, f.key0, f.key1, W * ck, Ch, fm, dM, dB, nullptr, neg);
                }
                if (any) {
                    if (!PX) {
                        if constexpr (NW == 4)
                            *reinterpret_cast<uint4*>(own) = make_uint4(Sw[0] ^ fm[0], Sw[1] ^ fm[1], Sw[2] ^ fm[2], Sw[3] ^ fm[3]);
                        else
                            *reinterpret_cast<uint2*>(own) = make_uint2(Sw[0] ^ fm[0], Sw[1] ^ fm[1]);
                    } else {
                        // byte stores (the row's wrap bytes may share a word), refreshing the
                        // wrap copies of columns 0 and Ch-1
#pragma unroll
                        for (int v = 0; v < NW; ++v) {
                            if (!fm[v]) continue;
#pragma unroll
                            for (int b = 0; b < 4; ++b) {
                                if (!((fm[v] >> (8 * b)) & 0xFFu)) continue;
                                const uint8_t nbyte = (uint8_t)((Sw[v] ^ fm[v]) >> (8 * b));
                                const int i = W * ck + 4 * v + b;
                                own[4 * v + b] = nbyte;
                                if (i == 0) row[16 + Ch] = nbyte;
                                if (i == Ch - 1) row[15] = nbyte;
                            }
                        }
                    }
                }
            }
            if (c == 3 && !fold_warp) {
                const int wM = warp_sum_i(dM), wB = warp_sum_i(dB);
                if ((threadIdx.x & 31) == 0 && (wM | wB)) {
                    red_add64<CLUSTER>(obs0, (long long)wM);
                    red_add64<CLUSTER>(obs0 + 8, (long long)wB);
                }
            }
            if (SPLIT) {
                // the barrier orders the reductions before the fold, and the fold's reset before
                // the next sweep's reductions
                cluster_arrive();
                pending = true;
                pf = false;
                const int cn = (c + 1) & 3;
                const long long tn = c == 3 ? t + 1 : t;
                if ((int)threadIdx.x < items && tn < s.nsweeps) {
                    const unsigned long long sn = (unsigned long long)(s.sweep0 + tn + 1);
                    const uint32_t qn = block_counter(f, cn, walk0.z, j0 + walk0.jr, W * walk0.ck);
                    philox10_xn<4>(qn, (uint32_t)sn, (uint32_t)(sn >> 32), 0u, f.key0, f.key1, pf_u);
                    pf = true;
                }
            } else {
                sync_all<CLUSTER>();    // orders the reductions before the fold, and the fold's reset
            }                           // before the next sweep's reductions
        }
        if (folder) { fold_t = t; fold_k = k; fold_pos = pos; fold_eq = k_eq; fold_tot = k_tot; }
        if (!SPLIT) fold_pending();
        ++pos;
    }
    if (SPLIT && pending) {
        cluster_wait();
        fold_pending();
    }
    if (folder) store_run_state(s.st, rs);

    // slab out: the site columns only (the wrap bytes and halo stay out of the global layout)
    const int cw = nck;   // 16-byte words holding columns 0 .. 16*nck-1
    for (int t = threadIdx.x; t < 4 * L * nown * cw; t += blockDim.x) {
        const int w = t % cw;
        const int rr = t / cw;
        const int jl = rr % nown, cz = rr / nown;
        uint4 v = reinterpret_cast<const uint4*>(film + ((size_t)cz * Jb + jl) * P + 16)[w];
        if (PX && Ch < 16 * nck && (Ch >> 4) == w) {
            // column Ch (a wrap byte) falls in this word: put the vacancy padding back
            uint32_t* vw = reinterpret_cast<uint32_t*>(&v);
            const int b = Ch & 15;
            vw[b >> 2] = (vw[b >> 2] & ~(0xFFu << (8 * (b & 3)))) | (0x01u << (8 * (b & 3)));
        }
        const int64_t off = addr8(f, cz / L, cz % L, j0 + jl, 0) + 16 * w;
        if (!ISF_CHECK(off >= 16 && off + 16 <= film_bytes_or(f), 9, off, film_bytes_or(f))) continue;
        *reinterpret_cast<uint4*>(f.s8 + off) = v;
    }
    sync_all<CLUSTER>();    // no CTA leaves while another may still address its shared memory
}

template <bool CLUSTER, bool PX, int NW>
__global__ void __launch_bounds__(max_threads_for<NW>(), 1) k_resident(const __grid_constant__ ResArgs a) {
    extern __shared__ __align__(16) uint8_t sm[];
    run_film<CLUSTER, PX, NW>(a, sm);
}

// Batched films: every CTA (or cluster) takes the next film of the queue, runs its sweeps with
// the film resident in its shared memory, and takes another until the queue is empty.  Films
// are independent Markov chains (each its own seed, schedule and state), so no film waits on
// another; the queue is a device counter.
template <bool CLUSTER>
__global__ void __launch_bounds__(kMaxResThreads, 1) k_batch(const ResArgs* films, int nfilms, unsigned* next) {
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ int film_s;
    const unsigned rank = CLUSTER ? cluster_rank() : 0u;
    const unsigned K = CLUSTER ? cluster_size() : 1u;
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            const int idx = (int)atomicAdd(next, 1u);
            for (unsigned r = 0; r < K; ++r) {
                int* dst = CLUSTER ? reinterpret_cast<int*>(map_rank(reinterpret_cast<uint8_t*>(&film_s), r)) : &film_s;
                *dst = idx;
            }
        }
        sync_all<CLUSTER>();
        const int idx = film_s;
        if (idx >= nfilms || !ISF_CHECK(idx >= 0, 11, idx, nfilms)) break;
        // the descriptor is read in place (it does not change during the launch); films with
        // periodic columns are not queued here
        run_film<CLUSTER, false>(films[idx], sm);
    }
}

template <bool CLUSTER, bool PX, int NW>
int launch_variant(const ResArgs& ra, const ResPlan& p, cudaStream_t s) {
    auto kern = k_resident<CLUSTER, PX, NW>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return (int)e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(p.K);
    cfg.blockDim = dim3(p.threads);
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (CLUSTER) {
        if (p.K > 8) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return (int)e;
        }
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = p.K;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return (int)cudaLaunchKernelEx(&cfg, kern, ra);
}

template <bool CLUSTER, bool PX, int NW>
int clusters_possible(const ResPlan& p, int* n) {
    auto kern = k_resident<CLUSTER, PX, NW>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return (int)e;
    if (!CLUSTER) { *n = 1; return 0; }
    if (p.K > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return (int)e;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(p.K);
    cfg.blockDim = dim3(p.threads);
    cfg.dynamicSmemBytes = p.smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = p.K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return (int)cudaOccupancyMaxActiveClusters(n, kern, &cfg);
}

inline uint32_t round16(uint32_t v) { return (v + 15u) & ~15u; }

bool layout_for(const DevFilm& f, int K, int threads, int max_smem, ResPlan* out) {
    if (K < 1 || K > kMaxK || K > f.Rh) return false;
    const int Jb = (f.Rh + K - 1) / K;           // the last CTAs may own fewer rows, or none
    const uint64_t rows = (uint64_t)4 * f.L * Jb;
    ResPlan p{};
    p.K = K;
    p.Jb = Jb;
    p.threads = threads;
    p.film_off = 0;
    p.vac_off = round16((uint32_t)(rows * f.P));
    p.ptr_off = round16(p.vac_off + (uint32_t)f.P);
    p.misc_off = round16(p.ptr_off + (uint32_t)(rows * 12 * 4));
    p.smem = round16(p.misc_off + kMiscBytes);
    if (rows * f.P > (uint64_t)max_smem || p.smem > (uint32_t)max_smem) return false;
    *out = p;
    return true;
}

}  // namespace

int resident_plan(const DevFilm& f, int want_K, int want_threads, int want_sites, ResPlan* out) {
    if (f.packed) return 1;                               // int8 layout only
    if (want_sites != 0 && want_sites != 8 && want_sites != 16) return 3;
    int dev = 0, max_smem = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 2;
    if (cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 2;
    const int threads = want_threads > 0 ? want_threads : 0;
    // Work of one colour pass per CTA: about 4096 lattice sites (one 16-site chunk per thread
    // of a 256-thread CTA); the smallest power of two that also fits the shared memory.
    const int64_t per_pass = (int64_t)f.L * f.Rh * f.Ch;
    int K0 = 1;
    while (K0 < kMaxK && per_pass / K0 > 4096) K0 *= 2;
    // candidates: K0, 2*K0, ..., 16, then K0/2, ..., 1 (or only the requested size)
    int cand[8], nc = 0;
    if (want_K > 0) {
        cand[nc++] = want_K;
    } else {
        for (int K = K0; K <= kMaxK; K *= 2) cand[nc++] = K;
        for (int K = K0 / 2; K >= 1; K /= 2) cand[nc++] = K;
    }
    for (int ci = 0; ci < nc; ++ci) {
        const int K = cand[ci];
        const int Jb = (f.Rh + K - 1) / K;
        const int64_t items16 = (int64_t)f.L * Jb * f.nck;
        // 8-site items when a quarter or more of the 16-site items' sites would be padding past
        // the row's last column (narrow rows); else 16, which costs fewer instructions per site
        int sites = want_sites;
        if (!sites) sites = 4 * (16 * f.nck - f.Ch) >= 16 * f.nck ? 8 : 16;
        const int64_t items = sites == 8 ? (int64_t)f.L * Jb * ((f.Ch + 7) / 8) : items16;
        const int tmax = sites == 8 ? kMaxResThreads8 : kMaxResThreads;
        // threads: one per work item of a pass, rounded to whole warps, plus the folding warp
        int th = threads;
        if (!th) {
            int64_t ith = (items + 31) / 32 * 32;
            if (ith > tmax - 32) ith = tmax - 32;
            th = (int)ith + 32;
        }
        if (th > tmax || th < 64) {
            if (want_sites) return 3;
            continue;
        }
        ResPlan p;
        if (!layout_for(f, K, th, max_smem, &p)) continue;
        p.item_sites = sites;
        int n = 0;
        const bool px = (f.flags & 1u) != 0;
        int e;
        if (sites == 8)
            e = K > 1 ? (px ? clusters_possible<true, true, 2>(p, &n) : clusters_possible<true, false, 2>(p, &n))
                      : (px ? clusters_possible<false, true, 2>(p, &n) : clusters_possible<false, false, 2>(p, &n));
        else
            e = K > 1 ? (px ? clusters_possible<true, true, 4>(p, &n) : clusters_possible<true, false, 4>(p, &n))
                      : (px ? clusters_possible<false, true, 4>(p, &n) : clusters_possible<false, false, 4>(p, &n));
        if (e == 0 && n >= 1) {
            *out = p;
            return 0;
        }
        cudaGetLastError();
    }
    return 3;
}

int read_checks(unsigned long long out[4]) {
    return (int)cudaMemcpyFromSymbol(out, g_isf_check, 4 * sizeof(unsigned long long));
}

ResArgs make_res_args(const SweepArgs& a, const ResPlan& p) {
    ResArgs ra{};
    ra.s = a;
    ra.K = p.K;
    ra.Jb = p.Jb;
    ra.film_off = p.film_off;
    ra.vac_off = p.vac_off;
    ra.ptr_off = p.ptr_off;
    ra.misc_off = p.misc_off;
    return ra;
}

namespace {
template <bool CLUSTER>
cudaLaunchConfig_t batch_config(int K, int threads, uint32_t smem, int units, cudaStream_t s,
                                cudaLaunchAttribute* attr, cudaError_t* err) {
    auto kern = k_batch<CLUSTER>;
    *err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (*err == cudaSuccess && CLUSTER && K > 8)
        *err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(units * (CLUSTER ? K : 1));
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    if (CLUSTER) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = K;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cfg;
}
}  // namespace

int batch_units_possible(int K, int threads, uint32_t smem, int* units) {
    cudaError_t e;
    cudaLaunchAttribute attr[1];
    if (K > 1) {
        cudaLaunchConfig_t cfg = batch_config<true>(K, threads, smem, 1, nullptr, attr, &e);
        if (e != cudaSuccess) return (int)e;
        return (int)cudaOccupancyMaxActiveClusters(units, k_batch<true>, &cfg);
    }
    cudaLaunchConfig_t cfg = batch_config<false>(1, threads, smem, 1, nullptr, attr, &e);
    if (e != cudaSuccess) return (int)e;
    int per = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<false>, threads, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *units = per * sms;
    return (int)e;
}

int launch_batch(const ResArgs* films, int n, unsigned* next, int K, int threads, uint32_t smem, int units,
                 void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    cudaLaunchAttribute attr[1];
    if (K > 1) {
        cudaLaunchConfig_t cfg = batch_config<true>(K, threads, smem, units, s, attr, &e);
        if (e != cudaSuccess) return (int)e;
        return (int)cudaLaunchKernelEx(&cfg, k_batch<true>, films, n, next);
    }
    cudaLaunchConfig_t cfg = batch_config<false>(1, threads, smem, units, s, attr, &e);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaLaunchKernelEx(&cfg, k_batch<false>, films, n, next);
}

int launch_resident(const SweepArgs& a, const ResPlan& p, void* stream) {
    ResArgs ra = make_res_args(a, p);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool px = (a.f.flags & 1u) != 0;
    if (p.item_sites == 8) {
        if (p.K > 1) return px ? launch_variant<true, true, 2>(ra, p, s) : launch_variant<true, false, 2>(ra, p, s);
        return px ? launch_variant<false, true, 2>(ra, p, s) : launch_variant<false, false, 2>(ra, p, s);
    }
    if (p.K > 1) return px ? launch_variant<true, true, 4>(ra, p, s) : launch_variant<true, false, 4>(ra, p, s);
    return px ? launch_variant<false, true, 4>(ra, p, s) : launch_variant<false, false, 4>(ra, p, s);
}

}  // namespace isf
