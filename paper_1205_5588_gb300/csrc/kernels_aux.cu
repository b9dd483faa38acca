// kernels_aux.cu — set-up and read-out kernels: initial spins (Philox stream 2, or all up /
// all down) with the occupancy of the height map (Sec. 3), full recomputation of M and B
// (Eq. 3) and of the occupied site and bond counts, unpack to / pack from [z][y][x] int8, and
// raw Philox blocks for checking the generator.
#include <cuda_runtime.h>

#include "../../include/isingfilm.h"
#include "device_common.cuh"
#include "sweep_core.cuh"

namespace isf {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t n) {
    int64_t g = (n + kThreads - 1) / kThreads;
    if (g > 152 * 64) g = 152 * 64;
    return g < 1 ? 1 : (int)g;
}

// One thread per 4-byte word of the int8 arrays, halo included: 4 sites = one Philox block.
__global__ void k_init_int8(DevFilm f, int init, const int8_t* src) {
    const int64_t wpr = f.P / 4;
    const int64_t total = (int64_t)4 * (f.L + 2) * (f.Rh + 2) * wpr;
    uint32_t* out = reinterpret_cast<uint32_t*>(f.s8);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / wpr;
        const int wd = (int)(t - row * wpr);
        const int jj = (int)(row % (f.Rh + 2));
        const int64_t r2 = row / (f.Rh + 2);
        const int zz = (int)(r2 % (f.L + 2));
        const int c = (int)(r2 / (f.L + 2));
        const int z = zz - 1, j = jj - 1, i0 = wd * 4 - 16;
        uint32_t word = 0x01010101u;   // vacancy in every byte
        if (z >= 0 && z < f.L && j >= 0 && j < f.Rh && i0 >= 0 && i0 < f.Ch) {
            const int zp = z & 1, px = (c & 1) ^ zp, py = ((c >> 1) & 1) ^ zp;
            const int y = 2 * j + py;
            uint4 rnd = make_uint4(0, 0, 0, 0);
            bool have = false;
            for (int b = 0; b < 4; ++b) {
                const int i = i0 + b, x = 2 * i + px;
                if (i >= f.Ch || x >= f.C || y >= f.R || !site_occupied(f, x, y, z)) continue;
                int s;
                if (src) {
                    s = src[((int64_t)z * f.R + y) * f.C + x];
                } else if (init == ISF_INIT_RANDOM) {
                    if (!have) {
                        rnd = philox10(make_uint4(block_counter(f, c, z, j, i0), 0u, 0u, 2u), f.key0, f.key1);
                        have = true;
                    }
                    s = (word_of(rnd, b) >> 31) ? -1 : 1;
                } else {
                    s = init == ISF_INIT_UP ? 1 : -1;
                }
                word = (word & ~(0xFFu << (8 * b))) | ((uint32_t)(s + 1) << (8 * b));
            }
        }
        out[t] = word;
    }
}

// One thread per word of the packed bit-planes, halo included: 32 sites = 8 Philox blocks.
__global__ void k_init_packed(DevFilm f, int init, const int8_t* src) {
    const int64_t total = (int64_t)4 * (f.L + 2) * (f.Rh + 2) * f.Wp;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / f.Wp;
        const int wd = (int)(t - row * f.Wp);
        const int jj = (int)(row % (f.Rh + 2));
        const int64_t r2 = row / (f.Rh + 2);
        const int zz = (int)(r2 % (f.L + 2));
        const int c = (int)(r2 / (f.L + 2));
        const int z = zz - 1, j = jj - 1, w = wd - 1;
        uint32_t sbits = 0, obits = 0;
        if (z >= 0 && z < f.L && j >= 0 && j < f.Rh && w >= 0 && w < f.nw) {
            const int zp = z & 1, px = (c & 1) ^ zp, py = ((c >> 1) & 1) ^ zp;
            const int y = 2 * j + py;
            for (int v = 0; v < 8; ++v) {
                uint4 rnd = make_uint4(0, 0, 0, 0);
                bool have = false;
                for (int b = 0; b < 4; ++b) {
                    const int lane = 4 * v + b, i = 32 * w + lane, x = 2 * i + px;
                    if (i >= f.Ch || x >= f.C || y >= f.R || !site_occupied(f, x, y, z)) continue;
                    int s;
                    if (src) {
                        s = src[((int64_t)z * f.R + y) * f.C + x];
                    } else if (init == ISF_INIT_RANDOM) {
                        if (!have) {
                            rnd = philox10(make_uint4(block_counter(f, c, z, j, 32 * w + 4 * v), 0u, 0u, 2u),
                                           f.key0, f.key1);
                            have = true;
                        }
                        s = (word_of(rnd, b) >> 31) ? -1 : 1;
                    } else {
                        s = init == ISF_INIT_UP ? 1 : -1;
                    }
                    obits |= 1u << lane;
                    if (s > 0) sbits |= 1u << lane;
                }
            }
        }
        f.sp[t] = sbits;
        f.op[t] = obits;
    }
}

// Per entry of the item lists: the word index (packed) or byte offset (int8) with the layer
// parity in bit 31, and the Philox counter, which the sweep kernels would derive from (z, row,
// item); packed films also the bit-sliced count of vacant neighbours of the word's 32 sites (1s,
// 2s, 4s, 8s) from the occupancy planes, i.e. the same 12 neighbour words a colour pass reads,
// three shifted by one column.  Occupancy never changes, so the sweep kernels read these records
// instead of decoding the entry (and, packed, loading and counting 12 occupancy words).
__global__ void k_init_entries(DevFilm f) {
    const int wb = f.item_wbits, jb = f.item_jbits;
    const uint32_t wmask = (1u << wb) - 1u, jmask = (1u << jb) - 1u;
    uint32_t* ent = const_cast<uint32_t*>(f.ient);
    uint4* vq = reinterpret_cast<uint4*>(const_cast<uint32_t*>(f.ivq));
    for (int c = 0; c < 4; ++c) {
        const uint32_t* list = f.items + (int64_t)c * f.item_cap;
        for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < f.nitems[c]; it += gridDim.x * blockDim.x) {
            const uint32_t e = list[it];
            const int z = (int)(e >> (jb + wb)), j = (int)((e >> wb) & jmask), w = (int)(e & wmask);
            const int64_t at = (int64_t)c * f.item_cap + it;
            if (!f.packed) {    // int8: a 16-site chunk's byte offset and Philox counter
                ent[2 * at] = (uint32_t)addr8(f, c, z, j, 16 * w) | ((uint32_t)(z & 1) << 31);
                ent[2 * at + 1] = block_counter(f, c, z, j, 16 * w);
                continue;
            }
            const int64_t base = addrw(f, c, z, j, w);
            const NbrClass& nc = f.nb[c][z & 1];
            const uint32_t* o = f.op + base;
            uint32_t vac[12];
            for (int k = 0; k < 9; ++k) vac[k] = ~o[nc.off[k]];
            for (int k = 9; k < 12; ++k)
                vac[k] = nc.sgn < 0 ? ~__funnelshift_l(o[nc.off[k] - 1], o[nc.off[k]], 1)
                                    : ~__funnelshift_r(o[nc.off[k]], o[nc.off[k] + 1], 1);
            uint4 v;
            popcount12(vac, v.x, v.y, v.z, v.w);
            vq[at] = v;
            ent[2 * at] = (uint32_t)base | ((uint32_t)(z & 1) << 31);
            ent[2 * at + 1] = block_counter(f, c, z, j, 32 * w);
        }
    }
}

// M = sum S, 2B = sum S * (neighbour sum), occupied sites, 2 * occupied bonds -> st->red[0..3]
// (a slab: over its own rows, with its halo rows as neighbours).
__global__ void k_recompute(DevFilm f, FilmState* st) {
    const int64_t total = (int64_t)f.L * f.R * f.C;
    long long m = 0, b2 = 0, occ = 0, nb2 = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(t % f.C);
        const int64_t r = t / f.C;
        const int y = (int)(r % f.R), z = (int)(r / f.R);
        if (f.slab && (y < 2 * f.jlo || y >= 2 * f.jhi)) continue;   // a slab counts its own rows
        if (!site_occupied(f, x, y, z)) continue;
        const int s = site_spin(f, x, y, z);
        int n = 0, no = 0;
        for (int k = 0; k < 12; ++k) {
            int a, b, c;
            if (!neighbour_of(f, x, y, z, k, a, b, c)) continue;
            if (!site_occupied(f, a, b, c)) continue;
            n += site_spin(f, a, b, c);
            ++no;
        }
        m += s;
        b2 += (long long)s * n;
        occ += 1;
        nb2 += no;
    }
    m = warp_sum(m);
    b2 = warp_sum(b2);
    occ = warp_sum(occ);
    nb2 = warp_sum(nb2);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&st->red[0]), (unsigned long long)m);
        atomicAdd(reinterpret_cast<unsigned long long*>(&st->red[1]), (unsigned long long)b2);
        atomicAdd(reinterpret_cast<unsigned long long*>(&st->red[2]), (unsigned long long)occ);
        atomicAdd(reinterpret_cast<unsigned long long*>(&st->red[3]), (unsigned long long)nb2);
    }
}

__global__ void k_unpack(DevFilm f, int8_t* out) {
    const int64_t total = (int64_t)f.L * f.R * f.C;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(t % f.C);
        const int64_t r = t / f.C;
        const int y = (int)(r % f.R), z = (int)(r / f.R);
        out[t] = (int8_t)site_spin(f, x, y, z);
    }
}

// Simulated PMOKE image (Sec. 6): per pixel the surface atom, which is at z = H(x,y) - 1 since
// a pixel fills its layers from the substrate up; 255 if its spin is up, 0 if down, 128 where
// the pixel holds no atom.  *up counts the white pixels.
__global__ void k_surface(DevFilm f, uint8_t* out, unsigned long long* up) {
    const int64_t total = (int64_t)f.R * f.C;
    unsigned long long n = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(t % f.C), y = (int)(t / f.C);
        const int H = f.heights[t];
        uint8_t v = 128;
        if (H > 0) {
            v = site_spin(f, x, y, H - 1) > 0 ? 255 : 0;
            n += v == 255;
        }
        out[t] = v;
    }
    n = (unsigned long long)warp_sum((long long)n);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(up, n);
}

// ---- domains of the PMOKE image (Sec. 6, Fig. 5) -------------------------------------------
// Pixels are neighbours when their columns are in-plane neighbours of the film: (x +- 1, y),
// (x, y +- 1), (x + 1, y - 1), (x - 1, y + 1), wrapping on periodic axes.  A domain is a
// connected set of white (up) or of black (down) pixels; pixels with no atom belong to none.
// Union-find: every pixel starts as its own root; each pixel links with its three "forward"
// neighbours of the same colour (roots linked smaller-index-wins by compare-and-swap, retried
// a bounded number of times); then every pixel takes its root as label.

constexpr int kUnionTries = 1 << 20;

__device__ __forceinline__ int dom_find(const int* parent, int x) {
    int guard = 0;
    while (parent[x] != x && ++guard < kUnionTries) x = parent[x];
    return x;
}

__device__ __forceinline__ bool dom_union(int* parent, int a, int b) {
    for (int tries = 0; tries < kUnionTries; ++tries) {
        a = dom_find(parent, a);
        b = dom_find(parent, b);
        if (a == b) return true;
        if (a < b) { const int t = a; a = b; b = t; }       // link the larger root under the smaller
        const int old = atomicCAS(&parent[a], a, b);
        if (old == a) return true;
        a = old;
    }
    return false;
}

__global__ void k_dom_init(int64_t n, const uint8_t* img, int* parent) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        parent[p] = (int)p;
}

__global__ void k_dom_merge(int R, int C, uint32_t flags, const uint8_t* img, int* parent, int* bad) {
    const int64_t n = (int64_t)R * C;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t v = img[p];
        if (v == 128) continue;
        const int x = (int)(p % C), y = (int)(p / C);
        const int dx[3] = {1, 0, -1}, dy[3] = {0, 1, 1};
        for (int k = 0; k < 3; ++k) {
            int xx = x + dx[k], yy = y + dy[k];
            if (xx < 0 || xx >= C) {
                if (!(flags & 1u)) continue;
                xx = (xx + C) % C;
            }
            if (yy >= R) {
                if (!(flags & 2u)) continue;
                yy -= R;
            }
            const int q = yy * C + xx;
            if (img[q] == v && !dom_union(parent, (int)p, q)) atomicExch(bad, 1);
        }
    }
}

// out: [0] white domains, [1] black domains, [2] largest white, [3] largest black
__global__ void k_dom_count(int64_t n, const uint8_t* img, int* parent, int* size, unsigned long long* out) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        if (img[p] == 128) continue;
        const int r = dom_find(parent, (int)p);
        const int s = atomicAdd(&size[r], 1) + 1;
        const int w = img[p] == 255 ? 0 : 1;
        atomicMax(&out[2 + w], (unsigned long long)s);
        if (r == (int)p) atomicAdd(&out[w], 1ull);
    }
}

__global__ void k_philox_blocks(uint64_t seed, uint32_t stream_id, uint64_t sweep, uint32_t q0,
                                int64_t n, uint4* out) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n;
         b += (int64_t)gridDim.x * blockDim.x) {
        out[b] = philox10(make_uint4(q0 + (uint32_t)b, (uint32_t)sweep, (uint32_t)(sweep >> 32), stream_id),
                          (uint32_t)seed, (uint32_t)(seed >> 32));
    }
}

}  // namespace

int launch_init(const DevFilm& f, int init, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (f.packed) {
        const int64_t total = (int64_t)4 * (f.L + 2) * (f.Rh + 2) * f.Wp;
        k_init_packed<<<grid_for(total), kThreads, 0, s>>>(f, init, nullptr);
    } else {
        const int64_t total = (int64_t)4 * (f.L + 2) * (f.Rh + 2) * (f.P / 4);
        k_init_int8<<<grid_for(total), kThreads, 0, s>>>(f, init, nullptr);
    }
    return (int)cudaGetLastError();
}

int launch_init_entries(const DevFilm& f, void* stream) {
    if (!f.items || !f.narrow || !f.ient || (f.packed && !f.ivq)) return (int)cudaErrorInvalidValue;
    int64_t n = 0;
    for (int c = 0; c < 4; ++c) n = n > f.nitems[c] ? n : f.nitems[c];
    if (n == 0) return (int)cudaSuccess;
    k_init_entries<<<grid_for(n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(f);
    return (int)cudaGetLastError();
}

int launch_pack(const DevFilm& f, const int8_t* dev_in, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (f.packed) {
        const int64_t total = (int64_t)4 * (f.L + 2) * (f.Rh + 2) * f.Wp;
        k_init_packed<<<grid_for(total), kThreads, 0, s>>>(f, 0, dev_in);
    } else {
        const int64_t total = (int64_t)4 * (f.L + 2) * (f.Rh + 2) * (f.P / 4);
        k_init_int8<<<grid_for(total), kThreads, 0, s>>>(f, 0, dev_in);
    }
    return (int)cudaGetLastError();
}

int launch_recompute(const DevFilm& f, FilmState* st, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(st->red, 0, sizeof(st->red), s);
    if (e != cudaSuccess) return (int)e;
    const int64_t total = (int64_t)f.L * f.R * f.C;
    k_recompute<<<grid_for(total), kThreads, 0, s>>>(f, st);
    return (int)cudaGetLastError();
}

int launch_unpack(const DevFilm& f, int8_t* dev_out, void* stream) {
    const int64_t total = (int64_t)f.L * f.R * f.C;
    k_unpack<<<grid_for(total), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(f, dev_out);
    return (int)cudaGetLastError();
}

int launch_surface(const DevFilm& f, uint8_t* dev_out, unsigned long long* dev_up, void* stream) {
    const int64_t total = (int64_t)f.R * f.C;
    k_surface<<<grid_for(total), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(f, dev_out, dev_up);
    return (int)cudaGetLastError();
}

int launch_surface_domains(const DevFilm& f, const uint8_t* dev_img, int* dev_scratch, unsigned long long* dev_out4,
                           int* dev_bad, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = (int64_t)f.R * f.C;
    int* parent = dev_scratch;
    int* size = dev_scratch + n;
    cudaError_t e = cudaMemsetAsync(size, 0, (size_t)n * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dev_out4, 0, 4 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dev_bad, 0, sizeof(int), s);
    if (e != cudaSuccess) return (int)e;
    k_dom_init<<<grid_for(n), kThreads, 0, s>>>(n, dev_img, parent);
    k_dom_merge<<<grid_for(n), kThreads, 0, s>>>(f.R, f.C, f.flags, dev_img, parent, dev_bad);
    k_dom_count<<<grid_for(n), kThreads, 0, s>>>(n, dev_img, parent, size, dev_out4);
    return (int)cudaGetLastError();
}

int launch_philox_blocks(uint64_t seed, uint32_t stream_id, uint64_t sweep, uint32_t q0,
                         int64_t nblocks, uint32_t* dev_out, void* stream) {
    k_philox_blocks<<<grid_for(nblocks), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        seed, stream_id, sweep, q0, nblocks, reinterpret_cast<uint4*>(dev_out));
    return (int)cudaGetLastError();
}

}  // namespace isf
