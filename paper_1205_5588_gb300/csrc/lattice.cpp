// lattice.cpp — host side of the film lattice: extents check, device layout, colouring proof
// and the per-class neighbour offsets the colour-pass kernels use.
//
// Geometry (Sec. 2 and item 2 of Sec. 3 fix only "coordination number 12"): FCC in primitive
// coordinates with constant-z planes as ABC-stacked triangular layers.  Neighbour offsets:
// (+-1,0,0), (0,+-1,0), +-(1,-1,0) in-plane, (0,0,1), (0,-1,1), (-1,0,1) up,
// (0,0,-1), (0,1,-1), (1,0,-1) down.
#include <algorithm>
#include <cstdio>

#include "isf_internal.h"
#include "../../include/isingfilm.h"

namespace isf {

namespace {

const int kStencil[12][3] = {
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {0, 0, 1}, {0, -1, 1}, {-1, 0, 1},
    {0, 0, -1}, {0, 1, -1}, {1, 0, -1},
};

inline int colour_of(long x, long y, long z) {
    return (int)(((x + z) & 1) | (((y + z) & 1) << 1));
}

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// floor division by 2 for small signed values
inline int fdiv2(int v) { return v >= 0 ? v / 2 : -((-v + 1) / 2); }

}  // namespace

int make_layout(int32_t rows, int32_t cols, int32_t layers, uint32_t flags, Layout* out,
                const char** why) {
    if (rows < 1 || cols < 1 || layers < 1) { *why = "rows, cols and layers must be >= 1"; return ISF_ERR_ARG; }
    if (rows > 65536 || cols > 65536) { *why = "rows and cols must be <= 65536"; return ISF_ERR_ARG; }
    if (layers > 255) { *why = "layers must be <= 255 (heights are uint8)"; return ISF_ERR_ARG; }
    const uint32_t known = ISF_PERIODIC_X | ISF_PERIODIC_Y | ISF_PERIODIC_Z | ISF_PACKED;
    if (flags & ~known) { *why = "unknown flag bits"; return ISF_ERR_ARG; }
    const bool packed = (flags & ISF_PACKED) != 0;
    const uint32_t per = flags & (ISF_PERIODIC_X | ISF_PERIODIC_Y | ISF_PERIODIC_Z);
    if (packed && per) { *why = "the packed layout supports open boundaries only (use int8 for periodic films)"; return ISF_ERR_ARG; }
    // Parity colouring survives a wrap only across an even extent; >= 4 keeps the +1 and -1
    // neighbours along the axis distinct.
    if ((per & ISF_PERIODIC_X) && (cols % 2 || cols < 4)) { *why = "periodic x needs an even cols >= 4"; return ISF_ERR_COLOURING; }
    if ((per & ISF_PERIODIC_Y) && (rows % 2 || rows < 4)) { *why = "periodic y needs an even rows >= 4"; return ISF_ERR_COLOURING; }
    if ((per & ISF_PERIODIC_Z) && (layers % 2 || layers < 4)) { *why = "periodic z needs an even layers >= 4"; return ISF_ERR_COLOURING; }

    Layout L{};
    L.R = rows; L.C = cols; L.L = layers; L.flags = flags; L.packed = packed;
    L.Rh = (rows + 1) / 2;
    L.Ch = (cols + 1) / 2;
    L.Qw = (L.Ch + 3) / 4;
    // Philox counter word q = ((c*L + z)*Rh + j)*Qw + i/4 must fit 32 bits.
    if ((uint64_t)4 * (uint64_t)layers * (uint64_t)L.Rh * (uint64_t)L.Qw > 0xFFFFFFFFull) {
        *why = "film too large for the 32-bit Philox site counter";
        return ISF_ERR_ARG;
    }
    L.nck = (L.Ch + 15) / 16;
    L.P = 16 * (L.nck + 2);
    L.ls8 = (int64_t)(L.Rh + 2) * L.P;
    L.cs8 = (int64_t)(layers + 2) * L.ls8;
    L.nw = (L.Ch + 31) / 32;
    L.Wp = L.nw + 2;
    L.lsw = (int64_t)(L.Rh + 2) * L.Wp;
    L.csw = (int64_t)(layers + 2) * L.lsw;
    L.spin_bytes = packed ? (size_t)2 * 4 * (size_t)L.csw * 4 : (size_t)4 * (size_t)L.cs8;
    L.heights_off = align256(L.spin_bytes);
    L.state_off = align256(L.heights_off + (size_t)rows * (size_t)cols);
    // occupied-item lists: 32-site words of packed films, 16-site chunks of int8 films with open
    // boundaries (periodic int8 films run the generic path, which walks every site)
    L.items_cap = packed ? (int64_t)layers * L.Rh * L.nw : (per ? 0 : (int64_t)layers * L.Rh * L.nck);
    L.items_off = align256(L.state_off + sizeof(FilmState));
    size_t end = L.items_off + (size_t)4 * (size_t)L.items_cap * sizeof(uint32_t);
    L.ient_off = align256(end);
    end = L.ient_off + (size_t)4 * (size_t)L.items_cap * 8;
    if (packed) {
        L.ivq_off = align256(end);
        end = L.ivq_off + (size_t)4 * (size_t)L.items_cap * 16;
        L.slab_gmax = std::min(kMaxSlabCTAs, L.Rh);
        L.roff_off = align256(end);
        L.part_off = align256(L.roff_off + (size_t)4 * (size_t)layers * (size_t)(L.Rh + 1) * sizeof(int32_t));
        L.done_off = align256(L.part_off + (size_t)(kMaxSlabCTAs + 1) * sizeof(int32_t));
        L.xbuf_off = align256(L.done_off + (size_t)L.slab_gmax * 32 * sizeof(uint32_t));
        L.series_off = align256(L.xbuf_off + (size_t)L.slab_gmax * 8 * (((size_t)layers * (size_t)L.nw + 3) & ~(size_t)3) * sizeof(uint32_t));
        end = L.series_off + (size_t)kSeriesChunk * 2 * sizeof(unsigned long long);
    }
    L.total_bytes = align256(end);
    *out = L;
    return ISF_OK;
}

static int bits_for(int64_t n) {
    int b = 0;
    while (((int64_t)1 << b) < n) ++b;
    return b;
}

bool build_word_items(const Layout& lay, const uint8_t* heights, std::vector<uint32_t>& out, int32_t n[4],
                      int32_t* wbits, int32_t* jbits, int32_t jlo, int32_t jhi, std::vector<int32_t>* roff) {
    // items of a colour row: 32-site words (packed) or 16-site chunks (int8)
    const int per_row = lay.packed ? (int)lay.nw : (int)lay.nck, shift = lay.packed ? 5 : 4;
    if (lay.items_cap == 0) return false;
    const int wb = bits_for(per_row), jb = bits_for(lay.Rh), zb = bits_for(lay.L);
    if (wb + jb + zb > 32) return false;
    out.assign((size_t)4 * (size_t)lay.items_cap, 0u);
    // tallest pixel among the columns of each (row y, column parity, item w): an item of layer z
    // holds an occupied site iff z < that height
    std::vector<uint8_t> top((size_t)lay.R * 2 * per_row, 0);
    for (int y = 0; y < lay.R; ++y)
        for (int x = 0; x < lay.C; ++x) {
            uint8_t& t = top[((size_t)y * 2 + (x & 1)) * per_row + ((x >> 1) >> shift)];
            t = std::max(t, heights[(size_t)y * lay.C + x]);
        }
    if (roff) roff->assign((size_t)4 * (size_t)lay.L * (size_t)(lay.Rh + 1), 0);
    for (int c = 0; c < 4; ++c) {
        uint32_t* dst = out.data() + (size_t)c * lay.items_cap;
        int64_t k = 0;
        for (int z = 0; z < lay.L; ++z) {
            const int zp = z & 1, px = (c & 1) ^ zp, py = ((c >> 1) & 1) ^ zp;
            int32_t* ro = roff ? roff->data() + ((size_t)c * lay.L + z) * (lay.Rh + 1) : nullptr;
            for (int j = 0; j < lay.Rh; ++j) {
                if (ro) ro[j] = (int32_t)k;
                const int y = 2 * j + py;
                if (j < jlo || j >= jhi || y >= lay.R) continue;
                for (int w = 0; w < per_row; ++w)
                    if (z < top[((size_t)y * 2 + px) * per_row + w])
                        dst[k++] = ((uint32_t)z << (jb + wb)) | ((uint32_t)j << wb) | (uint32_t)w;
            }
            if (ro) ro[lay.Rh] = (int32_t)k;
        }
        n[c] = (int32_t)k;
    }
    *wbits = wb;
    *jbits = jb;
    return true;
}

// Proof that no bond joins two sites of one colour on this film.  Away from a wrap the colour
// of (x+dx, y+dy, z+dz) depends only on the parities of x, y, z and on the offset, so all 8
// parity classes x 12 offsets are checked exhaustively; bonds that cross a periodic boundary
// are then checked one by one on the boundary faces.
int check_colouring(const Layout& lay, const char** why) {
    for (int px = 0; px < 2; ++px)
        for (int py = 0; py < 2; ++py)
            for (int pz = 0; pz < 2; ++pz)
                for (int k = 0; k < 12; ++k) {
                    int c0 = colour_of(px, py, pz);
                    int c1 = colour_of(px + kStencil[k][0], py + kStencil[k][1], pz + kStencil[k][2]);
                    if (c0 == c1) { *why = "stencil joins equal colours"; return ISF_ERR_COLOURING; }
                }
    const long ext[3] = {lay.C, lay.R, lay.L};
    const uint32_t pbit[3] = {ISF_PERIODIC_X, ISF_PERIODIC_Y, ISF_PERIODIC_Z};
    for (int ax = 0; ax < 3; ++ax) {
        if (!(lay.flags & pbit[ax])) continue;
        // every site on the two faces normal to this axis
        for (int face = 0; face < 2; ++face) {
            long a_fixed = face ? ext[ax] - 1 : 0;
            int o1 = (ax + 1) % 3, o2 = (ax + 2) % 3;
            for (long u = 0; u < ext[o1]; ++u)
                for (long v = 0; v < ext[o2]; ++v) {
                    long p[3];
                    p[ax] = a_fixed; p[o1] = u; p[o2] = v;
                    for (int k = 0; k < 12; ++k) {
                        long q[3];
                        bool inside = true;
                        for (int d = 0; d < 3; ++d) {
                            q[d] = p[d] + kStencil[k][d];
                            if (q[d] < 0 || q[d] >= ext[d]) {
                                if (!(lay.flags & pbit[d])) { inside = false; break; }
                                q[d] = (q[d] + ext[d]) % ext[d];
                            }
                        }
                        if (!inside) continue;
                        if (q[0] == p[0] && q[1] == p[1] && q[2] == p[2]) {
                            *why = "a site is its own neighbour across a wrap";
                            return ISF_ERR_COLOURING;
                        }
                        if (colour_of(p[0], p[1], p[2]) == colour_of(q[0], q[1], q[2])) {
                            *why = "a bond across a periodic boundary joins equal colours";
                            return ISF_ERR_COLOURING;
                        }
                    }
                }
        }
    }
    return ISF_OK;
}

// For colour c and layer parity zp, the site at column i, row j has x = 2i + px, y = 2j + py
// with px = (c&1)^zp, py = ((c>>1)&1)^zp.  Neighbour (dx,dy,dz) is at column i + floor((px+dx)/2)
// and row j + floor((py+dy)/2) of colour c' in layer z + dz: a constant offset per class.
void fill_neighbour_classes(const Layout& lay, DevFilm* f) {
    for (int c = 0; c < 4; ++c)
        for (int zp = 0; zp < 2; ++zp) {
            const int px = (c & 1) ^ zp, py = ((c >> 1) & 1) ^ zp;
            NbrClass nc{};
            int64_t plain8[12], plainw[12];
            int8_t pc[12], pz[12], pj[12], sc[3], sz[3], sj[3];
            int np = 0, ns = 0, sgn = 0;
            int64_t sh8[3] = {0, 0, 0}, shw[3] = {0, 0, 0};
            for (int k = 0; k < 12; ++k) {
                const int dx = kStencil[k][0], dy = kStencil[k][1], dz = kStencil[k][2];
                const int di = fdiv2(px + dx), dj = fdiv2(py + dy);
                const int c2 = colour_of(px + dx, py + dy, zp + dz);
                const int64_t row8 = (int64_t)(c2 - c) * lay.cs8 + dz * lay.ls8 + dj * lay.P;
                const int64_t roww = (int64_t)(c2 - c) * lay.csw + dz * lay.lsw + dj * lay.Wp;
                if (di == 0) {
                    plain8[np] = row8; plainw[np] = roww;
                    pc[np] = (int8_t)c2; pz[np] = (int8_t)dz; pj[np] = (int8_t)dj;
                    ++np;
                } else {
                    sgn = di;   // the same sign for all three: -1 when px = 0, +1 when px = 1
                    sh8[ns] = row8; shw[ns] = roww;
                    sc[ns] = (int8_t)c2; sz[ns] = (int8_t)dz; sj[ns] = (int8_t)dj;
                    ++ns;
                }
            }
            // np == 9, ns == 3 by construction of the stencil (checked by the caller's tests)
            for (int k = 0; k < 9; ++k) {
                nc.off[k] = lay.packed ? plainw[k] : plain8[k];
                nc.c2[k] = pc[k]; nc.dz[k] = pz[k]; nc.dj[k] = pj[k];
            }
            for (int k = 0; k < 3; ++k) {
                nc.off[9 + k] = lay.packed ? shw[k] : sh8[k];
                nc.c2[9 + k] = sc[k]; nc.dz[9 + k] = sz[k]; nc.dj[9 + k] = sj[k];
            }
            nc.sgn = sgn;
            f->nb[c][zp] = nc;
            (void)np; (void)ns;
        }
}

}  // namespace isf
