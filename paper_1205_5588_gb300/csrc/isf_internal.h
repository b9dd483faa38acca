// isf_internal.h — data layout and launch interfaces shared by the library's host and device
// translation units.  Not part of the public ABI.
//
// Spin storage (one array set per colour c = ((x+z)&1) | (((y+z)&1)<<1), Sec. 3 "checkerboard"):
// a site (x, y, z) of colour c lives at column i = x>>1, row j = y>>1, layer z of colour c's
// array.  Its x parity is (c&1)^(z&1) and its y parity ((c>>1)&1)^(z&1), so inside one
// (colour, layer parity) class every one of the 12 neighbours sits at a FIXED address offset
// (one of three of them shifted by one column), which is what makes the colour pass a
// stencil with constant offsets.
//
//  int8 layout  : per colour [L+2][Rh+2][P] bytes, halo layer/row on each side, 16 halo bytes
//                 left of column 0; P = 16*(nck+2), nck = ceil(Ch/16).  Byte values:
//                 0 = spin down, 1 = vacancy (also every halo/padding byte), 2 = spin up,
//                 i.e. S + 1, so a plain 32-bit add of 12 neighbour words gives n + 12 per
//                 byte (n = neighbour spin sum, no carries: at most 24).
//  packed layout: per colour two bit-planes [L+2][Rh+2][Wp] uint32 (spin bit = 1 for up,
//                 occupancy bit = 1 for occupied, both 0 on vacancies and halos); word w of a
//                 row holds columns 32w..32w+31 and sits at index w+1; Wp = nw + 2.
#pragma once
#include <stdint.h>
#include <vector>
#include <stddef.h>

#ifdef __CUDACC__
#define ISF_HD __host__ __device__
#else
#define ISF_HD
#endif

namespace isf {

constexpr uint32_t kAlways = 0xFFFFFFFFu;
constexpr int kTableStride = 52;    // per step: thr[n+12][s'] (50 words), gate threshold, flags
constexpr int kGateSlot = 50;
constexpr int kFlagSlot = 51;
// Step flag: a site whose 12 neighbours all share its spin still needs a random word (its
// threshold is neither 0 nor "always"), so nearly every group of sites draws words and the
// kernels skip the test of whether a group needs them.  A scheduling hint only: the words
// drawn and the decisions are the same either way.
constexpr uint32_t kFlagAlwaysDraw = 1u;
// Step flag: no threshold of the step is 0 ("never").  The packed kernel then decides a lane by
// the carry of u + (2^32 - thr) (no carry: accepted; "always" is stored as 0), which cannot
// encode "never".  The decisions are the same either way.
constexpr uint32_t kFlagNoNever = 2u;
constexpr int kMaxThreads = 1024;
constexpr int kMaxSlabCTAs = 192;     // row-slab kernel: most CTAs (one per SM)
constexpr int kSeriesChunk = 2048;    // row-slab kernel: most sweeps per launch
constexpr int kSlabMaxLayers = 16;    // row-slab kernel: most layers
constexpr uint32_t kSlabStaticSmem = 3072;   // row-slab kernel: its static shared arrays, rounded up

// Neighbour offsets of one (colour, layer parity) class: 9 unshifted, then 3 shifted by `sgn`
// columns (-1 or +1).  Units: bytes (int8) or words (packed).
struct NbrClass {
    int64_t off[12];
    int32_t sgn;
    int32_t pad_;
    int8_t c2[12], dz[12], dj[12];   // same order: neighbour colour, layer step, row step
    int8_t pad2_[4];
};

struct DevFilm {
    // geometry
    int32_t R, C, L;
    int32_t Rh, Ch, Qw;
    uint32_t flags;
    int32_t packed;
    uint32_t key0, key1;
    // int8 layout
    uint8_t* s8;
    int64_t P, ls8, cs8;          // row pitch, layer stride, colour stride (bytes)
    int32_t nck;                  // 16-site chunks per row
    // packed layout
    uint32_t* sp;                 // spin bit-planes
    uint32_t* op;                 // occupancy bit-planes

    int64_t Wp, lsw, csw;         // row pitch, layer stride, colour stride (words)
    int32_t nw;                   // words per row
    int32_t pad_;
    // per colour the items (packed: 32-site words; int8: 16-site chunks) holding at least one
    // occupied site, in (z, row, item) order, each (z << (jbits + wbits)) | (j << wbits) | w;
    // nullptr when not built
    const uint32_t* items;        // [4][item_cap]
    int64_t item_cap;
    int32_t nitems[4];
    int32_t item_wbits, item_jbits;
    int32_t narrow;               // 1 if every neighbour offset and index (words / bytes) fits 32 bits
    // with lists (only narrow films have them): per list entry (same indexing as items) the word
    // index (packed) or byte offset (int8) with the layer parity in bit 31 and the Philox counter
    // (ient, 2 words); packed: the bit-sliced count of vacant neighbours (1s, 2s, 4s, 8s) of its
    // 32 sites (ivq, 4 words, 16-byte aligned); fixed by the occupancy; nullptr when absent
    const uint32_t* ient;
    const uint32_t* ivq;
    // row slab of a larger film (0: a whole film).  Local colour-row j is row (j + cj0) mod cRh
    // of the whole film (its Philox counters are the whole film's); the sweep kernels update
    // rows [jlo, jhi) only, the others are halo copies of the neighbouring slabs' rows.
    int32_t slab;
    int32_t cRh, cj0, jlo, jhi;
    const uint8_t* heights;       // [y][x]
    NbrClass nb[4][2];            // [colour][layer parity]
};

// Running state of one film on the device (library scratch, 256-byte aligned).
struct FilmState {
    long long M, B;               // magnetisation sum, bond sum (after the last folded sweep)
    long long acc[2][2];          // per-sweep deltas (dM, dB), double-buffered by sweep parity
    unsigned int bar_count, bar_gen;
    int error;                    // isf_status set by a kernel (0 = fine)
    int error_where;
    long long n_meas, sumM, sumAbsM, sumB;      // running sums of the current step
    unsigned long long sumM2[2], sumB2[2], sumMB[2];
    long long red[4];             // reduction scratch of the recompute kernel
    long long pad_[6];
};

// Exact per-step record written by the device at the end of each step.
struct StepRec {
    long long M_last, B_last, n_meas, sumM, sumAbsM, sumB;
    unsigned long long sumM2[2], sumB2[2], sumMB[2];
};

// Arguments of one sweep launch.
struct SweepArgs {
    DevFilm f;
    FilmState* st;
    const uint32_t* tables;       // [nsteps][kTableStride]
    const int32_t* step_eq;       // [nsteps]
    const int32_t* step_total;    // [nsteps] eq + meas
    StepRec* recs;                // [nsteps]
    long long* trace;             // optional (M, B) per sweep
    long long trace_begin, trace_cap;  // trace index of the first sweep of this launch, capacity
    long long sweep0;             // sweeps done before this launch; first RNG sweep = sweep0 + 1
    long long nsweeps;
    int32_t k0, pos0;             // schedule cursor at launch: step, sweeps done in that step
    int32_t nsteps;
    int32_t use_gate;             // any step with a gate threshold != always
    int32_t pass_plus1;           // 0: whole sweeps; c + 1: colour c of one sweep only (slab mode)
};

// Host-side layout computation (lattice.cpp).
struct Layout {
    int32_t R, C, L, Rh, Ch, Qw;
    uint32_t flags;
    bool packed;
    int64_t P, ls8, cs8, nck;
    int64_t nw, Wp, lsw, csw;
    size_t spin_bytes;            // int8 array, or both bit-plane sets
    size_t heights_off, state_off, total_bytes;
    size_t items_off;             // occupied-item lists, 4 x items_cap uint32
    int64_t items_cap;            // packed: L * Rh * nw; int8 with open boundaries: L * Rh * nck; else 0
    size_t ient_off;              // 4 x items_cap x 8 B (DevFilm.ient)
    size_t ivq_off;               // packed: 4 x items_cap x 16 B (DevFilm.ivq)
    // packed: row-slab kernel scratch (kernels_slabs.cu)
    size_t roff_off;              // 4 x L x (Rh + 1) int32: first list entry of each (colour, z, row)
    size_t part_off;              // (kMaxSlabCTAs + 1) int32: first row of each CTA
    size_t done_off;              // slab_gmax x 32 uint32: boundary words published, one line per CTA
    size_t xbuf_off;              // slab_gmax x 4 x 2 rows of L x nw uint32 (stride rounded up to 4): boundary rows
    size_t series_off;            // kSeriesChunk x 2 uint64: dM, dB per sweep
    int32_t slab_gmax;            // most CTAs the slab kernel may use (min(kMaxSlabCTAs, Rh))
};

int make_layout(int32_t rows, int32_t cols, int32_t layers, uint32_t flags, Layout* out,
                const char** why);
int check_colouring(const Layout& lay, const char** why);
// Occupied-word lists of a packed film (host, from the height map): out gets 4 * items_cap
// entries (colour c's list at c * items_cap, n[c] of them, in (z, row, word) order); false when
// an entry's fields do not fit 32 bits (the kernels then walk every word).  Rows [jlo, jhi)
// only.  roff (optional): 4 x L x (Rh + 1) offsets, the words of colour c, layer z, row j being
// entries [roff[(c L + z)(Rh + 1) + j], roff[(c L + z)(Rh + 1) + j + 1]).
bool build_word_items(const Layout& lay, const uint8_t* heights, std::vector<uint32_t>& out, int32_t n[4],
                      int32_t* wbits, int32_t* jbits, int32_t jlo, int32_t jhi, std::vector<int32_t>* roff = nullptr);
void fill_neighbour_classes(const Layout& lay, DevFilm* f);
// Whether a film of this layout keeps item lists: its offsets, neighbours included, fit 32 bits.
bool lists_fit_32_bits(const Layout& lay);

// Host threshold table (schedule.cpp): thr[n+12][s'] for one step, plus the gate slot.
void build_step_table(double T, double h, double J, double h_s, uint32_t* out52);
// FP64 derivation from exact sums (schedule.cpp).
void derive_record(const StepRec& r, double T, double h, double J, long long n_occ,
                   double out[6]);

// Device launchers (kernels.cu); all return a cudaError_t as int.
int launch_init(const DevFilm& f, int init, void* stream);
// Fills f.ient and f.ivq from the word lists and the occupancy planes (packed, after launch_init).
int launch_init_entries(const DevFilm& f, void* stream);
int launch_recompute(const DevFilm& f, FilmState* st, void* stream);  // M, B, n_occ, bonds -> st->red
int launch_sweeps(const SweepArgs& a, int ctas, int threads, void* stream);
int launch_unpack(const DevFilm& f, int8_t* dev_out, void* stream);
int launch_pack(const DevFilm& f, const int8_t* dev_in, void* stream);
int launch_surface(const DevFilm& f, uint8_t* dev_out, unsigned long long* dev_up, void* stream);
// Domains of a surface image already on the device (R*C bytes): dev_scratch holds 2*R*C ints;
// dev_out4 = {white domains, black domains, largest white, largest black}; *dev_bad = 1 if a
// bounded union retry ran out.
int launch_surface_domains(const DevFilm& f, const uint8_t* dev_img, int* dev_scratch, unsigned long long* dev_out4,
                           int* dev_bad, void* stream);
int launch_philox_blocks(uint64_t seed, uint32_t stream_id, uint64_t sweep, uint32_t q0,
                         int64_t nblocks, uint32_t* dev_out, void* stream);
int sweep_max_ctas_for(const DevFilm& f, int threads, int* max_ctas);  // co-resident CTAs
// The packed word-list kernel (kernels_words.cu): a cooperative launch of ctas >= 2 CTAs for a
// bit-packed whole film with occupied-word lists; co-resident CTAs with this block size.
int launch_words(const SweepArgs& a, int ctas, int threads, void* stream);
int words_max_ctas(int threads, int* out);
// `ctas` co-resident CTAs wait at the grid barrier for an arrival nothing makes (kernels_sweep.cu);
// *status, *where: the status word and wait site the kernel recorded.
int wait_probe(int ctas, int* status, int* where);

// Row slabs in shared memory (kernels_slabs.cu): a packed film split by rows over G co-resident
// CTAs, each holding its rows and one halo row on each side in shared memory.  A CTA updates its
// two boundary rows first in every colour pass and publishes them (xbuf, done); at the end of
// the pass it imports its neighbours' boundary rows of that colour into its halo.  No grid
// barrier: a CTA waits only for its two neighbours.
struct alignas(16) SlabArgs {
    SweepArgs s;
    const int32_t* part;          // [G + 1] first colour row of each CTA (part[G] = Rh)
    const int32_t* roff;          // [4][L][Rh + 1] first list entry of each (colour, z, row)
    uint32_t* xbuf;               // [G][4][2] rows of L x nw words, stride rounded up to 4: boundary rows
                                  // (side 0: the first own row, 1: the last)
    unsigned* done;               // [G][32] 1 + boundary words each CTA has published this launch
    unsigned long long* series;   // [nsweeps][2] per-sweep dM, dB (two's complement sums)
    int32_t nrm;                  // most rows of any CTA
    int32_t pad_;
};
// Shared memory of a CTA of the row-slab kernel whose largest slab has nrm rows.
uint32_t slab_smem_bytes(const DevFilm& f, int nrm);
// Co-resident CTAs of the row-slab kernel with this block size and shared memory (0 when the
// shared memory does not fit).
int slab_units(int threads, uint32_t smem, int* units);
int launch_slabs(const SlabArgs& a, int G, int threads, uint32_t smem, void* stream);
// Folds a launch's per-sweep series into M, B, the step sums and records (one thread).
int launch_fold_series(const SweepArgs& a, const unsigned long long* series, void* stream);

// Cluster-resident sweeps (kernels_resident.cu): the film sits in the shared memory of one
// thread-block cluster of K CTAs (row slabs), int8 layout, any boundary flags.
struct ResPlan {
    int32_t K, Jb, threads;
    uint32_t film_off, vac_off, ptr_off, misc_off, smem;
    int32_t item_sites;     // 16 or 8 sites per work item
};
// Plan for a film: K = want_K (0: automatic), threads = want_threads (0: automatic), sites per
// work item = want_sites (0: automatic, 8 or 16).  Returns 0 and fills out when the film fits,
// else a nonzero code (no device work).
int resident_plan(const DevFilm& f, int want_K, int want_threads, int want_sites, ResPlan* out);
int launch_resident(const SweepArgs& a, const ResPlan& plan, void* stream);

// One film's launch arguments for the resident kernels (also the batch queue's entries).
struct alignas(16) ResArgs {
    SweepArgs s;
    int32_t K, Jb;
    uint32_t film_off, vac_off, ptr_off, misc_off;
};
static_assert(sizeof(ResArgs) % 16 == 0, "ResArgs is copied in 16-byte words");
ResArgs make_res_args(const SweepArgs& a, const ResPlan& p);
// First out-of-range access a resident / batch kernel skipped (all zeros when none).
int read_checks(unsigned long long out[4]);

// Batched films (kernels_resident.cu): a persistent launch of `units` CTAs (K = 1) or clusters
// of K CTAs, each taking films from the device queue `films[0..n)` via the counter *next.
int batch_units_possible(int K, int threads, uint32_t smem, int* units);
int launch_batch(const ResArgs* films, int n, unsigned* next, int K, int threads, uint32_t smem,
                 int units, void* stream);
int sweep_items_per_pass(const DevFilm& f);                            // work items per colour pass
// Batched films one CTA each in global memory (kernels_sweep.cu): `units` persistent CTAs take
// films from the device queue films[0..n) via the counter *next; any layout and boundary.
int batch_global_units(int threads, int* units);
// A resident queue whose films a global-memory queue kernel takes once its own queue is empty
// (films[0..n) claimed through the same counter *next as the resident kernel; n = 0: none).
struct StealQueue {
    const ResArgs* films;
    int32_t n;
    unsigned* next;
    unsigned* taken;    // films the global-memory kernel took from this queue
};
int launch_batch_global(const SweepArgs* films, int n, unsigned* next, int threads, int units, void* stream,
                        StealQueue steal);
// The same with one thread-block cluster of K (2, 4 or 8) CTAs per film.
int batch_cluster_global_units(int K, int threads, int* units);
int launch_batch_cluster_global(const SweepArgs* films, int n, unsigned* next, int K, int threads, int units,
                                void* stream, StealQueue steal);

}  // namespace isf
