/*
 * isingfilm_tuning.h — tuning, measurement and test hooks of libisingfilm.so.
 *
 * These calls are not part of the method's boundary (include/isingfilm.h, which this header
 * includes): they choose or report the kernel and launch shape that runs a film, expose the
 * host-built work lists and row bands for checking against their definitions, draw raw device
 * Philox blocks for checking the generator, and probe the integer-issue ceilings that the
 * benchmark reports its roofline against.  Trajectories never depend on any of them.
 * Conventions (status codes, last error, streams) are those of isingfilm.h.
 */
#ifndef ISINGFILM_TUNING_H
#define ISINGFILM_TUNING_H

#include "isingfilm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Which sweep kernel runs the film (trajectories are identical on all of them):
 *   ISF_PATH_RESIDENT: the whole film in the shared memory of one thread-block cluster of up to
 *     16 CTAs (row slabs, neighbour rows through distributed shared memory, hardware cluster
 *     barrier between colour passes) — the paper's row decomposition with CTAs as processes
 *     (Sec. 3, list items 1-2); int8 films that fit only;
 *   ISF_PATH_GLOBAL: spins in device memory, all SMs, a grid barrier between colour passes;
 *   ISF_PATH_SLABS: packed films only; the film split by rows over up to one CTA per SM, each
 *     CTA's band of rows (plus one halo row on each side) in its shared memory, the boundary
 *     rows exchanged through device memory after each colour pass, and each CTA waiting for
 *     its two neighbours only (the same row decomposition, over the whole GPU); launches of at
 *     most 2048 sweeps, each followed by a one-thread fold of the per-sweep M, B series;
 *   ISF_PATH_AUTO (default): int8 films resident when the film fits, else global; packed films
 *     slabs when a colour pass has more than 512 and at most 4096 occupied words (films of
 *     roughly 150^2 to 350^2 sites per layer), else global.
 * Errors: ISF_ERR_ARG (unknown path; resident for a packed film; slabs for an int8 film, a slab
 * film or a packed film whose word lists could not be built). */
enum { ISF_PATH_AUTO = 0, ISF_PATH_GLOBAL = 1, ISF_PATH_RESIDENT = 2, ISF_PATH_SLABS = 3 };
int isf_set_path(isf_lattice* lat, int32_t path);

/* Launch shape override: ctas = CTAs of the global kernel, cluster size (1..16) of the resident
 * kernel, or row bands of the row-slab kernel (one CTA each, at most min(192, colour rows), all
 * co-resident) (0 = automatic); threads per CTA (0 = automatic; else a multiple of 32 up to 1024;
 * the global kernel uses at most 512; the row-slab kernel 64..512; the resident kernel 64..512
 * with 16-site items and 64..768 with 8-site items, one warp of which folds the observables and
 * takes no sites).  A shape the row-slab kernel cannot run makes isf_run_sweeps fail with
 * ISF_ERR_ARG when that path is forced.  Trajectories do not depend on it. */
int isf_set_launch(isf_lattice* lat, int32_t ctas, int32_t threads);

/* Sites per work item of the resident kernel: 16, 8, or 0 = automatic (8 when a quarter or more
 * of the sites of 16-site items would be padding past the end of the row, i.e. narrow rows).  An item is one thread's
 * share of a colour pass: the same row, consecutive columns (Sec. 3's checkerboard update).
 * Trajectories do not depend on it.  Errors: ISF_ERR_ARG (other values).  No device work. */
int isf_set_item_sites(isf_lattice* lat, int32_t sites);

/* The resident and batch kernels check every address they derive from a film's description and
 * skip (and record) an out-of-range access instead of making it.  This returns the first one
 * recorded in the process as (code, value, value, 0); all zeros when none.  The read functions
 * also report it as ISF_ERR_STATE. */
int isf_debug_checks(uint64_t* out4);

/* The occupied-item lists the library keeps for a film of this shape (host only, no device
 * work): per colour c the entries (z << (jbits + wbits)) | (j << wbits) | w, in (z, row, item)
 * order, of the items holding an occupied site — 32-site words (ISF_PACKED) or 16-site chunks
 * (int8 with open boundaries) of colour row j, layer z, where item w covers columns i (= x>>1)
 * 32w..32w+31 or 16w..16w+15 (Sec. 3's rows of one colour; occupancy as in isf_lattice_create).
 * heights: host, rows*cols; n_out[4]: entries per colour; out: 4 x cap uint32, colour c's list
 * from out[c * cap]; cap >= layers * ceil(rows/2) * items per row; bits_out[2] = (wbits, jbits).
 * The same checks as isf_lattice_create: a film it would refuse, or one it would keep without
 * lists, is refused here too.
 * Errors: ISF_ERR_ARG (bad shape or pointers, cap too small, a film without lists: periodic int8,
 * or offsets or fields that do not fit 32 bits), ISF_ERR_COLOURING. */
int isf_debug_item_lists(const uint8_t* heights, int32_t rows, int32_t cols, int32_t layers, uint32_t flags,
                         int32_t* n_out, uint32_t* out, int64_t cap, int32_t* bits_out);

/* The row bands ISF_PATH_SLABS would give a packed film of this shape split over `bands` CTAs
 * of at most max_rows colour rows each (host only, no device work): part_out[0..bands] (bands + 1
 * int32), band g holding colour rows [part_out[g], part_out[g+1]); contiguous, 1..max_rows rows
 * each, cut where the running count of occupied words (all colours and layers) is closest to an
 * even share (Sec. 3's split of the image rows between processes).  Errors: ISF_ERR_ARG (bad
 * shape or pointers, bands outside 1..colour rows, bands x max_rows below the colour rows, a film
 * the library keeps without word lists, which the row-slab path refuses). */
int isf_debug_slab_partition(const uint8_t* heights, int32_t rows, int32_t cols, int32_t layers, int32_t bands,
                             int32_t max_rows, int32_t* part_out);

/* Shape of the last isf_run_sweeps launch: path (ISF_PATH_GLOBAL / ISF_PATH_RESIDENT /
 * ISF_PATH_SLABS, 0 before any launch), CTAs (global), cluster size (resident) or row bands
 * (slabs), threads per CTA.  No device work. */
int isf_launch_info(isf_lattice* lat, int32_t* path, int32_t* ctas, int32_t* threads);
/* Sites per work item of the last isf_run_sweeps launch (16 or 8 resident, 16 int8 global, 32
 * packed global; 0 before any launch).  No device work. */
int isf_launch_item_sites(isf_lattice* lat, int32_t* sites);

/* Films of the last isf_batch_run_sweeps that a global-memory queue kernel took from a resident
 * queue of its size class once its own queue was empty: out2[0] from the single-CTA resident
 * queue, out2[1] from the cluster resident queue.  Waits for the run. */
int isf_batch_taken(isf_batch* batch, int32_t* out2);

/* Test of the bounded device waits: `ctas` (>= 2, all co-resident) CTAs of one cooperative launch
 * arrive at the grid barrier of the sweep kernels and then wait, with the kernels' own bounded
 * wait, for one arrival more than there are CTAs, which nothing makes.  The wait gives up after
 * 2^22 polls (a few seconds), records ISF_ERR_TIMEOUT and its site in a status word, and the
 * kernel returns: *status_out = that status (ISF_ERR_TIMEOUT), *where_out = the site (1: grid
 * barrier).  No fault, no trap; the context stays usable.  Synchronous.
 * Errors: ISF_ERR_ARG (ctas < 2 or more than can be co-resident), ISF_ERR_CUDA. */
int isf_debug_wait_timeout(int32_t ctas, int32_t* status_out, int32_t* where_out);

/* Device Philox4x32-10 blocks for checking the generator: for b in [0, nblocks), the block
 * with key (seed_lo, seed_hi) and counter (q0 + b, sweep_lo, sweep_hi, stream) goes to
 * host_out[4b .. 4b+3].  Synchronous. */
int isf_philox_blocks(uint64_t seed, uint32_t stream, uint64_t sweep, uint32_t q0,
                      int64_t nblocks, uint32_t* host_out);

/* Integer-issue ceilings of the current GPU, for the roofline of the sweep kernels (they do
 * no contraction, and with the film L2-resident they are bound by integer issue).  One
 * register-only launch of `ctas` CTAs (0 = SMs x the CTAs one SM holds) of `threads` threads
 * (a multiple of 32, 32..1024, 32..512 for ISF_PEAK_ATTEMPT; 0 = 256), `iters` iterations per
 * thread, asynchronous on cuda_stream (time it with events on that stream).  Nothing is read
 * from memory; one word is stored only if the final value equals a fixed word, so that no chain
 * is dead code.  *units_out = the work of the launch:
 *   ISF_PEAK_LOP3:    three-input logic operations, each reading three different chains (lane-ops);
 *   ISF_PEAK_MIX:     lane-ops of the random-number integer mix, one instruction each:
 *                     32x32 -> 64-bit multiply, three-input XOR, three-input majority, 32-bit add;
 *   ISF_PEAK_PHILOX:  Philox4x32-10 blocks (four interleaved per thread, the sweeps' own code),
 *                     the generator every Metropolis attempt of Eq. 8 draws its word from;
 *   ISF_PEAK_ATTEMPT: Metropolis attempts: the whole arithmetic of a bit-packed 32-site word with
 *                     every random word drawn (its 8 Philox blocks, the bit-sliced count of up
 *                     and vacant neighbours, the transpose to table offsets, the 32 table lookups
 *                     and comparisons, the flip mask and its dM, dB), inputs made from its own
 *                     random words, no loads of a film and no barrier between colour passes.
 * Errors: ISF_ERR_ARG (mode, threads, ctas or iters out of range), ISF_ERR_CUDA. */
enum { ISF_PEAK_LOP3 = 0, ISF_PEAK_MIX = 1, ISF_PEAK_PHILOX = 2, ISF_PEAK_ATTEMPT = 3 };
int isf_peak_probe(int32_t mode, int32_t ctas, int32_t threads, int64_t iters, void* cuda_stream,
                   double* units_out);

#ifdef __cplusplus
}
#endif
#endif
