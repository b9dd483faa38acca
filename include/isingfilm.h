/*
 * isingfilm.h — C ABI of the GB300 (sm_103a) Metropolis engine for Ising nanofilms.
 *
 * The method (Kapitan & Nefedev, "High Performance Calculation of Magnetic Properties and
 * Simulation of Nonequilibrium Phenomena in nanofilms"):
 *   - Sec. 2 and Sec. 3: a 3-D spin array of rows (image height) x columns (image width) x
 *     layers (number of Co layers), sites occupied where the height image reaches the layer,
 *     each spin with up to z = 12 nearest neighbours;
 *   - Eq. 3: H = -J sum_bonds S S' - h sum S, S = +-1, k = 1;
 *   - Eq. 8 and items 1-3 of Sec. 5: Metropolis single-spin flips, p = 1 if dE <= 0 else
 *     exp(-dE/T), accepted when p exceeds a uniform random number in (0,1);
 *   - Eq. 9 and items 4-5 of Sec. 5: optional switching-field gate with probability
 *     exp(-|h_s|/T), drawn before the Metropolis step;
 *   - Sec. 3, Fig. 1: "checkerboard" updates of one part of the spins while the rest is fixed;
 *     here four conflict-free colours c = ((x+z)&1) | (((y+z)&1)<<1), order 0,1,2,3;
 *   - Sec. 3 and Fig. 3/Fig. 5: temperature scans and field hysteresis loops, state carried
 *     from one temperature or field step to the next.
 *
 * Lattice (the paper fixes only z = 12): FCC in primitive coordinates; a site (x, y, z) has
 * the neighbours (+-1,0,0), (0,+-1,0), +-(1,-1,0) in its layer, (0,0,1), (0,-1,1), (-1,0,1)
 * above and (0,0,-1), (0,1,-1), (1,0,-1) below.  Site (x, y, z) is occupied iff
 * z < heights[y*cols + x].
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed, counter
 * (q, sweep_lo, sweep_hi, stream), q = ((c*layers + z)*ceil(rows/2) + (y>>1))*ceil(ceil(cols/2)/4)
 * + ((x>>1)>>2), word (x>>1)&3; stream 0 = Metropolis, 1 = switching gate, 2 = initial spins
 * (sweep 0).  A site flips iff thr == 0xFFFFFFFF or u < thr, thr = ceil(p*2^32 - 0.5)
 * clamped (the random number of Eq. 8 is r = (u + 0.5)*2^-32).  Trajectories are therefore a
 * pure function of (heights, layers, flags, seed, init, schedule): the same on every launch
 * configuration, spin layout and batch mix.
 *
 * Conventions.  Every function returns an isf_status (0 = ISF_OK) and, on failure, sets a
 * thread-local message readable with isf_last_error().  Host arrays passed in are copied;
 * the caller keeps them.  Device memory belongs to the library unless the *_in variant is
 * given a caller-owned buffer, which must then outlive the lattice.  isf_run_sweeps is
 * asynchronous on the given CUDA stream (a cudaStream_t, e.g. torch.cuda.Stream.cuda_stream;
 * NULL = legacy default stream); the read functions synchronise.  Kernels report problems
 * through a device status word; nothing traps.
 */
#ifndef ISINGFILM_H
#define ISINGFILM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct isf_lattice isf_lattice;

typedef enum {
    ISF_OK = 0,
    ISF_ERR_ARG = -1,        /* bad argument (size, pointer, value range) */
    ISF_ERR_OOM = -2,        /* device or host allocation failed, or caller buffer too small */
    ISF_ERR_CUDA = -3,       /* a CUDA runtime call failed (message has the CUDA error) */
    ISF_ERR_COLOURING = -4,  /* periodic extent odd or < 4: the 4-colouring would not be conflict-free */
    ISF_ERR_SCHEDULE = -5,   /* bad schedule, or running past its end */
    ISF_ERR_TIMEOUT = -6,    /* a bounded device wait expired; the kernel returned early */
    ISF_ERR_STATE = -7       /* call not valid in the current state (e.g. no schedule set) */
} isf_status;

enum {
    ISF_PERIODIC_X = 1,      /* wrap x (columns); needs cols even and >= 4 */
    ISF_PERIODIC_Y = 2,      /* wrap y (rows);    needs rows even and >= 4 */
    ISF_PERIODIC_Z = 4,      /* wrap z (layers);  needs layers even and >= 4 (bulk tests) */
    ISF_PACKED = 8           /* one bit per spin (32 spins per uint32) + occupancy bit-plane;
                                open boundaries only */
};

enum { ISF_INIT_RANDOM = 0, ISF_INIT_UP = 1, ISF_INIT_DOWN = 2 };

/* Per-step record.  The integer fields are exact sums over the step's measured sweeps (the
 * last sweeps_meas sweeps of the step), taken after each sweep; the doubles are derived from
 * them on the host (N = number of occupied sites, E = -J*B - h*M per Eq. 3):
 *   m = <M>/N, abs_m = <|M|>/N, e = <E>/N, chi = (<M^2> - <M>^2)/(N T),
 *   chi_abs = (<M^2> - <|M|>^2)/(N T), C = (<E^2> - <E>^2)/(N T^2).
 * B is the bond sum sum_bonds S S' (each bond once).  128-bit sums are two little-endian
 * uint64 words; sumMB is two's complement.  Derived values are NaN when n_meas = 0. */
typedef struct {
    double T, h;
    int64_t M_last, B_last, n_meas;
    int64_t sumM, sumAbsM;
    uint64_t sumM2[2], sumB2[2], sumMB[2];
    int64_t sumB;
    double m, abs_m, e, chi, chi_abs, C;
} isf_step_obs;

/* Device bytes a lattice of this shape needs (spins, heights, state; packed films also their
 * occupied-word lists with a 24-byte record per entry and the row-slab kernel's scratch).  0 if
 * invalid. */
size_t isf_lattice_bytes(int32_t rows, int32_t cols, int32_t layers, uint32_t flags);

/* Build a film on the current CUDA device from a host height map.
 *   heights: host, rows*cols bytes, row-major [y][x], each value in 0..layers (Sec. 3).
 *   flags:   ISF_PERIODIC_* | ISF_PACKED.   seed: Philox key.   init: ISF_INIT_*.
 *   cuda_stream: stream for the set-up kernels (the call returns once they are done).
 * Errors: ISF_ERR_ARG (sizes, heights > layers, packed with periodic axes, null pointers),
 * ISF_ERR_COLOURING, ISF_ERR_OOM, ISF_ERR_CUDA. */
int isf_lattice_create(const uint8_t* heights, int32_t rows, int32_t cols, int32_t layers,
                       uint32_t flags, uint64_t seed, int32_t init, void* cuda_stream,
                       isf_lattice** out);

/* As isf_lattice_create, but the film lives in a caller-owned device buffer of dev_bytes
 * (>= isf_lattice_bytes, 256-byte aligned), e.g. a torch tensor.  ISF_ERR_OOM if too small. */
int isf_lattice_create_in(const uint8_t* heights, int32_t rows, int32_t cols, int32_t layers,
                          uint32_t flags, uint64_t seed, int32_t init, void* cuda_stream,
                          void* dev_buf, size_t dev_bytes, isf_lattice** out);

/* Set the temperature / field schedule (Sec. 3: one "step of temperature or field" after
 * another).  Step k: temperature T[k] >= 0 (T = +inf allowed), field h[k] (finite),
 * sweeps_eq[k] discarded then sweeps_meas[k] measured sweeps, eq + meas >= 1.  J: exchange
 * (Eq. 3).  h_s: switching field of Eq. 9 (0 disables the gate).  Host arrays of nsteps
 * entries, copied.  Resets the schedule cursor and records; the spins and the sweep counter
 * carry on.  The threshold tables are built here on the host in fp64 (std::exp).
 * Errors: ISF_ERR_ARG, ISF_ERR_SCHEDULE, ISF_ERR_OOM, ISF_ERR_CUDA. */
int isf_set_schedule(isf_lattice* lat, int32_t nsteps, const double* T, const double* h,
                     const int32_t* sweeps_eq, const int32_t* sweeps_meas, double J, double h_s);

/* Enqueue nsweeps Metropolis sweeps (each: colours 0..3, every occupied site once) on
 * cuda_stream; nsweeps = -1 runs to the end of the schedule.  Asynchronous.
 * Errors: ISF_ERR_STATE (no schedule), ISF_ERR_SCHEDULE (past the end), ISF_ERR_CUDA,
 * ISF_ERR_TIMEOUT (reported by a previous launch's status word). */
int isf_run_sweeps(isf_lattice* lat, int64_t nsweeps, void* cuda_stream);

/* Copy the records of the completed schedule steps (at most max) to out; *n_out = count.
 * Synchronises with the lattice's last stream.  Errors: ISF_ERR_ARG, ISF_ERR_CUDA,
 * ISF_ERR_TIMEOUT. */
int isf_read_observables(isf_lattice* lat, isf_step_obs* out, int32_t max, int32_t* n_out);

/* Spins to host_out (layers*rows*cols int8, [z][y][x], +1 / -1, 0 on vacancies).  Syncs. */
int isf_read_spins(isf_lattice* lat, int8_t* host_out);

/* Simulated PMOKE image of the film (Sec. 6): only the surface atoms are shown, white for spin
 * up and black for spin down.  host_out: rows*cols bytes [y][x]; 255 where the pixel's top atom
 * (z = height - 1) is up, 0 where it is down, 128 where the pixel has no atom.  *n_up (may be
 * NULL): white pixels.  Synchronises. */
int isf_read_surface_image(isf_lattice* lat, uint8_t* host_out, int64_t* n_up);

/* Domains of the simulated PMOKE image (Sec. 6, Fig. 5): out4 = {white domains, black
 * domains, pixels of the largest white domain, of the largest black one}.  Two pixels touch when
 * their columns are in-plane neighbours of the film ((x +- 1, y), (x, y +- 1), (x + 1, y - 1),
 * (x - 1, y + 1), wrapping on periodic axes); a domain is a connected set of pixels of one colour;
 * pixels with no atom belong to none.  Synchronises.  Errors: ISF_ERR_ARG, ISF_ERR_CUDA,
 * ISF_ERR_TIMEOUT (a bounded retry of the device union-find ran out). */
int isf_surface_domains(isf_lattice* lat, int64_t* out4);

/* Lattice statistics of Sec. 4 / Table 1: concentration p = occupied sites / (rows*cols*layers),
 * mean coordination zbar = 2 * occupied bonds / occupied sites and the critical concentration
 * p_c = 2 / zbar of Eq. 2 (inf when there are no bonds).  No device work. */
int isf_lattice_stats(isf_lattice* lat, double* p, double* zbar, double* p_c);

/* Curie-temperature estimate of a temperature scan (Sec. 4, Table 1; Fig. 3): a finite film has
 * no sharp transition, so T_c is read as the temperature of the largest susceptibility
 * chi' = (<M^2> - <|M|>^2) / (N T) among the scan's steps.  recs: n step records as
 * isf_read_observables returns them (host); chi' is formed from their exact integer sums, and
 * only steps with n_meas > 0 and a finite T > 0 take part; the first of equal maxima wins.
 * *T_c = that step's T, *index (may be NULL) = its position.  Host only, no device work.
 * Errors: ISF_ERR_ARG (NULL pointers, n < 1), ISF_ERR_STATE (no step takes part). */
int isf_estimate_tc(const isf_step_obs* recs, int32_t n, double* T_c, int32_t* index);

/* Replace the spins (same layout; must be +-1 exactly on occupied sites, 0 elsewhere) and
 * set the film-local sweep counter (the next sweep draws sweep + 1), e.g. to resume from a
 * state.  Recomputes M and B.  Synchronous.  Errors: ISF_ERR_ARG, ISF_ERR_CUDA. */
int isf_write_spins(isf_lattice* lat, const int8_t* host_in, int64_t sweep);

/* Occupied sites, occupied bonds, mean coordination zbar = 2*bonds/sites (Sec. 4, Table 1),
 * sweeps done.  Any pointer may be NULL.  No device work. */
int isf_lattice_info(isf_lattice* lat, int64_t* n_occ, int64_t* n_bonds, double* zbar,
                     int64_t* sweep);

/* Current magnetisation sum M and bond sum B from the incremental bookkeeping (synchronises),
 * and, if recompute != 0, recomputed from the spins on the device for comparison. */
int isf_read_state(isf_lattice* lat, int64_t* M, int64_t* B, int32_t recompute,
                   int64_t* M_full, int64_t* B_full);

/* Keep M and B after every sweep for the next max_sweeps sweeps (0 = off); read them with
 * isf_read_trace as (M, B) int64 pairs in sweep order. */
int isf_enable_trace(isf_lattice* lat, int64_t max_sweeps);
int isf_read_trace(isf_lattice* lat, int64_t* host_out, int64_t max_pairs, int64_t* n_out);

/* Save the film (shape, flags, seed, spins, sweep counter) to a file; load it back onto the
 * current device (schedule not saved).  Errors: ISF_ERR_ARG, ISF_ERR_CUDA, ISF_ERR_OOM. */
int isf_save(isf_lattice* lat, const char* path);
int isf_load(const char* path, void* cuda_stream, isf_lattice** out);

void isf_lattice_destroy(isf_lattice* lat);

/* Message of the last failure on this thread ("" if none); valid until the next call. */
const char* isf_last_error(void);

/* ---- Row slabs of one film (several GPUs) ---------------------------------------------------
 * Sec. 3 splits the film by rows between processes, each updating its own rows and exchanging
 * the boundary rows with its neighbours.  A slab film holds whole-film rows [y0, y1) (y0 even,
 * y1 even or the last row, at least two rows) plus one halo row pair on each side (wrapping
 * when the film is periodic in y; none at an open edge).  Its sites carry the whole film's
 * Philox counters, so with halos refreshed after every colour pass the slabs together follow
 * the whole film's trajectory exactly.  It starts from the seed (random, up or down) with its
 * halo rows already equal to the neighbours' rows.  A slab advances one colour pass at a time
 * with isf_run_pass; isf_run_sweeps, batches, isf_write_spins and isf_save refuse it
 * (ISF_ERR_STATE).  Its trace (isf_enable_trace / isf_read_trace) records its own rows' change
 * of M and B since creation after each sweep; the whole film's M and B per sweep are the sums
 * over slabs plus the sums of the slabs' creation shares (isf_slab_info), and isf_fold_series
 * turns that series into step records.  The heights argument is the whole film's map. */
int isf_lattice_create_slab(const uint8_t* heights, int32_t rows, int32_t cols, int32_t layers, uint32_t flags,
                            uint64_t seed, int32_t init, int32_t y0, int32_t y1, void* cuda_stream,
                            isf_lattice** out);
/* out6 = {y0, y1, ya (whole-film row of local row 0; may be negative or past the end when it
 * wraps), local rows, first own colour-row, end of own colour-rows}; *halo_bytes = bytes of one
 * colour-row over all layers (the size of an export / import buffer); out3 = {own share of M,
 * own share of 2B (over own sites, halo neighbours included), own occupied sites} at creation. */
int isf_slab_info(isf_lattice* lat, int32_t* out6, size_t* halo_bytes, int64_t* out3);
/* After colour pass `colour`, copy the slab's own boundary colour-row of that colour (all layers)
 * next to side 0 (low y) or 1 (high y) into dev_buf, or copy dev_buf into the halo row on that
 * side.  Device buffers of isf_slab_info's halo_bytes; asynchronous on cuda_stream.
 * Errors: ISF_ERR_ARG (no halo on that side of an open film's edge slab). */
int isf_slab_export(isf_lattice* lat, int32_t colour, int32_t side, void* dev_buf, void* cuda_stream);
int isf_slab_import(isf_lattice* lat, int32_t colour, int32_t side, const void* dev_buf, void* cuda_stream);
/* One colour pass (colours 0, 1, 2, 3 in turn) of the next sweep of the schedule on the slab's
 * own rows; after colour 3 the sweep is complete.  Asynchronous.  Errors: ISF_ERR_STATE (not a
 * slab, no schedule, out of order), ISF_ERR_SCHEDULE (schedule done). */
int isf_run_pass(isf_lattice* lat, int32_t colour, void* cuda_stream);
/* Host only: step records (as isf_read_observables) of a per-sweep series M[t], B[t] of a whole
 * film under a schedule, with n_occ occupied sites (Eq. 3 sums and the Fig. 3 estimators). */
int isf_fold_series(int32_t nsteps, const double* T, const double* h, const int32_t* sweeps_eq,
                    const int32_t* sweeps_meas, double J, int64_t n_occ, const int64_t* M, const int64_t* B,
                    isf_step_obs* out);

/* ---- Batched films -------------------------------------------------------------------------
 * Many independent films (each its own height map, seed and temperature / field schedule: the
 * paper's scans and loops, Sec. 3, Fig. 3, Fig. 5, for many samples at once) advanced together.
 * A batch references lattices created with isf_lattice_create (it does not own them); each needs
 * a schedule.  isf_batch_run advances every member to the end of its schedule: int8 films that
 * fit one CTA's shared memory are taken from a device queue by a persistent single-CTA kernel,
 * films that need a cluster by a persistent cluster kernel (cluster size K), and the other films
 * (bit-packed, periodic-column, or too large for a cluster) by persistent kernels that run each
 * with its state in device memory on one CTA (up to 2^20 lattice sites, and at most an even share
 * of the whole batch's work per such CTA, so that no film finishes last on its own CTA) or one
 * cluster of 8 CTAs (up to 2^24), all concurrently on forked streams (when only the two
 * global-memory classes have films, the SMs are shared between them in proportion to their work,
 * so that both are resident from the start; a global-memory kernel whose own films are done
 * takes the resident films of its size class that have not started, and runs them in global
 * memory); larger films run after them on the multi-CTA global path.  Each film's
 * trajectory is the one it has alone.  Asynchronous on cuda_stream; read each film with
 * isf_read_observables / isf_read_spins afterwards. */
typedef struct isf_batch isf_batch;
int isf_batch_create(isf_batch** out);
int isf_batch_add(isf_batch* batch, isf_lattice* lat);        /* ISF_ERR_STATE: no schedule */
int isf_batch_clear(isf_batch* batch);
/* Launch shapes: threads of the single-CTA kernel, cluster size K (1..16) and threads of the
 * cluster kernel (multiples of 32 in 64..512, one warp folding); 0 = tuned or default (256; 16
 * and 512). */
int isf_batch_set_launch(isf_batch* batch, int32_t threads_single, int32_t cluster_K, int32_t threads_cluster);
/* on != 0: capture each persistent queue launch in its own single-kernel CUDA graph once and
 * replay them on later runs with the same shapes (the per-film arguments are uploaded each run).
 * With or without graphs the queue kernels are launched in one fixed order, so the way they
 * share the SMs does not change from run to run.  With graphs on, a run must not itself be
 * captured into a caller's graph (its capture would nest). */
int isf_batch_set_graph(isf_batch* batch, int32_t on);
/* Autotuner: times short probe runs (copies, not the members) over threads {128, 256, 384, 512}:
 * of the largest single-CTA film, keeping the fastest threads; and, for cluster sizes {8, 16},
 * of the largest cluster film that fits that size, keeping the (size, threads) with the least
 * probe time x rounds of the queue (the films that fit, over the co-resident clusters; films
 * that fit only 16 CTAs then run on the global-memory cluster kernel).  Probe times are cached
 * per (device, cluster size, threads, layers, row and column size class) for the process. */
int isf_batch_tune(isf_batch* batch, void* cuda_stream);
int isf_batch_run(isf_batch* batch, void* cuda_stream);
/* As isf_batch_run, but every member advances at most max_sweeps sweeps (>= 1; -1 = to the end). */
int isf_batch_run_sweeps(isf_batch* batch, int64_t max_sweeps, void* cuda_stream);
/* Last run (12 int32): films in the single-CTA / cluster / multi-CTA global classes, CTAs and
 * clusters launched, cluster size, threads of the two resident kernels; then films in the
 * one-CTA global-memory class (bit-packed, periodic-column or over-sized int8 films of at most
 * 2^20 lattice sites and an even share of the work) and CTAs launched for it; then films in the one-cluster (8 CTAs)
 * global-memory class (the same kinds, up to 2^24 sites) and clusters launched for it. */
int isf_batch_info(isf_batch* batch, int32_t* out12);
void isf_batch_destroy(isf_batch* batch);

/* ---- Serving ---------------------------------------------------------------------------------
 * Continuous batching of jobs (a hysteresis loop or a temperature scan on one film, Sec. 3,
 * Fig. 3, Fig. 5).  A worker thread on the device current at isf_server_create admits queued
 * jobs while their films fit device_budget_bytes (each admitted job holds its film until it
 * finishes), advances all admitted films by at most sweeps_per_tick sweeps per batched launch,
 * retires finished ones and admits more; jobs submitted while a tick runs join the next one.  A
 * job's result equals the result of the same job run alone.  The job's arrays are copied at
 * submit.  A job whose film alone exceeds the budget fails with ISF_ERR_OOM. */
enum { ISF_JOB_QUEUED = 0, ISF_JOB_RUNNING = 1, ISF_JOB_DONE = 2, ISF_JOB_FAILED = 3 };
typedef struct {
    const uint8_t* heights;                 /* host, rows*cols, as isf_lattice_create */
    int32_t rows, cols, layers;
    uint32_t flags;
    uint64_t seed;
    int32_t init;
    int32_t nsteps;                         /* schedule, as isf_set_schedule */
    const double* T;
    const double* h;
    const int32_t* sweeps_eq;
    const int32_t* sweeps_meas;
    double J, h_s;
} isf_job;
typedef struct isf_server isf_server;
int isf_server_create(size_t device_budget_bytes, int64_t sweeps_per_tick, isf_server** out);
int isf_server_submit(isf_server* srv, const isf_job* job, int64_t* id);
/* Wait up to timeout_s seconds for the job to finish; *state = ISF_JOB_*. */
int isf_server_wait(isf_server* srv, int64_t id, double timeout_s, int32_t* state);
/* State; when done, its records (as isf_read_observables, at most max) and the latency from
 * submit to completion.  A failed job returns its error. */
int isf_server_poll(isf_server* srv, int64_t id, int32_t* state, isf_step_obs* out, int32_t max,
                    int32_t* n_out, double* latency_s);
/* The batched launches ("ticks", numbered from 0 in the order the worker runs them) a job was
 * advanced in: out3 = {first tick, last tick, number of ticks}; {-1, -1, 0} before its first.
 * Two jobs whose tick ranges intersect had their films advanced by the same launches, i.e. on
 * the device at the same time. */
int isf_server_job_ticks(isf_server* srv, int64_t id, int64_t* out3);
/* Forget a finished job (frees its records). */
int isf_server_release(isf_server* srv, int64_t id);
/* out8: submitted, completed, failed, active, queued, ticks, attempts completed, peak budget
 * bytes in use; out4: seconds of batched launches, seconds since create, bytes in use, budget. */
int isf_server_stats(isf_server* srv, int64_t* out8, double* out4);
/* Finishes the jobs already submitted, then stops the worker and frees everything. */
void isf_server_destroy(isf_server* srv);

/* No-allocation run (no counterpart in the paper; it exists for callers of this library).
 * Some callers must not allocate device memory: code living inside a process whose device
 * memory is owned by another allocator's pool (a foreign cudaMalloc then fails, or fragments the
 * pool), latency-bound loops in which cudaMalloc/cudaFree would synchronise the device and stall
 * other streams, and deployments that forbid allocation after start-up.  isf_run_noalloc runs a
 * whole schedule on one film and allocates nothing: the film, its state, the threshold tables and
 * the step records live in one fixed library-owned device array of ISF_NOALLOC_MAX_BYTES, which
 * every GPU that loads the library keeps until the process exits.
 *   Inputs as isf_lattice_create + isf_set_schedule (host arrays; the film starts at sweep 0).
 *   dev_spins_out: caller-owned device buffer of layers*rows*cols int8, [z][y][x], final spins.
 *   obs_out: caller-owned host array of nsteps records, as isf_read_observables fills them.
 * Results equal those of the allocating path.  The call blocks until its work is done: it
 * synchronises cuda_stream several times and stages the tables and records through host stack
 * buffers, so no call (the first or any later one) may be made while a stream is being captured.
 * Its first call on a device looks up the array's device address (cudaGetSymbolAddress) and keeps
 * it for the process; do not use the library across a cudaDeviceReset (the kept address would be
 * stale).  Every call reuses the same array and clears what must start at zero; calls whose work
 * overlaps on the GPU (other streams, other host threads) race on the array and must not be made.  A film and schedule needing more scratch than the array holds is
 * refused with ISF_ERR_ARG before any device work; other errors as isf_lattice_create,
 * isf_set_schedule and isf_run_sweeps. */
#define ISF_NOALLOC_MAX_BYTES (8u << 20)
int isf_run_noalloc(const uint8_t* heights, int32_t rows, int32_t cols, int32_t layers, uint32_t flags,
                    uint64_t seed, int32_t init, int32_t nsteps, const double* T, const double* h,
                    const int32_t* sweeps_eq, const int32_t* sweeps_meas, double J, double h_s,
                    int8_t* dev_spins_out, isf_step_obs* obs_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
