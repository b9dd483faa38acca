/*
 * isf_oracle.h — plain, slow, single-threaded CPU oracle for Metropolis sweeps of the
 * ferromagnetic Ising model on the z = 12 film lattice built from a height map
 * (Kapitan & Nefedev, "High Performance Calculation of Magnetic Properties and Simulation
 * of Nonequilibrium Phenomena in nanofilms").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or calls this
 * code; only the test suite, the package's smoke check and the CPU baseline leg of the
 * benchmark do.  It shares no code with the CUDA path: lattice, stencil, colouring, Philox,
 * threshold table and sweep are written again here, from the definitions, in the order the
 * paper states them.
 *
 * Readings of the paper that the oracle fixes (the paper is silent on them):
 *   - geometry: FCC in primitive coordinates, constant-z planes are ABC-stacked triangular
 *     layers; the 12 neighbours are 6 in-plane, 3 up, 3 down (Sec. 2 and Sec. 3 only say
 *     "coordination number 12").
 *   - occupancy: site (x, y, z) is occupied iff z < H(x, y)  (Sec. 3: rows = image height,
 *     columns = image width, depth = number of Co layers).
 *   - "checkerboard" (Sec. 3, Fig. 1): four conflict-free colours
 *     c = ((x+z)&1) | (((y+z)&1)<<1), updated in the order 0, 1, 2, 3 every sweep.
 *   - random number in (0,1) of Eq. 8: r = (u + 0.5) 2^-32 with u a Philox4x32-10 word.
 *   - acceptance (Eq. 8, items 1-3 of Sec. 5): p = 1 when dE <= 0, else exp(-dE/T);
 *     accept iff p > r.  Encoded as a uint32 threshold (see or_threshold).
 */
#ifndef ISF_ORACLE_H
#define ISF_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define OR_ALWAYS 0xFFFFFFFFu

enum { OR_OK = 0, OR_ERR_ARG = -1, OR_ERR_OOM = -2, OR_ERR_COLOURING = -4,
       OR_ERR_SCHEDULE = -5, OR_ERR_STATE = -7 };
enum { OR_PERIODIC_X = 1, OR_PERIODIC_Y = 2, OR_PERIODIC_Z = 4 };
enum { OR_INIT_RANDOM = 0, OR_INIT_UP = 1, OR_INIT_DOWN = 2 };
enum { OR_STREAM_METROPOLIS = 0, OR_STREAM_GATE = 1, OR_STREAM_INIT = 2 };

typedef struct or_film or_film;

/* Per-step record: exact integer sums over the measured sweeps, FP64 values derived from them. */
typedef struct {
    double T, h;
    int64_t M_last, B_last, n_meas;
    int64_t sumM, sumAbsM;
    uint64_t sumM2[2], sumB2[2], sumMB[2];   /* 128-bit, little-endian words; sumMB two's complement */
    int64_t sumB;
    double m, abs_m, e, chi, chi_abs, C;
} or_step_obs;

/* Philox4x32-10 block function (Salmon et al., SC'11): 10 rounds on a 4x32 counter, 2x32 key. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Colour of a site, and the 32-bit random word a site draws at a given sweep from a stream. */
int or_colour(int x, int y, int z);
uint32_t or_site_word(const or_film* f, uint32_t stream, uint64_t sweep, int x, int y, int z);

/* Acceptance threshold for current spin s (+1/-1) with neighbour sum n at (T, h, J) (Eq. 8). */
uint32_t or_threshold(double T, double h, double J, int n, int s);

/* Threshold of the switching-field gate of Eq. 9 (pass probability exp(-|h_s| / T), |S_i| = 1),
 * in the same encoding; h_s = 0 gives "always" (the gate is off). */
uint32_t or_gate_threshold(double T, double h_s);

int  or_film_create(const uint8_t* heights, int rows, int cols, int layers, unsigned flags,
                    uint64_t seed, int init, or_film** out);
void or_film_destroy(or_film* f);
int  or_film_info(const or_film* f, int64_t* n_occ, int64_t* n_bonds, int64_t* M, int64_t* B,
                  int64_t* sweep);
int  or_neighbours(const or_film* f, int x, int y, int z, int* out_xyz /* 12*3 ints */);
int  or_check_colouring(const or_film* f);
int  or_get_spins(const or_film* f, int8_t* out /* [z][y][x] */);
int  or_set_spins(or_film* f, const int8_t* in /* [z][y][x], 0 exactly on vacancies */);
int  or_set_sweep(or_film* f, int64_t sweep);
int  or_recompute(const or_film* f, int64_t* M, int64_t* B);

/* Run whole schedule steps.  h_s = 0 disables the switching-field gate of Eq. 9.
 * series (optional, may be NULL): M and B after every sweep, 2 int64 per sweep. */
int  or_run(or_film* f, int nsteps, const double* T, const double* h, const int* sweeps_eq,
            const int* sweeps_meas, double J, double h_s, or_step_obs* rec, int64_t* series);

/* FP64 quantities of one record derived from its integer sums (n_occ sites, J). */
void or_derive(or_step_obs* r, int64_t n_occ, double J);

/* Curie-temperature estimate of a temperature scan (Sec. 4, Table 1): the T of the step with the
 * largest chi_abs among the steps with n_meas > 0 and a finite T > 0 (first of equal maxima).
 * Returns that step's index (and *T_c), or -1 when no step qualifies. */
int  or_estimate_tc(const or_step_obs* r, int n, double* T_c);

/* Simulated PMOKE image (Sec. 6): for every pixel the topmost occupied site z = H(x,y) - 1;
 * 255 (white) if its spin is up, 0 (black) if down, 128 where the pixel holds no atom.
 * out: rows*cols bytes, [y][x].  Returns the number of up surface pixels. */
int64_t or_surface_image(const or_film* f, uint8_t* out);

/* Exact Gibbs averages over all 2^N states of the occupied sites (Eqs. 4-5), N <= 24.
 * out: <M>, <|M|>, <M^2>, <E>, <E^2>, <B>. */
int  or_exact(const or_film* f, double T, double h, double J, double* out);

#ifdef __cplusplus
}
#endif
#endif
