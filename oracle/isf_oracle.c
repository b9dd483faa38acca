/*
 * isf_oracle.c — the CPU oracle.  TEST INFRASTRUCTURE ONLY (see isf_oracle.h): only the
 * tests, the smoke check and the benchmark's CPU-baseline leg load it.
 *
 * Everything here is written the plain way: one site at a time, the neighbour list built
 * from the stencil definition, fp64 host libm for exp(), 128-bit integer sums.  No blocking,
 * no bit tricks, no vectorisation.  The Markov chain it computes is fixed by
 *   - Eq. 3 (Hamiltonian H = -J sum_bonds S_n S_n' - h sum_n S_n),
 *   - Eq. 8 and items 1-3 of Sec. 5 (Metropolis acceptance),
 *   - Eq. 9 and items 4-5 of Sec. 5 (switching-field gate, applied first; h_s = 0 disables it),
 *   - Sec. 3 and Fig. 1 ("checkerboard": sites of one colour are updated together),
 * plus the readings listed in isf_oracle.h.
 */
#include "isf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

struct or_film {
    int R, C, L;            /* rows (y), columns (x), layers (z) */
    unsigned flags;
    uint64_t seed;
    int Rh, Ch, Qw;         /* ceil(R/2), ceil(C/2), ceil(Ch/4): RNG counter layout */
    uint8_t* occ;           /* [z][y][x], 1 = occupied */
    int8_t* spin;           /* [z][y][x], +1 / -1, 0 on vacancies */
    int64_t n_occ, n_bonds;
    int64_t M, B;           /* magnetisation sum S and bond sum sum_bonds S S' */
    int64_t sweep;          /* number of Metropolis sweeps done so far */
};

/* ---------------------------------------------------------------- Philox4x32-10 -------- */
/* Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
 * one round maps (c0,c1,c2,c3) with multipliers M0, M1 to
 *   (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0)),
 * and the key is bumped by the Weyl constants between rounds; 10 rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ---------------------------------------------------------------- lattice ------------ */
/* Colour of a site: the four sublattices of the "checkerboard decomposition" (Sec. 3). */
int or_colour(int x, int y, int z)
{
    return ((x + z) & 1) | (((y + z) & 1) << 1);
}

/* The 12 nearest-neighbour offsets (dx, dy, dz) of FCC in primitive coordinates
 * (z = 12, Sec. 2 and item 2 of Sec. 3): 6 in the same triangular layer, 3 in the layer
 * above, 3 in the layer below. */
static const int STENCIL[12][3] = {
    { 1, 0, 0}, {-1, 0, 0}, { 0, 1, 0}, { 0,-1, 0}, { 1,-1, 0}, {-1, 1, 0},
    { 0, 0, 1}, { 0,-1, 1}, {-1, 0, 1},
    { 0, 0,-1}, { 0, 1,-1}, { 1, 0,-1},
};

static size_t site_of(const or_film* f, int x, int y, int z)
{
    return ((size_t)z * (size_t)f->R + (size_t)y) * (size_t)f->C + (size_t)x;
}

/* Coordinates of neighbour k of (x,y,z), or 0 if it falls outside an open boundary. */
static int neighbour(const or_film* f, int x, int y, int z, int k, int* nx, int* ny, int* nz)
{
    int a = x + STENCIL[k][0], b = y + STENCIL[k][1], c = z + STENCIL[k][2];
    if (a < 0 || a >= f->C) {
        if (!(f->flags & OR_PERIODIC_X)) return 0;
        a = (a + f->C) % f->C;
    }
    if (b < 0 || b >= f->R) {
        if (!(f->flags & OR_PERIODIC_Y)) return 0;
        b = (b + f->R) % f->R;
    }
    if (c < 0 || c >= f->L) {
        if (!(f->flags & OR_PERIODIC_Z)) return 0;
        c = (c + f->L) % f->L;
    }
    *nx = a; *ny = b; *nz = c;
    return 1;
}

int or_neighbours(const or_film* f, int x, int y, int z, int* out_xyz)
{
    if (!f || x < 0 || y < 0 || z < 0 || x >= f->C || y >= f->R || z >= f->L) return OR_ERR_ARG;
    int n = 0;
    for (int k = 0; k < 12; ++k) {
        int a, b, c;
        if (neighbour(f, x, y, z, k, &a, &b, &c)) {
            out_xyz[3 * n + 0] = a; out_xyz[3 * n + 1] = b; out_xyz[3 * n + 2] = c;
            ++n;
        }
    }
    return n;
}

/* Sum of the spins of the occupied neighbours (vacancies hold spin 0). */
static int neighbour_sum(const or_film* f, int x, int y, int z)
{
    int n = 0;
    for (int k = 0; k < 12; ++k) {
        int a, b, c;
        if (neighbour(f, x, y, z, k, &a, &b, &c)) n += f->spin[site_of(f, a, b, c)];
    }
    return n;
}

/* No occupied bond may join two sites of the same colour, across periodic wraps included:
 * only then do the sites of one colour not interact, so updating them in any order (or all
 * at once) is the same Markov chain. */
int or_check_colouring(const or_film* f)
{
    for (int z = 0; z < f->L; ++z)
        for (int y = 0; y < f->R; ++y)
            for (int x = 0; x < f->C; ++x) {
                if (!f->occ[site_of(f, x, y, z)]) continue;
                for (int k = 0; k < 12; ++k) {
                    int a, b, c;
                    if (!neighbour(f, x, y, z, k, &a, &b, &c)) continue;
                    if (!f->occ[site_of(f, a, b, c)]) continue;
                    if (or_colour(a, b, c) == or_colour(x, y, z)) return OR_ERR_COLOURING;
                }
            }
    return OR_OK;
}

/* ---------------------------------------------------------------- random words ------- */
/* The 32-bit word a site draws: Philox4x32-10 keyed by the seed, counter
 * (q, sweep_lo, sweep_hi, stream) with q = ((c*L + z)*Rh + (y>>1))*Qw + ((x>>1)>>2);
 * word (x>>1) & 3 of the block. */
uint32_t or_site_word(const or_film* f, uint32_t stream, uint64_t sweep, int x, int y, int z)
{
    int c = or_colour(x, y, z);
    int i = x >> 1, j = y >> 1;
    uint64_t q = (((uint64_t)c * (uint64_t)f->L + (uint64_t)z) * (uint64_t)f->Rh + (uint64_t)j)
                 * (uint64_t)f->Qw + (uint64_t)(i >> 2);
    uint32_t ctr[4] = { (uint32_t)q, (uint32_t)sweep, (uint32_t)(sweep >> 32), stream };
    uint32_t key[2] = { (uint32_t)f->seed, (uint32_t)(f->seed >> 32) };
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return out[i & 3];
}

/* ---------------------------------------------------------------- acceptance --------- */
/* Eq. 8: a flip of spin s with neighbour sum n changes the energy of Eq. 3 by
 * dE = E2 - E1 = 2 s (J n + h).  It is accepted with probability p = 1 if dE <= 0 and
 * p = exp(-dE/T) otherwise, "if p is greater than" a random number r in (0,1).
 * With r = (u + 0.5) 2^-32, u uniform on [0, 2^32), the accepted u are exactly
 * u < thr, thr = #{u : (u + 0.5) 2^-32 < p} = ceil(p 2^32 - 0.5) (0 when that is <= 0).
 * OR_ALWAYS marks "accept every u": dE <= 0, or a count of 2^32 - 1 or more (the clamp
 * moves the acceptance probability by at most 2^-32). */
static uint32_t threshold_of_probability(double p)
{
    double X = p * 4294967296.0 - 0.5;   /* exact: power-of-two scaling, then a half-ulp-exact subtraction */
    if (!(X > 0.0)) return 0;
    double count = ceil(X);
    if (count >= 4294967295.0) return OR_ALWAYS;
    return (uint32_t)count;
}

uint32_t or_threshold(double T, double h, double J, int n, int s)
{
    double dE = 2.0 * (double)s * (J * (double)n + h);
    if (dE <= 0.0) return OR_ALWAYS;
    double p = exp(-dE / T);
    return threshold_of_probability(p);
}

/* Eq. 9: the switching-field gate passes with probability exp(-|S_i h_s| / T); |S_i| = 1.
 * Same encoding as the Eq. 8 threshold: the gate word g passes iff g < the count (or always). */
uint32_t or_gate_threshold(double T, double h_s)
{
    double a = fabs(h_s);
    if (a == 0.0) return OR_ALWAYS;
    return threshold_of_probability(exp(-a / T));
}

/* ---------------------------------------------------------------- film --------------- */
int or_recompute(const or_film* f, int64_t* M, int64_t* B)
{
    int64_t m = 0, twob = 0;
    for (int z = 0; z < f->L; ++z)
        for (int y = 0; y < f->R; ++y)
            for (int x = 0; x < f->C; ++x) {
                int s = f->spin[site_of(f, x, y, z)];
                if (!s) continue;
                m += s;
                twob += (int64_t)s * neighbour_sum(f, x, y, z);   /* each bond seen twice */
            }
    *M = m;
    *B = twob / 2;
    return OR_OK;
}

int or_film_create(const uint8_t* heights, int rows, int cols, int layers, unsigned flags,
                   uint64_t seed, int init, or_film** out)
{
    if (!out) return OR_ERR_ARG;
    *out = NULL;
    if (!heights || rows < 1 || cols < 1 || layers < 1) return OR_ERR_ARG;
    if (flags & ~(unsigned)(OR_PERIODIC_X | OR_PERIODIC_Y | OR_PERIODIC_Z)) return OR_ERR_ARG;
    if (init < OR_INIT_RANDOM || init > OR_INIT_DOWN) return OR_ERR_ARG;
    for (size_t p = 0; p < (size_t)rows * (size_t)cols; ++p)
        if (heights[p] > layers) return OR_ERR_ARG;
    /* A periodic axis keeps the colouring only with an even extent, and needs at least 4 so
     * that the +1 and -1 neighbours along it are different sites. */
    if ((flags & OR_PERIODIC_X) && (cols % 2 || cols < 4)) return OR_ERR_COLOURING;
    if ((flags & OR_PERIODIC_Y) && (rows % 2 || rows < 4)) return OR_ERR_COLOURING;
    if ((flags & OR_PERIODIC_Z) && (layers % 2 || layers < 4)) return OR_ERR_COLOURING;

    or_film* f = (or_film*)calloc(1, sizeof(or_film));
    if (!f) return OR_ERR_OOM;
    f->R = rows; f->C = cols; f->L = layers; f->flags = flags; f->seed = seed;
    f->Rh = (rows + 1) / 2; f->Ch = (cols + 1) / 2; f->Qw = (f->Ch + 3) / 4;
    size_t n = (size_t)rows * (size_t)cols * (size_t)layers;
    f->occ = (uint8_t*)calloc(n, 1);
    f->spin = (int8_t*)calloc(n, 1);
    if (!f->occ || !f->spin) { or_film_destroy(f); return OR_ERR_OOM; }

    for (int z = 0; z < layers; ++z)
        for (int y = 0; y < rows; ++y)
            for (int x = 0; x < cols; ++x) {
                int occupied = z < heights[(size_t)y * (size_t)cols + (size_t)x];
                size_t p = site_of(f, x, y, z);
                f->occ[p] = (uint8_t)occupied;
                if (!occupied) { f->spin[p] = 0; continue; }
                f->n_occ += 1;
                if (init == OR_INIT_UP) f->spin[p] = 1;
                else if (init == OR_INIT_DOWN) f->spin[p] = -1;
                else {
                    uint32_t u = or_site_word(f, OR_STREAM_INIT, 0, x, y, z);
                    f->spin[p] = (u >> 31) ? -1 : 1;
                }
            }
    int64_t half_bonds = 0;
    for (int z = 0; z < layers; ++z)
        for (int y = 0; y < rows; ++y)
            for (int x = 0; x < cols; ++x) {
                if (!f->occ[site_of(f, x, y, z)]) continue;
                for (int k = 0; k < 12; ++k) {
                    int a, b, c;
                    if (neighbour(f, x, y, z, k, &a, &b, &c) && f->occ[site_of(f, a, b, c)])
                        half_bonds += 1;
                }
            }
    f->n_bonds = half_bonds / 2;
    if (or_check_colouring(f) != OR_OK) { or_film_destroy(f); return OR_ERR_COLOURING; }
    or_recompute(f, &f->M, &f->B);
    *out = f;
    return OR_OK;
}

void or_film_destroy(or_film* f)
{
    if (!f) return;
    free(f->occ);
    free(f->spin);
    free(f);
}

int or_film_info(const or_film* f, int64_t* n_occ, int64_t* n_bonds, int64_t* M, int64_t* B,
                 int64_t* sweep)
{
    if (!f) return OR_ERR_ARG;
    if (n_occ) *n_occ = f->n_occ;
    if (n_bonds) *n_bonds = f->n_bonds;
    if (M) *M = f->M;
    if (B) *B = f->B;
    if (sweep) *sweep = f->sweep;
    return OR_OK;
}

int or_get_spins(const or_film* f, int8_t* out)
{
    if (!f || !out) return OR_ERR_ARG;
    memcpy(out, f->spin, (size_t)f->R * (size_t)f->C * (size_t)f->L);
    return OR_OK;
}

int or_set_spins(or_film* f, const int8_t* in)
{
    if (!f || !in) return OR_ERR_ARG;
    size_t n = (size_t)f->R * (size_t)f->C * (size_t)f->L;
    for (size_t p = 0; p < n; ++p) {
        if (f->occ[p] ? (in[p] != 1 && in[p] != -1) : (in[p] != 0)) return OR_ERR_ARG;
    }
    memcpy(f->spin, in, n);
    or_recompute(f, &f->M, &f->B);
    return OR_OK;
}

int or_set_sweep(or_film* f, int64_t sweep)
{
    if (!f || sweep < 0) return OR_ERR_ARG;
    f->sweep = sweep;
    return OR_OK;
}

/* ---------------------------------------------------------------- statistics --------- */
static void put128(uint64_t w[2], i128 v)
{
    u128 u = (u128)v;
    w[0] = (uint64_t)u;
    w[1] = (uint64_t)(u >> 64);
}

static i128 get128(const uint64_t w[2])
{
    u128 u = ((u128)w[1] << 64) | (u128)w[0];
    return (i128)u;
}

/* Fluctuation estimators from exact integer sums over n measured sweeps:
 * m = <M>/N, |m| = <|M|>/N, e = <E>/N with E = -J B - h M (Eq. 3),
 * chi = (<M^2> - <M>^2)/(N T), chi' = (<M^2> - <|M|>^2)/(N T),
 * C = (<E^2> - <E>^2)/(N T^2) with Var E = J^2 Var B + h^2 Var M + 2 J h Cov(M, B).
 * Each variance numerator n*sum(x^2) - sum(x)^2 is formed exactly in 128-bit integers. */
void or_derive(or_step_obs* r, int64_t n_occ, double J)
{
    double nan = NAN;
    if (r->n_meas <= 0 || n_occ <= 0) {
        r->m = r->abs_m = r->e = r->chi = r->chi_abs = r->C = nan;
        return;
    }
    i128 n = r->n_meas;
    double nn = (double)r->n_meas;
    double N = (double)n_occ;
    double T = r->T, h = r->h;
    i128 sM = r->sumM, sA = r->sumAbsM, sB = r->sumB;
    i128 sM2 = get128(r->sumM2), sB2 = get128(r->sumB2), sMB = get128(r->sumMB);
    double varM = (double)(n * sM2 - sM * sM) / (nn * nn);
    double varA = (double)(n * sM2 - sA * sA) / (nn * nn);
    double varB = (double)(n * sB2 - sB * sB) / (nn * nn);
    double covMB = (double)(n * sMB - sM * sB) / (nn * nn);
    double meanM = (double)r->sumM / nn;
    double meanA = (double)r->sumAbsM / nn;
    double meanB = (double)r->sumB / nn;
    r->m = meanM / N;
    r->abs_m = meanA / N;
    r->e = (-J * meanB - h * meanM) / N;
    r->chi = varM / (N * T);
    r->chi_abs = varA / (N * T);
    double varE = J * J * varB + h * h * varM + 2.0 * J * h * covMB;
    r->C = varE / (N * T * T);
}

/* Curie temperature of a scan (Sec. 4, Table 1; Fig. 3): the T whose step has the largest
 * chi' = (<M^2> - <|M|>^2)/(N T) (the derived chi_abs), over the steps with measured sweeps at a
 * finite T > 0; the first of equal maxima.  Returns the step's index, or -1 if none qualifies. */
int or_estimate_tc(const or_step_obs* r, int n, double* T_c)
{
    int best = -1;
    for (int k = 0; k < n; ++k) {
        if (r[k].n_meas <= 0 || !(r[k].T > 0.0) || isinf(r[k].T)) continue;
        if (best < 0 || r[k].chi_abs > r[best].chi_abs) best = k;
    }
    if (best >= 0 && T_c) *T_c = r[best].T;
    return best;
}

/* ---------------------------------------------------------------- the sweep ---------- */
/* One schedule step after another; the state carries over (Sec. 3: "for each step of
 * temperature or field").  Each sweep visits colour 0, 1, 2, 3 and, within a colour, every
 * occupied site once (items 1-5 of Sec. 5 for each). */
int or_run(or_film* f, int nsteps, const double* T, const double* h, const int* sweeps_eq,
           const int* sweeps_meas, double J, double h_s, or_step_obs* rec, int64_t* series)
{
    if (!f || nsteps < 0 || (nsteps > 0 && (!T || !h || !sweeps_eq || !sweeps_meas || !rec)))
        return OR_ERR_ARG;
    if (!isfinite(J) || !isfinite(h_s)) return OR_ERR_SCHEDULE;
    for (int k = 0; k < nsteps; ++k) {
        if (!(T[k] >= 0.0) || isnan(T[k]) || !isfinite(h[k]) || sweeps_eq[k] < 0 || sweeps_meas[k] < 0)
            return OR_ERR_SCHEDULE;
    }
    int64_t nser = 0;
    for (int k = 0; k < nsteps; ++k) {
        uint32_t thr[25][2];
        for (int n = -12; n <= 12; ++n) {
            thr[n + 12][0] = or_threshold(T[k], h[k], J, n, -1);
            thr[n + 12][1] = or_threshold(T[k], h[k], J, n, +1);
        }
        uint32_t gate = or_gate_threshold(T[k], h_s);

        or_step_obs* r = &rec[k];
        memset(r, 0, sizeof(*r));
        r->T = T[k];
        r->h = h[k];
        i128 sM2 = 0, sB2 = 0, sMB = 0;
        int total = sweeps_eq[k] + sweeps_meas[k];
        for (int t = 0; t < total; ++t) {
            uint64_t sweep = (uint64_t)(f->sweep + 1);
            for (int colour = 0; colour < 4; ++colour) {
                for (int z = 0; z < f->L; ++z)
                    for (int y = 0; y < f->R; ++y)
                        for (int x = 0; x < f->C; ++x) {
                            if (or_colour(x, y, z) != colour) continue;
                            size_t p = site_of(f, x, y, z);
                            if (!f->occ[p]) continue;
                            /* Eq. 9 gate first (items 4-5), from its own stream. */
                            if (gate != OR_ALWAYS) {
                                uint32_t g = or_site_word(f, OR_STREAM_GATE, sweep, x, y, z);
                                if (!(g < gate)) continue;
                            }
                            int s = f->spin[p];
                            int n = neighbour_sum(f, x, y, z);
                            uint32_t a = thr[n + 12][s > 0 ? 1 : 0];
                            int accept;
                            if (a == OR_ALWAYS) {
                                accept = 1;          /* E2 <= E1: p = 1 > r */
                            } else {
                                uint32_t u = or_site_word(f, OR_STREAM_METROPOLIS, sweep, x, y, z);
                                accept = u < a;
                            }
                            if (accept) {
                                f->spin[p] = (int8_t)(-s);
                                f->M += -2 * s;
                                f->B += -2 * (int64_t)s * n;
                            }
                        }
            }
            f->sweep += 1;
            if (series) {
                series[2 * nser + 0] = f->M;
                series[2 * nser + 1] = f->B;
            }
            ++nser;
            if (t >= sweeps_eq[k]) {
                r->n_meas += 1;
                r->sumM += f->M;
                r->sumAbsM += f->M < 0 ? -f->M : f->M;
                r->sumB += f->B;
                sM2 += (i128)f->M * f->M;
                sB2 += (i128)f->B * f->B;
                sMB += (i128)f->M * f->B;
            }
        }
        r->M_last = f->M;
        r->B_last = f->B;
        put128(r->sumM2, sM2);
        put128(r->sumB2, sB2);
        put128(r->sumMB, sMB);
        or_derive(r, f->n_occ, J);

        int64_t M, B;
        or_recompute(f, &M, &B);
        if (M != f->M || B != f->B) return OR_ERR_STATE;   /* incremental bookkeeping broke */
    }
    return OR_OK;
}

/* ---------------------------------------------------------------- PMOKE image -------- */
/* Sec. 6: only the surface atoms are shown, white for spin up and black for spin down. */
int64_t or_surface_image(const or_film* f, uint8_t* out)
{
    int64_t up = 0;
    for (int y = 0; y < f->R; ++y)
        for (int x = 0; x < f->C; ++x) {
            int top = -1;
            for (int z = 0; z < f->L; ++z)
                if (f->occ[site_of(f, x, y, z)]) top = z;
            uint8_t v = 128;
            if (top >= 0) {
                v = f->spin[site_of(f, x, y, top)] > 0 ? 255 : 0;
                if (v == 255) ++up;
            }
            out[(size_t)y * (size_t)f->C + (size_t)x] = v;
        }
    return up;
}

/* ---------------------------------------------------------------- exact enumeration -- */
/* Eqs. 4-5: Z = sum over the 2^N configurations of exp(-H/T); each configuration has
 * probability exp(-H/T)/Z.  Weights are taken relative to the lowest energy for range. */
int or_exact(const or_film* f, double T, double h, double J, double* out)
{
    if (!f || !out || !(T > 0.0)) return OR_ERR_ARG;
    int N = (int)f->n_occ;
    if (N < 1 || N > 24) return OR_ERR_ARG;
    int* idx = (int*)malloc(sizeof(int) * (size_t)N);
    int* bi = (int*)malloc(sizeof(int) * (size_t)(12 * N));
    int* bj = (int*)malloc(sizeof(int) * (size_t)(12 * N));
    int8_t* s = (int8_t*)malloc((size_t)N);
    if (!idx || !bi || !bj || !s) { free(idx); free(bi); free(bj); free(s); return OR_ERR_OOM; }
    size_t nsites = (size_t)f->R * (size_t)f->C * (size_t)f->L;
    int* rank = (int*)malloc(sizeof(int) * nsites);
    if (!rank) { free(idx); free(bi); free(bj); free(s); return OR_ERR_OOM; }
    int cnt = 0;
    for (int z = 0; z < f->L; ++z)
        for (int y = 0; y < f->R; ++y)
            for (int x = 0; x < f->C; ++x) {
                size_t p = site_of(f, x, y, z);
                rank[p] = -1;
                if (f->occ[p]) { rank[p] = cnt; idx[cnt] = (int)p; ++cnt; }
            }
    int nb = 0;
    for (int z = 0; z < f->L; ++z)
        for (int y = 0; y < f->R; ++y)
            for (int x = 0; x < f->C; ++x) {
                size_t p = site_of(f, x, y, z);
                if (!f->occ[p]) continue;
                for (int k = 0; k < 12; ++k) {
                    int a, b, c;
                    if (!neighbour(f, x, y, z, k, &a, &b, &c)) continue;
                    size_t q = site_of(f, a, b, c);
                    if (!f->occ[q] || rank[q] <= rank[p]) continue;   /* each bond once */
                    bi[nb] = rank[p]; bj[nb] = rank[q]; ++nb;
                }
            }
    /* lowest energy over all states, for numerically safe weights */
    uint64_t nstates = 1ull << N;
    double Emin = INFINITY;
    for (uint64_t st = 0; st < nstates; ++st) {
        int64_t M = 0, B = 0;
        for (int i = 0; i < N; ++i) { s[i] = ((st >> i) & 1) ? 1 : -1; M += s[i]; }
        for (int b = 0; b < nb; ++b) B += s[bi[b]] * s[bj[b]];
        double E = -J * (double)B - h * (double)M;
        if (E < Emin) Emin = E;
    }
    long double Z = 0, aM = 0, aA = 0, aM2 = 0, aE = 0, aE2 = 0, aB = 0;
    for (uint64_t st = 0; st < nstates; ++st) {
        int64_t M = 0, B = 0;
        for (int i = 0; i < N; ++i) { s[i] = ((st >> i) & 1) ? 1 : -1; M += s[i]; }
        for (int b = 0; b < nb; ++b) B += s[bi[b]] * s[bj[b]];
        double E = -J * (double)B - h * (double)M;
        long double w = expl(-(long double)(E - Emin) / (long double)T);
        Z += w;
        aM += w * M;
        aA += w * (M < 0 ? -M : M);
        aM2 += w * (long double)M * M;
        aE += w * E;
        aE2 += w * (long double)E * E;
        aB += w * B;
    }
    out[0] = (double)(aM / Z);
    out[1] = (double)(aA / Z);
    out[2] = (double)(aM2 / Z);
    out[3] = (double)(aE / Z);
    out[4] = (double)(aE2 / Z);
    out[5] = (double)(aB / Z);
    free(idx); free(bi); free(bj); free(s); free(rank);
    return OR_OK;
}
