// capi_internal.h — the library's film object and helpers shared by the C-ABI translation
// units (capi.cpp, batch.cpp).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "isf_internal.h"
#include "trace.h"
#include "../../include/isingfilm_tuning.h"

using isf::Layout;
using isf::DevFilm;
using isf::FilmState;
using isf::StepRec;

struct isf_lattice {
    Layout lay{};
    uint64_t seed = 0;
    int32_t init = 0;
    int device = 0;
    uint8_t* dev = nullptr;         // film buffer: spins | heights | state
    bool owns_dev = false;
    DevFilm f{};
    FilmState* st = nullptr;
    std::vector<uint8_t> heights;   // host copy (validation of written spins, save)
    int64_t n_occ = 0, n_bonds = 0;
    int64_t sweep = 0;              // Metropolis sweeps done
    // schedule
    int32_t nsteps = 0;
    std::vector<double> T, h;
    std::vector<int32_t> eq, tot;
    double J = 1.0, h_s = 0.0;
    bool use_gate = false;
    uint8_t* sched = nullptr;       // tables | eq | tot | records
    uint32_t* d_tables = nullptr;
    int32_t* d_eq = nullptr;
    int32_t* d_tot = nullptr;
    StepRec* d_recs = nullptr;
    int32_t k = 0, pos = 0;         // cursor: step, sweeps done in it
    // trace
    long long* d_trace = nullptr;
    int64_t trace_cap = 0, trace_n = 0;
    // launch shape and path
    int32_t ctas = 0, threads = 0;
    int32_t item_sites = 0;         // resident kernel's sites per work item (0: automatic)
    int32_t path = ISF_PATH_AUTO;
    int32_t last_path = 0, last_ctas = 0, last_threads = 0;   // shape of the last sweep launch
    int32_t last_sites = 0;
    // row-slab kernel (packed whole films with word lists): host copy of the row offsets of the
    // row-major lists, and the row partition last uploaded (part_G CTAs, at most part_nrm rows each)
    std::vector<int32_t> roff_h;
    std::vector<int32_t> part_h;
    int32_t part_G = 0, part_nrm = 0;
    // row slab of a larger film (f.slab): whole-film rows [y0, y1) are this film's own rows,
    // local row 0 is whole-film row ya; the next colour pass isf_run_pass expects
    int32_t slab_y0 = 0, slab_y1 = 0, slab_ya = 0, slab_rows = 0;
    int32_t pass_next = 0;
    int64_t slab_m0 = 0, slab_b2 = 0;   // own share of the whole film's M and 2B at creation
    cudaStream_t last = nullptr;
};


namespace isf {
int set_last_error(int code, const char* msg);
// Sweep arguments for the next nsweeps of the film's schedule (no device work).
SweepArgs sweep_args(const isf_lattice* L, int64_t nsweeps);
// Sweeps left in the film's schedule.
int64_t sweeps_remaining(const isf_lattice* L);
// Move the film's schedule cursor, sweep counter and trace cursor past nsweeps sweeps.
void advance_cursor(isf_lattice* L, int64_t nsweeps);
}  // namespace isf
