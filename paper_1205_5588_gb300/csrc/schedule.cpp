// schedule.cpp — host fp64 threshold tables (Eq. 8, Eq. 9) and fp64 observables derived from
// the device's exact integer sums.
#include <cmath>
#include <cstdint>

#include "isf_internal.h"

namespace isf {

namespace {

// Number of 32-bit words u with (u + 0.5) * 2^-32 < p, i.e. ceil(p * 2^32 - 0.5) (0 when
// that is not positive): the flips Eq. 8 accepts when r = (u + 0.5) * 2^-32.  Counts of
// 2^32 - 1 and 2^32 both become kAlways ("every u"), an error of at most 2^-32.
uint32_t count_below(double p) {
    const double x = p * 4294967296.0 - 0.5;
    if (!(x > 0.0)) return 0u;
    const double n = std::ceil(x);
    if (n >= 4294967295.0) return kAlways;
    return static_cast<uint32_t>(n);
}

}  // namespace

// thr[(n + 12) * 2 + s'] for n = -12..12 (sum of the occupied neighbours' spins) and
// s' = 0 (spin -1) / 1 (spin +1): the flip costs dE = 2 s (J n + h) (Eq. 3); it is always taken
// when dE <= 0 and otherwise with probability exp(-dE / T) (Eq. 8).  Slot 50: the switching
// gate of Eq. 9, passed with probability exp(-|h_s| / T) (always when h_s = 0).
void build_step_table(double T, double h, double J, double h_s, uint32_t* out52) {
    for (int n = -12; n <= 12; ++n) {
        for (int sp = 0; sp < 2; ++sp) {
            const double s = sp ? 1.0 : -1.0;
            const double dE = 2.0 * s * (J * static_cast<double>(n) + h);
            uint32_t thr;
            if (dE <= 0.0) thr = kAlways;
            else thr = count_below(std::exp(-dE / T));
            out52[(n + 12) * 2 + sp] = thr;
        }
    }
    const double a = std::fabs(h_s);
    out52[kGateSlot] = (a == 0.0) ? kAlways : count_below(std::exp(-a / T));
    // aligned sites: n = +12 with s = +1, n = -12 with s = -1
    auto needs_word = [](uint32_t t) { return t != 0u && t != kAlways; };
    const bool always = needs_word(out52[(12 + 12) * 2 + 1]) || needs_word(out52[(-12 + 12) * 2 + 0]);
    bool never = false;
    for (int i = 0; i < 50; ++i) never |= out52[i] == 0u;
    out52[kFlagSlot] = (always ? kFlagAlwaysDraw : 0u) | (never ? 0u : kFlagNoNever);
}

namespace {
typedef __int128 i128;
typedef unsigned __int128 u128;
inline i128 from_words(const unsigned long long w[2]) {
    return static_cast<i128>((static_cast<u128>(w[1]) << 64) | static_cast<u128>(w[0]));
}
}  // namespace

// Fluctuation estimators over the n measured sweeps of a step (variance numerators
// n*sum(x^2) - sum(x)^2 formed exactly in 128-bit integers):
// out = {m, |m|, e, chi, chi', C}; E = -J B - h M (Eq. 3), N = occupied sites.
void derive_record(const StepRec& r, double T, double h, double J, long long n_occ, double out[6]) {
    if (r.n_meas <= 0 || n_occ <= 0) {
        for (int i = 0; i < 6; ++i) out[i] = NAN;
        return;
    }
    const i128 n = r.n_meas;
    const double nd = static_cast<double>(r.n_meas);
    const double N = static_cast<double>(n_occ);
    const i128 sM = r.sumM, sA = r.sumAbsM, sB = r.sumB;
    const i128 sM2 = from_words(r.sumM2), sB2 = from_words(r.sumB2), sMB = from_words(r.sumMB);
    const double var_m = static_cast<double>(n * sM2 - sM * sM) / (nd * nd);
    const double var_a = static_cast<double>(n * sM2 - sA * sA) / (nd * nd);
    const double var_b = static_cast<double>(n * sB2 - sB * sB) / (nd * nd);
    const double cov_mb = static_cast<double>(n * sMB - sM * sB) / (nd * nd);
    const double mean_m = static_cast<double>(r.sumM) / nd;
    const double mean_a = static_cast<double>(r.sumAbsM) / nd;
    const double mean_b = static_cast<double>(r.sumB) / nd;
    out[0] = mean_m / N;
    out[1] = mean_a / N;
    out[2] = (-J * mean_b - h * mean_m) / N;
    out[3] = var_m / (N * T);
    out[4] = var_a / (N * T);
    const double var_e = J * J * var_b + h * h * var_m + 2.0 * J * h * cov_mb;
    out[5] = var_e / (N * T * T);
}

}  // namespace isf
