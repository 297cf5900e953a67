// pf_average.cu -- Definition 1's average over filters, exact in FP64.
//
// When the M filters of an ensemble are split over several processes, each
// process holds the estimates of its own filters and the average
// (1/M) sum_m phi_m (Definition 1) is formed from all of them.  The sum here
// is exact: every double is added into one wide fixed-point integer (a
// Kulisch-style accumulator spanning the whole binary64 range, in units of
// the smallest subnormal 2^-1074), and the exact total is rounded once to the
// nearest double (ties to even).  The rounded sum therefore does not depend
// on the order of the terms or on how they were split over processes, and
// the average is that sum divided by M (one more IEEE rounding).  Host code
// only: the sum is n_stat x M values, gathered once per observation.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>

#include "pf.h"

namespace {

// 2^-1074 .. 2^1024 is 2098 bits; the 32-bit limbs below leave room for the
// carries of 2^31 terms of either sign.
constexpr int kLimbs = 70;

struct ExactSum {
    int64_t limb[kLimbs];  // limb k holds a signed multiple of 2^(32k - 1074)
    bool nan = false;
    int inf_sign = 0;      // +1 / -1: an infinity of that sign was added; 2: both signs
    ExactSum() { std::memset(limb, 0, sizeof(limb)); }

    void add(double x)
    {
        if (std::isnan(x)) { nan = true; return; }
        if (std::isinf(x)) {
            const int s = x > 0 ? 1 : -1;
            inf_sign = inf_sign == 0 ? s : (inf_sign == s ? s : 2);
            return;
        }
        uint64_t bits;
        std::memcpy(&bits, &x, sizeof(bits));
        const bool neg = bits >> 63;
        const int e = (int)((bits >> 52) & 0x7ff);
        uint64_t m = bits & ((uint64_t(1) << 52) - 1);
        if (e) m |= uint64_t(1) << 52;
        if (!m) return;
        // x = m 2^(max(e,1) - 1075) = m 2^-1074 2^shift
        const int shift = (e ? e : 1) - 1;
        const int k = shift >> 5, off = shift & 31;
        // m << off spans at most 85 bits: three 32-bit pieces
        const unsigned __int128 v = (unsigned __int128)m << off;
        const int64_t p0 = (int64_t)(uint32_t)v, p1 = (int64_t)(uint32_t)(v >> 32), p2 = (int64_t)(uint32_t)(v >> 64);
        if (neg) { limb[k] -= p0; limb[k + 1] -= p1; limb[k + 2] -= p2; }
        else { limb[k] += p0; limb[k + 1] += p1; limb[k + 2] += p2; }
    }

    // Carries so that limbs 0..kLimbs-2 lie in [0, 2^32); the top limb keeps the sign.
    void normalise()
    {
        for (int k = 0; k + 1 < kLimbs; ++k) {
            const int64_t carry = limb[k] >> 32;  // floor division by 2^32
            limb[k] -= carry * (int64_t(1) << 32);
            limb[k + 1] += carry;
        }
    }

    int bit(int i) const { return (int)((limb[i >> 5] >> (i & 31)) & 1); }

    // The exact total rounded to the nearest double, ties to even.
    double rounded()
    {
        if (nan || inf_sign == 2) return std::numeric_limits<double>::quiet_NaN();
        if (inf_sign) return inf_sign * std::numeric_limits<double>::infinity();
        normalise();
        bool neg = false;
        if (limb[kLimbs - 1] < 0) {  // negate: two's complement over the limbs
            neg = true;
            for (int k = 0; k < kLimbs; ++k) limb[k] = -limb[k];
            normalise();
        }
        int top = kLimbs - 1;
        while (top >= 0 && limb[top] == 0) --top;
        if (top < 0) return 0.0;
        int lead = 31;
        while (!((limb[top] >> lead) & 1)) --lead;
        const int nbits = 32 * top + lead + 1;  // the magnitude has nbits significant bits
        double r;
        if (nbits <= 53) {
            uint64_t v = 0;
            for (int i = nbits - 1; i >= 0; --i) v = (v << 1) | (uint64_t)bit(i);
            r = std::ldexp((double)v, -1074);  // exact: fewer than 54 bits, at or above 2^-1074
        } else {
            const int lo = nbits - 53;
            uint64_t v = 0;
            for (int i = nbits - 1; i >= lo; --i) v = (v << 1) | (uint64_t)bit(i);
            const int half = bit(lo - 1);
            bool sticky = false;
            for (int i = lo - 2; i >= 0 && !sticky; --i) sticky = bit(i);
            if (half && (sticky || (v & 1))) ++v;  // v may reach 2^53: still exact in a double
            r = std::ldexp((double)v, lo - 1074);  // overflows to infinity past the binary64 range
        }
        return neg ? -r : r;
    }
};

}  // namespace

extern "C" {

pf_status pf_ensemble_average(int32_t M, int32_t n_stat, const double *h_est, double *h_out)
{
    if (M < 1 || n_stat < 1 || !h_est || !h_out) return PF_EINVAL;
    for (int32_t s = 0; s < n_stat; ++s) {
        ExactSum acc;
        for (int32_t m = 0; m < M; ++m) acc.add(h_est[(size_t)m * n_stat + s]);
        h_out[s] = acc.rounded() / (double)M;
    }
    return PF_OK;
}

}  // extern "C"
