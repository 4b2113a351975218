// Correctly rounded Gamma of Eq. (1) from exact integer sums (the fold kernel).
//
// Gamma = RN(RN(num) / RN(N * N)) with num = N S_ab - S_a S_b exact in int64:
// the same two IEEE round-to-nearest-even operations a plain C evaluation of
// (double)num / ((double)N * (double)N) performs.  GB300's FP64 pipe runs at a
// small fraction of its FP32 rate and an IEEE double division costs a dozen
// FP64 instructions, so the quotient is taken as one FP64 multiply by the
// reciprocal of the common divisor D = N^2 (within 2 ulp) and its last bit is
// fixed exactly with integer arithmetic: q = M 2^E is the correctly rounded
// A / D iff (2M - 1) D <= 2 A 2^-E <= (2M + 1) D, ties to even.
#pragma once
#include <cstdint>

namespace cpi {

struct U128 {
    uint64_t hi, lo;
};
__device__ __forceinline__ U128 mul64(uint64_t a, uint64_t b) { return {__umul64hi(a, b), a * b}; }
__device__ __forceinline__ U128 shl(uint64_t a, int s) {   // a * 2^s, 1 <= s <= 127
    if (s >= 64) return {a << (s - 64), 0};
    return {a >> (64 - s), a << s};
}
__device__ __forceinline__ int cmp(U128 x, U128 y) {
    if (x.hi != y.hi) return x.hi < y.hi ? -1 : 1;
    if (x.lo != y.lo) return x.lo < y.lo ? -1 : 1;
    return 0;
}

// Correctly rounded A / D for 1 <= A < 2^53 and 2 <= D < 2^52 (integers), given
// an estimate q0 within a few ulp.  Returns the double's bit pattern.  The
// candidate M * 2^E (M in [2^52, 2^53)) rounds A / D iff the quotient lies in
// its rounding interval: [(M - 1/2), (M + 1/2)] 2^E, except that the lower end is
// (M - 1/4) 2^E for M = 2^52, whose lower neighbour has half the spacing.
static __device__ __noinline__ uint64_t div_rn_bits(uint64_t A, uint64_t D, double q0) {
    const uint64_t b = (uint64_t)__double_as_longlong(q0);
    uint64_t M = (b & ((1ull << 52) - 1)) | (1ull << 52);
    int E = (int)((b >> 52) & 0x7ff) - 1075;
    constexpr uint64_t kLo = 1ull << 52, kHi = 1ull << 53;
#pragma unroll 1
    for (int it = 0; it < 6; ++it) {
        const U128 X = shl(A, 1 - E);                   // 2 A 2^-E, compared with (2M +- 1) D
        const int ch = cmp(X, mul64(2 * M + 1, D));
        if (ch > 0) {                                    // above the interval: step up
            if (++M == kHi) { M = kLo; E += 1; }
            continue;
        }
        if (M == kLo) {
            if (cmp(X, mul64(2 * M, D)) < 0) {           // below M itself: previous binade
                M = kHi - 1;
                E -= 1;
                continue;
            }
        } else {
            const int cl = cmp(X, mul64(2 * M - 1, D));
            if (cl < 0) {                                // below the interval: step down
                --M;
                continue;
            }
            if (cl == 0) {                               // half-way to M - 1: ties to even
                if (M & 1) --M;
                break;
            }
        }
        if (ch == 0 && (M & 1)) {                        // half-way to M + 1: ties to even
            if (++M == kHi) { M = kLo; E += 1; }
        }
        break;
    }
    return ((uint64_t)(E + 1075) << 52) | (M & (kLo - 1));
}

// Fast path of div_rn_bits: with q0 = M * 2^E within 2 ulp of A / D, the
// residual R = A 2^-E - M D satisfies |R| < 3 D < 2^62, so its low 64 bits
// (wrap-around arithmetic) are R itself; q is the nearest double iff
// -D < 2R < D.  Two unit steps reach it.  Candidates near a power of two (where
// the spacing of doubles changes) take the 128-bit routine.
__device__ __forceinline__ uint64_t div_rn_bits_fast(uint64_t A, uint64_t D, double q0) {
    const uint64_t b = (uint64_t)__double_as_longlong(q0);
    int64_t M = (int64_t)((b & ((1ull << 52) - 1)) | (1ull << 52));
    const int E = (int)((b >> 52) & 0x7ff) - 1075;
    if (M <= (1ll << 52) + 2 || M >= (1ll << 53) - 3) return div_rn_bits(A, D, q0);
    const int s = -E;                                          // 1 .. 106
    const uint64_t As = s < 64 ? (A << s) : 0ull;
    int64_t R = (int64_t)(As - (uint64_t)M * D);
    const int64_t Dd = (int64_t)D;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        if (2 * R > Dd) { ++M; R -= Dd; }
        else if (2 * R < -Dd) { --M; R += Dd; }
    }
    if (2 * R == Dd && (M & 1)) ++M;                            // ties to even
    else if (2 * R == -Dd && (M & 1)) --M;
    return ((uint64_t)(E + 1075) << 52) | ((uint64_t)M & ((1ull << 52) - 1));
}

// Exact double of an integer 1 <= A < 2^53, built from its bits (no FP64 pipe).
__device__ __forceinline__ double u53_to_double(uint64_t A) {
    const int e = 63 - __clzll((long long)A);                 // position of the leading one, <= 52
    const uint64_t m = A << (52 - e);
    return __longlong_as_double((long long)(((uint64_t)(e + 1023) << 52) | (m & ((1ull << 52) - 1))));
}

// Round-to-nearest-even double -> float for |x| in the normal float range,
// done on the integer bits; other magnitudes use the hardware conversion.
__device__ __forceinline__ float double_to_float_rn(double x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    if (e < -126 || e > 127) return __double2float_rn(x);
    const uint64_t m = b & ((1ull << 52) - 1);
    uint32_t f = ((uint32_t)(e + 127) << 23) | (uint32_t)(m >> 29);
    const uint64_t rem = m & ((1ull << 29) - 1);
    if (rem > (1ull << 28) || (rem == (1ull << 28) && (f & 1u))) ++f;   // carry may bump the exponent
    f |= (uint32_t)(b >> 32) & 0x80000000u;
    return __uint_as_float(f);
}


// Parameters of the finalisation shared by every entry of one correlation.
struct GammaDiv {
    int64_t n;          // frame count N
    double d;           // RN(N * N)
    double inv;         // RN(1 / d)
    int fast;           // 1 when d is an exact integer in [2, 2^52)
};

inline GammaDiv make_gamma_div(int64_t n_frames) {
    GammaDiv g;
    g.n = n_frames;
    const double nd = (double)n_frames;
    g.d = nd * nd;
    g.inv = 1.0 / g.d;
    g.fast = (n_frames >= 2 && g.d < 4503599627370496.0) ? 1 : 0;
    return g;
}

// Round-to-nearest-even double of a signed 128-bit integer (hi, lo), built from
// its bits: the leading 53 bits, then the next bit and a sticky bit of the rest.
__device__ __forceinline__ double i128_to_double_rn(int64_t hi, uint64_t lo) {
    const bool neg = hi < 0;
    uint64_t H = (uint64_t)hi, L = lo;
    if (neg) {                                                   // |x|: two's complement negation
        L = ~L + 1ull;
        H = ~H + (L == 0 ? 1ull : 0ull);
    }
    if (H == 0 && L == 0) return 0.0;
    int e;                                                      // position of the leading one
    uint64_t top, rest;                                         // leading 64 bits from the one; bits below
    if (H != 0) {
        const int z = __clzll((long long)H);
        e = 127 - z;
        top = z == 0 ? H : (H << z) | (L >> (64 - z));
        rest = z == 0 ? L : (L << z);
    } else {
        const int z = __clzll((long long)L);
        e = 63 - z;
        top = L << z;
        rest = 0;
    }
    uint64_t m = top >> 11;                                     // 53 bits, leading one at bit 52
    const uint64_t r = top & 0x7ffull;                          // the 11 bits below the mantissa
    const bool sticky = (r & 0x3ffull) != 0 || rest != 0;
    if ((r & 0x400ull) && (sticky || (m & 1ull))) {
        if (++m == (1ull << 53)) {
            m >>= 1;
            ++e;
        }
    }
    const uint64_t bits = ((uint64_t)(e + 1023) << 52) | (m & ((1ull << 52) - 1)) | (neg ? (1ull << 63) : 0ull);
    return __longlong_as_double((long long)bits);
}

// Gamma from the exact numerator num = N S_ab - S_a S_b.
__device__ __forceinline__ double gamma_from_num(int64_t num, const GammaDiv& gd) {
    if (num == 0) return 0.0;
    const uint64_t A = num < 0 ? (uint64_t)(-num) : (uint64_t)num;
    if (gd.fast && A < (1ull << 53)) {
        const double q0 = u53_to_double(A) * gd.inv;
        uint64_t bits = div_rn_bits_fast(A, (uint64_t)gd.d, q0);
        if (num < 0) bits |= 1ull << 63;
        return __longlong_as_double((long long)bits);
    }
    return __ddiv_rn(__ll2double_rn(num), gd.d);
}

// Gamma from arbitrary int64 sums (cpi_correlate_finalize: sums accumulated over
// many calls, whose products may leave int64): num = N S_ab - S_a S_b formed
// exactly in 128 bits.  A numerator that fits int64 takes gamma_from_num; a wider
// one is rounded once to double and divided by RN(N * N), the same two
// round-to-nearest operations as in the narrow case.
__device__ __forceinline__ double gamma_from_sums_wide(int64_t s_ab, int64_t s_a, int64_t s_b, const GammaDiv& gd) {
    const uint64_t lo1 = (uint64_t)gd.n * (uint64_t)s_ab, lo2 = (uint64_t)s_a * (uint64_t)s_b;
    const int64_t hi1 = __mul64hi((long long)gd.n, (long long)s_ab);
    const int64_t hi2 = __mul64hi((long long)s_a, (long long)s_b);
    const uint64_t lo = lo1 - lo2;
    const int64_t hi = hi1 - hi2 - (lo1 < lo2 ? 1 : 0);
    if (hi == ((int64_t)lo >> 63)) return gamma_from_num((int64_t)lo, gd);
    return __ddiv_rn(i128_to_double_rn(hi, lo), gd.d);
}

}  // namespace cpi
