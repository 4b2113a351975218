// Step a4: fold the exact int32 partial sums of the raw-moment step into the
// int64 S_ab and apply Eq. (1):
//     Gamma = (1/N) S_ab - (S_a/N)(S_b/N) = (N S_ab - S_a S_b) / N^2.
// The numerator is computed exactly in int64 (the host refuses inputs for which
// N^2 max(A) max(B) could reach 2^63), converted to double with one rounding
// and divided once, both correctly rounded (IEEE round-to-nearest-even), so
// Gamma equals the exact-numerator formula bit for bit.  When the numerator is
// below 2^53 the conversion is exact and Gamma is the correctly rounded value
// of Eq. (1) itself.
//
// Division: GB300's FP64 pipe runs at a small fraction of its FP32 rate, and an
// IEEE double division costs a dozen FP64 instructions.  With the divisor
// D = N^2 the same for every entry, the kernel takes one FP64 multiply by the
// host-computed reciprocal (within 2 ulp of the quotient) and then fixes the
// last bit exactly with 128-bit integer arithmetic: q = M * 2^E is the
// correctly rounded A / D iff (2M - 1) D <= 2 A 2^-E <= (2M + 1) D, ties to even.
// Numerators of 2^53 or more (possible only for very long acquisitions) take
// the IEEE division.
//
// The optional FP32 copy is written slice-major ([b][a]) for the refocusing
// step, through a shared-memory transpose.
#include "kernels.cuh"

namespace cpi {
namespace {

constexpr int kTile = 32;

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
__device__ __forceinline__ uint64_t div_rn_bits(uint64_t A, uint64_t D, double q0) {
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

__global__ void __launch_bounds__(256) fold_kernel(const int32_t* __restrict__ partial,
                                                   int n_chunks, int64_t M, int64_t N,
                                                   int64_t* s_ab, int accumulate, int write_sab,
                                                   const int64_t* __restrict__ s_a,
                                                   const int64_t* __restrict__ s_b,
                                                   int64_t n_frames, double d_div, double d_inv,
                                                   int fast_div, double* gamma, float* gamma_f32) {
    __shared__ float tile[kTile][kTile + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;    // 32 x 8
    const int64_t b = (int64_t)blockIdx.x * kTile + tx;
    const bool want_g = gamma != nullptr || gamma_f32 != nullptr;
    const int64_t plane = M * N;
    const int64_t row_tiles = (M + kTile - 1) / kTile;
    const uint64_t Dint = (uint64_t)d_div;
    for (int64_t rt = blockIdx.y; rt < row_tiles; rt += gridDim.y) {
        const int64_t a0 = rt * kTile;
#pragma unroll
        for (int k = 0; k < kTile / 8; ++k) {
            const int64_t a = a0 + ty + 8 * k;
            if (a < M && b < N) {
                const int64_t idx = a * N + b;
                int64_t s = accumulate ? s_ab[idx] : 0;
                for (int c = 0; c < n_chunks; ++c) s += (int64_t)__ldg(partial + (int64_t)c * plane + idx);
                if (write_sab) s_ab[idx] = s;
                if (want_g) {
                    const int64_t num = n_frames * s - __ldg(s_a + a) * __ldg(s_b + b);
                    const uint64_t A = num < 0 ? (uint64_t)(-num) : (uint64_t)num;
                    double g;
                    if (num == 0) {
                        g = 0.0;
                    } else if (fast_div && A < (1ull << 53)) {
                        const double q0 = (double)A * d_inv;
                        uint64_t bits = div_rn_bits(A, Dint, q0);
                        if (num < 0) bits |= 1ull << 63;
                        g = __longlong_as_double((long long)bits);
                    } else {
                        g = __ddiv_rn(__ll2double_rn(num), d_div);
                    }
                    if (gamma) gamma[idx] = g;
                    tile[ty + 8 * k][tx] = __double2float_rn(g);
                }
            }
        }
        if (gamma_f32 != nullptr) {
            __syncthreads();
            // slice-major copy: gamma_f32[b][a]
#pragma unroll
            for (int k = 0; k < kTile / 8; ++k) {
                const int64_t bb = (int64_t)blockIdx.x * kTile + ty + 8 * k;
                const int64_t aa = a0 + tx;
                if (aa < M && bb < N) gamma_f32[bb * M + aa] = tile[tx][ty + 8 * k];
            }
            __syncthreads();
        }
    }
}

}  // namespace

cudaError_t launch_fold(const int32_t* partial, int n_chunks, int64_t M, int64_t N,
                        int64_t* s_ab, int accumulate, int write_sab, const int64_t* s_a,
                        const int64_t* s_b, int64_t n_frames, double* gamma, float* gamma_f32,
                        cudaStream_t st) {
    const int64_t gx = (N + kTile - 1) / kTile, gy = (M + kTile - 1) / kTile;
    const unsigned gyl = (unsigned)(gy < 65535 ? gy : 65535);
    const double nd = (double)n_frames;
    const double d_div = nd * nd;                    // the divisor of Eq. (1), as a double
    const double d_inv = 1.0 / d_div;
    // integer-checked division: needs D an exact integer in [2, 2^52)
    const int fast = (n_frames >= 2 && d_div < 4503599627370496.0) ? 1 : 0;
    fold_kernel<<<dim3((unsigned)gx, gyl), 256, 0, st>>>(partial, n_chunks, M, N, s_ab, accumulate,
                                                         write_sab, s_a, s_b, n_frames, d_div, d_inv,
                                                         fast, gamma, gamma_f32);
    return cudaGetLastError();
}

}  // namespace cpi
