// Step a4: fold the exact partial sums of the raw-moment step (uint32, one per
// frame chunk) into the int64 S_ab and apply Eq. (1):
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
// the IEEE division.  Sums handed to cpi_correlate_finalize may come from many
// accumulating calls, so there (wide != 0) the numerator is formed in 128 bits;
// one that does not fit int64 is rounded once to double and divided the same way.
//
// The optional FP32 copy is written slice-major ([b][a]) for the refocusing
// step, through a shared-memory transpose.
#include "gamma_div.cuh"
#include "kernels.cuh"

namespace cpi {
namespace {

constexpr int kTile = 32;
constexpr int kRowsPerThread = kTile / 8;

// CTA = 32 x 32 entries (32 x 8 threads, 4 rows each).  Every load of a
// thread's 4 entries is issued before any of them is used, so their latencies
// overlap; then the 4 quotients are formed and stored.  Idx: int32_t when every
// index (chunk slots included) fits, else int64_t.
template <typename Idx>
__global__ void __launch_bounds__(256, 4) fold_kernel(const int32_t* __restrict__ partial,
                                                   int n_chunks, int64_t M, int64_t N,
                                                   int64_t* s_ab, int accumulate, int write_sab,
                                                   const int64_t* __restrict__ s_a,
                                                   const int64_t* __restrict__ s_b,
                                                   const GammaDiv gd, int wide, double* gamma,
                                                   float* gamma_f32) {
    __shared__ float tile[kTile][kTile + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;    // 32 x 8
    const Idx b = (Idx)blockIdx.x * kTile + tx;
    const bool want_g = gamma != nullptr || gamma_f32 != nullptr;
    const Idx plane = (Idx)(M * N);
    const Idx row_tiles = (Idx)((M + kTile - 1) / kTile);
    const int64_t sb = (want_g && b < N) ? __ldg(s_b + b) : 0;
    for (Idx rt = blockIdx.y; rt < row_tiles; rt += gridDim.y) {
        const Idx a0 = rt * kTile;
        int64_t sum[kRowsPerThread], sa[kRowsPerThread];
#pragma unroll
        for (int k = 0; k < kRowsPerThread; ++k) {
            const Idx a = a0 + ty + 8 * k;
            sum[k] = (accumulate && a < M && b < N) ? s_ab[a * N + b] : 0;
            sa[k] = (want_g && a < M) ? __ldg(s_a + a) : 0;
        }
        for (int c = 0; c < n_chunks; ++c) {
#pragma unroll
            for (int k = 0; k < kRowsPerThread; ++k) {
                const Idx a = a0 + ty + 8 * k;
                if (a < M && b < N) sum[k] += (int64_t)(uint32_t)__ldg(partial + (Idx)c * plane + a * (Idx)N + b);
            }
        }
#pragma unroll
        for (int k = 0; k < kRowsPerThread; ++k) {
            const Idx a = a0 + ty + 8 * k;
            if (a < M && b < N) {
                const Idx idx = a * (Idx)N + b;
                if (write_sab) s_ab[idx] = sum[k];
                if (want_g) {
                    const double g = wide ? gamma_from_sums_wide(sum[k], sa[k], sb, gd)
                                          : gamma_from_num(gd.n * sum[k] - sa[k] * sb, gd);
                    if (gamma) gamma[idx] = g;
                    tile[ty + 8 * k][tx] = double_to_float_rn(g);
                }
            }
        }
        if (gamma_f32 != nullptr) {
            __syncthreads();
            // slice-major copy: gamma_f32[b][a]
#pragma unroll
            for (int k = 0; k < kTile / 8; ++k) {
                const Idx bb = (Idx)blockIdx.x * kTile + ty + 8 * k;
                const Idx aa = a0 + tx;
                if (aa < M && bb < N) gamma_f32[bb * (Idx)M + aa] = tile[tx][ty + 8 * k];
            }
            __syncthreads();
        }
    }
}

}  // namespace

cudaError_t launch_fold(const int32_t* partial, int n_chunks, int64_t M, int64_t N,
                        int64_t* s_ab, int accumulate, int write_sab, const int64_t* s_a,
                        const int64_t* s_b, int64_t n_frames, double* gamma, float* gamma_f32,
                        cudaStream_t st, int wide) {
    const int64_t gx = (N + kTile - 1) / kTile, gy = (M + kTile - 1) / kTile;
    const unsigned gyl = (unsigned)(gy < 65535 ? gy : 65535);
    const int64_t span = M * N * (n_chunks > 1 ? n_chunks : 1) + (int64_t)kTile * (M + N);
    if (span < ((int64_t)1 << 31))
        fold_kernel<int32_t><<<dim3((unsigned)gx, gyl), 256, 0, st>>>(
            partial, n_chunks, M, N, s_ab, accumulate, write_sab, s_a, s_b, make_gamma_div(n_frames), wide, gamma,
            gamma_f32);
    else
        fold_kernel<int64_t><<<dim3((unsigned)gx, gyl), 256, 0, st>>>(
            partial, n_chunks, M, N, s_ab, accumulate, write_sab, s_a, s_b, make_gamma_div(n_frames), wide, gamma,
            gamma_f32);
    return cudaGetLastError();
}

}  // namespace cpi
