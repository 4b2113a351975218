// Step a4: fold the exact int32 partial sums of the raw-moment step into the
// int64 S_ab and apply Eq. (1):
//     Gamma = (1/N) S_ab - (S_a/N)(S_b/N) = (N S_ab - S_a S_b) / N^2.
// The numerator is computed exactly in int64 (the host refuses inputs for which
// N^2 max(A) max(B) could reach 2^63), converted to double with one rounding
// and divided once, both correctly rounded (IEEE round-to-nearest), so Gamma
// equals the exact-numerator formula bit for bit.  When the numerator is below
// 2^53 the conversion is exact and Gamma is the correctly rounded value of
// Eq. (1) itself.  The optional FP32 copy is written slice-major ([b][a]) for the
// refocusing step, through a shared-memory transpose.
#include "kernels.cuh"

namespace cpi {
namespace {

constexpr int kTile = 32;

__global__ void __launch_bounds__(256) fold_kernel(const int32_t* __restrict__ partial,
                                                   int n_chunks, int64_t M, int64_t N,
                                                   int64_t* s_ab, int accumulate, int write_sab,
                                                   const int64_t* __restrict__ s_a,
                                                   const int64_t* __restrict__ s_b,
                                                   int64_t n_frames, double* gamma,
                                                   float* gamma_f32) {
    __shared__ float tile[kTile][kTile + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;    // 32 x 8
    const int64_t b = (int64_t)blockIdx.x * kTile + tx;
    const bool want_g = gamma != nullptr || gamma_f32 != nullptr;
    const double nd = (double)n_frames;
    const double n2 = nd * nd;
    const int64_t plane = M * N;
    const int64_t row_tiles = (M + kTile - 1) / kTile;
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
                    const double g = __ddiv_rn(__ll2double_rn(num), n2);
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
    fold_kernel<<<dim3((unsigned)gx, gyl), 256, 0, st>>>(partial, n_chunks, M, N, s_ab, accumulate,
                                                         write_sab, s_a, s_b, n_frames, gamma,
                                                         gamma_f32);
    return cudaGetLastError();
}

}  // namespace cpi
