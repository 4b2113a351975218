// Learned denoiser of Gamma (the paper has none; the network is the project's
// "learned denoiser" row): a 4-layer 3 x 3 convolutional network that maps
// Gamma measured from few frames to Gamma of many frames, trained on pairs the
// method generates.  The plain Gamma of Eq. (1) stays the fallback and the
// reference its error is measured against.
//
// Network, per angular slice b = (br, bc) of Gamma (float [Mb][ha * wa]):
//   input x: 9 channels, the slices of the 3 x 3 angular neighbourhood
//            (br + dy, bc + dx), channel 3 (dy + 1) + (dx + 1), zero outside the
//            angular grid, the whole of Gamma scaled by s = 1 / rms(Gamma_in);
//   a1 = relu(conv(x; 9 -> 32)), a2 = relu(conv(a1; 32 -> 32)),
//   a3 = relu(conv(a2; 32 -> 32)), y = x[4] + conv(a3; 32 -> 1)
//   (3 x 3 kernels, zero padding 1, biases); Gamma_out = y / s.
// Storage: x, a1..a3 and the weights in use are bfloat16 (round to nearest
// even from float32); every sum is float32; y, the gradients and the float32
// master weights are float32.  Training minimises mean((y - s Gamma_target)^2)
// with Adam.
//
// The forward network runs on the tensor cores for image widths 32, 64 and 128
// (dn_conv_tc_kernel: implicit GEMMs over channels-last activations, below).
// Other widths and the backward pass use direct convolutions on the FP32 pipe:
// a CTA computes a tile of 8 x 32 output pixels of one slice for every output
// channel, each thread two pixels (rows r and r + 4 of its column) times all
// output channels, the input tile (with its 1-pixel halo) and the bf16-rounded
// weights staged in shared memory ([Cin][tap][Cout], so the output channels of
// one tap are read as broadcast vectors).  Weight gradients are summed per CTA
// over a fixed range of slices and the per-CTA partials added in a fixed order,
// so every result is deterministic.
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "ptx.cuh"

namespace cpi {
namespace {

constexpr int kTH = 8, kTW = 32;           // output tile: 8 rows x 32 columns
constexpr int kConvThreads = 128;          // 2 pixels per thread
constexpr int kSumBlocks = 256;

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// ------------------------------------------------------------------ scale
__global__ void dn_sumsq_kernel(const float* __restrict__ g, int64_t n, double* __restrict__ part) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)g[i];
        acc += v * v;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// s = 1 / rms, from the per-block sums in block order
__global__ void dn_scale_kernel(const double* __restrict__ part, int nparts, int64_t n, float* __restrict__ scale) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t = 0.0;
    for (int i = 0; i < nparts; ++i) t += part[i];
    const double ms = t / (double)n;
    *scale = ms > 0.0 ? (float)(1.0 / sqrt(ms)) : 1.0f;
}

// ------------------------------------------------------------------ input stack
// x[b][c][p] = bf16(Gamma[nb(b, c)][p] * s), zero outside the angular grid.
__global__ void dn_stack_kernel(const float* __restrict__ g, const float* __restrict__ scale, int hb, int wb,
                                int64_t ma, __nv_bfloat16* __restrict__ x) {
    const int b = blockIdx.z, c = blockIdx.y;
    const int br = b / wb, bc = b - br * wb;
    const int r = br + c / 3 - 1, q = bc + c % 3 - 1;
    const bool in = r >= 0 && r < hb && q >= 0 && q < wb;
    const float s = *scale;
    const float* src = in ? g + (int64_t)(r * wb + q) * ma : g;
    __nv_bfloat16* dst = x + ((int64_t)b * 9 + c) * ma;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < ma; p += (int64_t)gridDim.x * blockDim.x)
        dst[p] = __float2bfloat16_rn(in ? src[p] * s : 0.0f);
}

// ------------------------------------------------------------------ convolution
// MODE 0: hidden layer forward, bf16 in, out = bf16(relu(conv + bias)).
// MODE 1: last layer forward (COUT = 1), out (float) = x[4] + conv + bias.
// MODE 2: gradient with respect to a layer's input: "input" = the gradient at
//         the layer's output (float), masked by mask > 0 (the layer's ReLU) when
//         mask is given; kernel flipped and transposed; no bias; out float.
enum { kFwdHidden = 0, kFwdLast = 1, kBwdData = 2 };

template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(kConvThreads)
    dn_conv_kernel(const void* __restrict__ in_v, const __nv_bfloat16* __restrict__ mask,
                   const float* __restrict__ w, const float* __restrict__ bias,
                   const __nv_bfloat16* __restrict__ x0, void* __restrict__ out_v, int H, int W) {
    extern __shared__ __align__(16) float sm[];
    constexpr int TP = (kTH + 2) * (kTW + 2);
    float* sIn = sm;                          // [CIN][kTH + 2][kTW + 2]
    float* sW = sm + CIN * TP;                // [CIN][9][COUT]
    const int b = blockIdx.z;
    const int y0 = blockIdx.y * kTH, x0c = blockIdx.x * kTW;
    const int64_t HW = (int64_t)H * W;
    const int tid = threadIdx.x;

    // weights, rounded to bf16
    for (int i = tid; i < CIN * 9 * COUT; i += kConvThreads) {
        const int co = i % COUT, rest = i / COUT;
        const int tap = rest % 9, ci = rest / 9;
        float v;
        if (MODE == kBwdData) {
            // this kernel's input channel ci is the layer's output channel;
            // its output channel co is the layer's input channel; taps flipped
            v = w[((int64_t)ci * COUT + co) * 9 + (8 - tap)];
        } else {
            v = w[((int64_t)co * CIN + ci) * 9 + tap];
        }
        sW[i] = bf16r(v);
    }
    // input tile with halo
    for (int i = tid; i < CIN * TP; i += kConvThreads) {
        const int ci = i / TP, rem = i - ci * TP;
        const int ty = rem / (kTW + 2), tx = rem - ty * (kTW + 2);
        const int yy = y0 + ty - 1, xx = x0c + tx - 1;
        float v = 0.0f;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
            const int64_t idx = ((int64_t)b * CIN + ci) * HW + (int64_t)yy * W + xx;
            if (MODE == kBwdData) {
                v = static_cast<const float*>(in_v)[idx];
                if (mask != nullptr && !(__bfloat162float(mask[idx]) > 0.0f)) v = 0.0f;
            } else {
                v = __bfloat162float(static_cast<const __nv_bfloat16*>(in_v)[idx]);
            }
        }
        sIn[i] = v;
    }
    __syncthreads();

    const int cx = tid % kTW, ry = tid / kTW;      // column, first row (0..3); second row ry + 4
    float acc[2][COUT];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[k][co] = 0.0f;
#pragma unroll 1
    for (int ci = 0; ci < CIN; ++ci) {
        const float* src = sIn + ci * TP;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap % 3;
            const float v0 = src[(ry + ky) * (kTW + 2) + cx + kx];
            const float v1 = src[(ry + 4 + ky) * (kTW + 2) + cx + kx];
            const float* wt = sW + (ci * 9 + tap) * COUT;
            if constexpr (COUT % 4 == 0) {
#pragma unroll
                for (int co = 0; co < COUT; co += 4) {
                    const float4 q = *reinterpret_cast<const float4*>(wt + co);
                    acc[0][co] = __fmaf_rn(q.x, v0, acc[0][co]);
                    acc[1][co] = __fmaf_rn(q.x, v1, acc[1][co]);
                    acc[0][co + 1] = __fmaf_rn(q.y, v0, acc[0][co + 1]);
                    acc[1][co + 1] = __fmaf_rn(q.y, v1, acc[1][co + 1]);
                    acc[0][co + 2] = __fmaf_rn(q.z, v0, acc[0][co + 2]);
                    acc[1][co + 2] = __fmaf_rn(q.z, v1, acc[1][co + 2]);
                    acc[0][co + 3] = __fmaf_rn(q.w, v0, acc[0][co + 3]);
                    acc[1][co + 3] = __fmaf_rn(q.w, v1, acc[1][co + 3]);
                }
            } else {
#pragma unroll
                for (int co = 0; co < COUT; ++co) {
                    acc[0][co] = __fmaf_rn(wt[co], v0, acc[0][co]);
                    acc[1][co] = __fmaf_rn(wt[co], v1, acc[1][co]);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int yy = y0 + ry + 4 * k, xx = x0c + cx;
        if (yy >= H || xx >= W) continue;
        const int64_t p = (int64_t)yy * W + xx;
        if (MODE == kFwdHidden) {
            __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out_v);
#pragma unroll
            for (int co = 0; co < COUT; ++co)
                o[((int64_t)b * COUT + co) * HW + p] = __float2bfloat16_rn(fmaxf(acc[k][co] + bias[co], 0.0f));
        } else if (MODE == kFwdLast) {
            float* o = static_cast<float*>(out_v);
            const float xc = __bfloat162float(x0[((int64_t)b * 9 + 4) * HW + p]);
            o[(int64_t)b * HW + p] = xc + (acc[k][0] + bias[0]);
        } else {
            float* o = static_cast<float*>(out_v);
#pragma unroll
            for (int co = 0; co < COUT; ++co) o[((int64_t)b * COUT + co) * HW + p] = acc[k][co];
        }
    }
}

// ------------------------------------------------------------------ tensor-core forward
// Layers 0..2 (32 -> 32 channels; the 9-channel input is padded to 32 with zero
// channels and zero weights) as implicit GEMMs on tcgen05, for image widths 32,
// 64 and 128.  A unit is R = 256 / W output rows of one slice (two tiles of
// M = 128 pixels) for the 32 output channels.  The layer input is channels-last
// bf16 (64 bytes per pixel); TMA loads three copies of rows y0 - 1 .. y0 + R
// with the columns shifted by -1, 0, +1 (zeros outside the image), 64-byte
// swizzled, so that the A operand of tap (ky, kx) is copy kx from row ky on: an
// 8-row aligned slice, as W is a multiple of 8.  Weights: bf16 [tap][Cout][Cin],
// one TMA box.  Per tile 9 taps x 2 MMAs (M = 128, N = 32, K = 16) accumulate in
// 32 TMEM columns (FP32 sums); the epilogue adds the bias, applies ReLU, rounds
// to bf16 and writes channels-first (for the backward pass and the last layer)
// and channels-last (the next layer's input), each only if asked (inference
// needs no channels-first activations).  The last layer runs the same kernel
// with 16 output columns.
constexpr int kTcWBytes = 9 * 32 * 64;     // weights of one layer, bf16

inline int tc_rows(int W) { return 256 / W; }
inline size_t tc_copy_stride(int W) { return ((size_t)(tc_rows(W) + 2) * W * 64 + 1023) / 1024 * 1024; }
inline size_t tc_smem(int W) { return 1024 + 6 * tc_copy_stride(W) + kTcWBytes + 128; }   // 2 stages, NOUT <= 32

// NOUT = 32: hidden layer (bias, ReLU, bf16 out).  NOUT = 16: the last layer
// (32 -> 1, output channel 0 of 16; rows 1..15 of its weights are zero):
// y = x0[centre channel] + sum + bias, float, channels-first.
//
// Persistent: one CTA per SM walks the units u = (slice, block of R rows).
// Warp 0 (one thread) loads the weights once and then each unit's three copies
// into one of two stages; warp 1 (one thread) issues the unit's MMAs into one
// of two TMEM accumulators (2 tiles x NOUT columns each) and frees the stage;
// warps 2..5 drain an accumulator (TMEM lane quarter = warp % 4) while the next
// unit is loaded and multiplied.  Every wait is bounded; on a time-out the CTA
// records it, drains its own copies and MMAs, frees its tensor memory and stops.
//
// BWD: the input gradient of a hidden layer, g = conv(delta; flipped, transposed
// weights), no bias: delta arrives as two channels-last bf16 terms (hi, lo),
// loaded one after the other into the two stages of a unit and multiplied by
// the same weights into the same accumulator; the epilogue writes the FP32 sums
// channels-first to y_out [slice][32][H * W].
constexpr int kTcThreadsP = 192;          // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue
template <int NOUT, bool BWD = false>
__global__ void __launch_bounds__(kTcThreadsP, 1) dn_conv_tc_kernel(const __grid_constant__ CUtensorMap in_map,
                                                                   const __grid_constant__ CUtensorMap in_map_lo,
                                                                   const __grid_constant__ CUtensorMap w_map,
                                                                   const float* __restrict__ bias,
                                                                   __nv_bfloat16* __restrict__ out_cf,
                                                                   __nv_bfloat16* __restrict__ out_cl,
                                                                   const __nv_bfloat16* __restrict__ x0,
                                                                   float* __restrict__ y_out, int H, int W,
                                                                   int n_slices, unsigned int* status,
                                                                   unsigned long long timeout_ns) {
    constexpr bool kLast = NOUT == 16;
    constexpr int kWBytes = 9 * NOUT * 64;
    constexpr uint32_t kCols = 4 * NOUT;                        // 2 accumulators x 2 tiles x NOUT (64 or 128)
    extern __shared__ uint8_t smem_tc[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_tc) + 1023) & ~(uintptr_t)1023);
    const int R = 256 / W;
    const int nrb = (H + R - 1) / R, n_units = nrb * n_slices;
    const size_t cstride = ((size_t)(R + 2) * W * 64 + 1023) / 1024 * 1024;
    const uint32_t copy_bytes = (uint32_t)((R + 2) * W * 64);
    uint8_t* sw = sm + 6 * cstride;                             // stages: [2][3 copies]
    uint64_t* full = reinterpret_cast<uint64_t*>(sw + kWBytes);
    uint64_t* empty = full + 2;
    uint64_t* tfull = empty + 2;
    uint64_t* tempty = tfull + 2;
    uint64_t* wbar = tempty + 2;
    uint64_t* drain = wbar + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], 1);
            mbar_init(&tfull[k], 1);
            mbar_init(&tempty[k], 128);
        }
        mbar_init(wbar, 1);
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, kCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------------ producer
            mbar_arrive_expect_tx(wbar, (uint32_t)kWBytes);
            tma_load_3d(sw, &w_map, wbar, 0, 0, 0);
            int stage = 0;
            uint32_t phase = 0, issued = 0, issued_phase = 0;
            bool go = true;
            for (int u = blockIdx.x; go && u < n_units; u += gridDim.x) {
                const int b = u / nrb, y0 = (u - b * nrb) * R;
                for (int part = 0; part < (BWD ? 2 : 1); ++part) {   // BWD: the hi, then the lo term
                    if (!mbar_wait_bounded(&empty[stage], phase ^ 1, abort_flag, status, timeout_ns)) {
                        go = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[stage], 3 * copy_bytes);
                    const CUtensorMap* m = part == 0 ? &in_map : &in_map_lo;
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx)
                        tma_load_4d(sm + (size_t)(stage * 3 + kx) * cstride, m, &full[stage], 0, kx - 1, y0 - 1, b);
                    issued |= 1u << stage;
                    issued_phase = (issued_phase & ~(1u << stage)) | (phase << stage);
                    if (++stage == 2) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
            }
            if (*abort_flag) {   // copies of this thread still in flight must land before the CTA ends
                mbar_wait_bounded(wbar, 0, nullptr, nullptr, timeout_ns);
                for (int k = 0; k < 2; ++k)
                    if (issued & (1u << k)) mbar_wait_bounded(&full[k], (issued_phase >> k) & 1u, nullptr, nullptr, timeout_ns);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------------ MMA issuer
            constexpr uint32_t idesc = idesc_f32acc<true>(128, NOUT);
            bool ok = mbar_wait_bounded(wbar, 0, abort_flag, status, timeout_ns), any = false;
            int stage = 0, acc = 0;
            uint32_t phase = 0, acc_phase = 0;
            for (int u = blockIdx.x; ok && u < n_units; u += gridDim.x) {
                if (!mbar_wait_bounded(&tempty[acc], acc_phase ^ 1, abort_flag, status, timeout_ns)) {
                    ok = false;
                    break;
                }
                const uint32_t d0 = tmem_base + (uint32_t)(acc * 2 * NOUT);
                for (int part = 0; part < (BWD ? 2 : 1); ++part) {
                    if (!mbar_wait_bounded(&full[stage], phase, abort_flag, status, timeout_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int t = 0; t < 2; ++t)
#pragma unroll
                        for (int tap = 0; tap < 9; ++tap) {
                            const int ky = tap / 3, kx = tap % 3;
                            const uint64_t a = sdesc_kmajor_sw64(
                                smem_u32(sm + (size_t)(stage * 3 + kx) * cstride + (size_t)(ky * W + t * 128) * 64));
                            const uint64_t bd = sdesc_kmajor_sw64(smem_u32(sw + tap * NOUT * 64));
#pragma unroll
                            for (int h = 0; h < 2; ++h)   // second half of the 64-byte rows: +32 bytes
                                umma_f32<true>(d0 + (uint32_t)(t * NOUT), a + (uint64_t)(2 * h),
                                               bd + (uint64_t)(2 * h), idesc, (part | tap | h) ? 1u : 0u);
                        }
                    any = true;
                    umma_commit(&empty[stage]);
                    if (++stage == 2) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
                umma_commit(&tfull[acc]);
                if (++acc == 2) {
                    acc = 0;
                    acc_phase ^= 1;
                }
            }
            if (!ok && any) {   // the MMAs issued must finish before the tensor memory is freed
                umma_commit(drain);
                mbar_wait_bounded(drain, 0, nullptr, nullptr, timeout_ns);
            }
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int q = warp & 3;                                   // TMEM lane quarter
        const int64_t HW = (int64_t)H * W;
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
            const int b = u / nrb, y0 = (u - b * nrb) * R;
            if (!mbar_wait_bounded(&tfull[acc], acc_phase, abort_flag, status, timeout_ns)) break;
            tc_fence_after();
            const uint32_t d0 = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * 2 * NOUT);
#pragma unroll 1
            for (int t = 0; t < 2; ++t) {
                const int pl = t * 128 + 32 * q + lane;
                const int y = y0 + pl / W, x = pl - (pl / W) * W;
                if constexpr (kLast) {
                    uint32_t r[16];
                    tmem_ld_32x32b_x16(d0 + (uint32_t)(t * NOUT), r);
                    tmem_ld_wait();
                    if (y < H) {
                        const int64_t pix = (int64_t)y * W + x;
                        const float xcen = __bfloat162float(x0[((int64_t)b * 9 + 4) * HW + pix]);
                        y_out[(int64_t)b * HW + pix] = xcen + (__uint_as_float(r[0]) + __ldg(bias));
                    }
                    continue;
                }
                uint32_t r[32];
                tmem_ld_32x32b_x32(d0 + (uint32_t)(t * NOUT), r);
                tmem_ld_wait();
                if (y >= H) continue;
                const int64_t pix = (int64_t)y * W + x;
                if constexpr (BWD) {   // raw sums, channels-first float
#pragma unroll
                    for (int co = 0; co < 32; ++co) y_out[((int64_t)b * 32 + co) * HW + pix] = __uint_as_float(r[co]);
                } else {
                uint32_t pk[16];
#pragma unroll
                for (int co = 0; co < 32; co += 2) {
                    const __nv_bfloat16 v0 = __float2bfloat16_rn(fmaxf(__uint_as_float(r[co]) + __ldg(bias + co), 0.0f));
                    const __nv_bfloat16 v1 =
                        __float2bfloat16_rn(fmaxf(__uint_as_float(r[co + 1]) + __ldg(bias + co + 1), 0.0f));
                    if (out_cf != nullptr) {
                        out_cf[((int64_t)b * 32 + co) * HW + pix] = v0;
                        out_cf[((int64_t)b * 32 + co + 1) * HW + pix] = v1;
                    }
                    pk[co / 2] = (uint32_t)__bfloat16_as_ushort(v0) | ((uint32_t)__bfloat16_as_ushort(v1) << 16);
                }
                if (out_cl != nullptr) {
                    uint4* dst = reinterpret_cast<uint4*>(out_cl + ((int64_t)b * HW + pix) * 32);
#pragma unroll
                    for (int k = 0; k < 4; ++k) dst[k] = make_uint4(pk[4 * k], pk[4 * k + 1], pk[4 * k + 2], pk[4 * k + 3]);
                }
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty[acc]);
            if (++acc == 2) {
                acc = 0;
                acc_phase ^= 1;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kCols);
    }
}

// The stacked input in both layouts, one thread per (slice, pixel):
// x[b][c][p] = bf16(Gamma[nb(b, c)][p] * s) channels-first (9 channels) and
// channels-last with 32 channels (9..31 zero).
__global__ void dn_stack_both_kernel(const float* __restrict__ g, const float* __restrict__ scale, int hb, int wb,
                                     int64_t HW, int64_t n_pix, __nv_bfloat16* __restrict__ x,
                                     __nv_bfloat16* __restrict__ xc) {
    const float s = *scale;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pix; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / HW, p = i - b * HW;
        const int br = (int)(b / wb), bc = (int)(b - (int64_t)br * wb);
        uint32_t pk[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) pk[c] = 0u;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            const int r = br + c / 3 - 1, q = bc + c % 3 - 1;
            const bool in = r >= 0 && r < hb && q >= 0 && q < wb;
            const __nv_bfloat16 v = __float2bfloat16_rn(in ? g[(int64_t)(r * wb + q) * HW + p] * s : 0.0f);
            x[(b * 9 + c) * HW + p] = v;
            const uint32_t u = __bfloat16_as_ushort(v);
            pk[c / 2] |= (c & 1) ? (u << 16) : u;
        }
        uint4* dst = reinterpret_cast<uint4*>(xc + i * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
    }
}

// Weights of layers 0..2 as bf16 [layer][tap][Cout][Cin = 32] (layer 0: Cin 9,
// zero beyond), then the last layer as [tap][16][32] (output channel 0 of 16).
__global__ void dn_wprep_kernel(const float* __restrict__ model, int64_t w0, int64_t w1, int64_t w2, int64_t w3,
                                __nv_bfloat16* __restrict__ wt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * 9 * 32 * 32 + 9 * 16 * 32) return;
    if (i >= 3 * 9 * 32 * 32) {   // last layer: [tap][16][32], output channel 0 only
        const int rem = i - 3 * 9 * 32 * 32;
        const int tap = rem / (16 * 32), co = (rem / 32) % 16, ci = rem % 32;
        wt[i] = __float2bfloat16_rn(co == 0 ? model[w3 + (int64_t)ci * 9 + tap] : 0.0f);
        return;
    }
    const int l = i / (9 * 32 * 32), rem = i - l * 9 * 32 * 32;
    const int tap = rem / (32 * 32), co = (rem / 32) % 32, ci = rem % 32;
    const int cin = l == 0 ? 9 : 32;
    const int64_t base = l == 0 ? w0 : (l == 1 ? w1 : w2);
    wt[i] = __float2bfloat16_rn(ci < cin ? model[base + ((int64_t)co * cin + ci) * 9 + tap] : 0.0f);
}

// Weights of the input-gradient convolutions of layers 1 and 2 as bf16
// [layer - 1][tap][Cin][Cout]: tap t of the flipped kernel, W[co][ci][8 - t],
// output channel ci, input channel co.
__global__ void dn_wprep_bwd_kernel(const float* __restrict__ model, int64_t w1, int64_t w2,
                                    __nv_bfloat16* __restrict__ wt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * 9 * 32 * 32) return;
    const int l = i / (9 * 32 * 32), rem = i - l * 9 * 32 * 32;
    const int tap = rem / (32 * 32), ci = (rem / 32) % 32, co = rem % 32;
    const int64_t base = l == 0 ? w1 : w2;
    wt[i] = __float2bfloat16_rn(model[base + ((int64_t)co * 32 + ci) * 9 + (8 - tap)]);
}

// ------------------------------------------------------------------ weight gradients
// Partial gradient of one layer over slices [b0, b1): thread t < CIN * 9 owns
// (ci, tap) = (t / 9, t % 9) and all COUT output channels; threads t < COUT also
// sum the bias gradient.  d = gradient at the layer's output (masked by mask > 0
// when given), in = the layer's input (bf16).
template <int CIN, int COUT>
__global__ void __launch_bounds__(((CIN * 9 + 31) / 32) * 32)
    dn_wgrad_kernel(const __nv_bfloat16* __restrict__ in, const float* __restrict__ d,
                    const __nv_bfloat16* __restrict__ mask, int B, int H, int W, int slices_per_cta,
                    float* __restrict__ part) {
    constexpr int NT = ((CIN * 9 + 31) / 32) * 32;
    constexpr int TP = (kTH + 2) * (kTW + 2);
    extern __shared__ __align__(16) float sm[];
    float* sIn = sm;                              // [CIN][kTH + 2][kTW + 2]
    float* sD = sm + CIN * TP;                    // [kTH * kTW][COUT]
    const int tid = threadIdx.x;
    const bool owner = tid < CIN * 9;
    const int ci = tid / 9, tap = tid % 9, ky = tap / 3, kx = tap % 3;
    const int64_t HW = (int64_t)H * W;
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = 0.0f;
    float bacc = 0.0f;
    const int b0 = blockIdx.x * slices_per_cta, b1 = min(b0 + slices_per_cta, B);
    for (int b = b0; b < b1; ++b) {
        for (int y0 = 0; y0 < H; y0 += kTH) {
            for (int x0 = 0; x0 < W; x0 += kTW) {
                __syncthreads();   // previous tile consumed
                for (int i = tid; i < CIN * TP; i += NT) {
                    const int c = i / TP, rem = i - c * TP;
                    const int ty = rem / (kTW + 2), tx = rem - ty * (kTW + 2);
                    const int yy = y0 + ty - 1, xx = x0 + tx - 1;
                    float v = 0.0f;
                    if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                        v = __bfloat162float(in[((int64_t)b * CIN + c) * HW + (int64_t)yy * W + xx]);
                    sIn[i] = v;
                }
                for (int i = tid; i < kTH * kTW * COUT; i += NT) {
                    const int co = i / (kTH * kTW), p = i - co * (kTH * kTW);
                    const int yy = y0 + p / kTW, xx = x0 + p % kTW;
                    float v = 0.0f;
                    if (yy < H && xx < W) {
                        const int64_t idx = ((int64_t)b * COUT + co) * HW + (int64_t)yy * W + xx;
                        v = d[idx];
                        if (mask != nullptr && !(__bfloat162float(mask[idx]) > 0.0f)) v = 0.0f;
                    }
                    sD[p * COUT + co] = v;
                }
                __syncthreads();
                if (owner) {
#pragma unroll 4
                    for (int p = 0; p < kTH * kTW; ++p) {
                        const int py = p / kTW, px = p % kTW;
                        const float v = sIn[ci * TP + (py + ky) * (kTW + 2) + px + kx];
                        const float* dd = sD + p * COUT;
                        if constexpr (COUT % 4 == 0) {
#pragma unroll
                            for (int co = 0; co < COUT; co += 4) {
                                const float4 q = *reinterpret_cast<const float4*>(dd + co);
                                acc[co] = __fmaf_rn(q.x, v, acc[co]);
                                acc[co + 1] = __fmaf_rn(q.y, v, acc[co + 1]);
                                acc[co + 2] = __fmaf_rn(q.z, v, acc[co + 2]);
                                acc[co + 3] = __fmaf_rn(q.w, v, acc[co + 3]);
                            }
                        } else {
#pragma unroll
                            for (int co = 0; co < COUT; ++co) acc[co] = __fmaf_rn(dd[co], v, acc[co]);
                        }
                    }
                }
                if (tid < COUT)
                    for (int p = 0; p < kTH * kTW; ++p) bacc += sD[p * COUT + tid];
            }
        }
    }
    constexpr int NWB = COUT * CIN * 9 + COUT;
    float* out = part + (int64_t)blockIdx.x * NWB;
    if (owner)
#pragma unroll
        for (int co = 0; co < COUT; ++co) out[(co * CIN + ci) * 9 + tap] = acc[co];
    if (tid < COUT) out[COUT * CIN * 9 + tid] = bacc;
}

// ------------------------------------------------------------------ tensor-core weight gradients
// For images 64 pixels wide the weight gradient of a layer,
//     dW[co][ci][ky][kx] = sum over pixels of delta[co](y, x) in[ci](y + ky - 1, x + kx - 1),
// is a GEMM whose K dimension is the pixels.  delta (float32) is split into two
// bf16 terms, hi = bf16(delta) and lo = bf16(delta - hi) (the difference is exact
// in float32), so hi + lo is delta within 2^-17 and every product of a bf16 term
// with a bf16 input is exact in the FP32 accumulator.

// delta = d masked by mask > 0, as [slice][2 COUT][H * W] bf16 (hi channels
// 0 .. COUT-1, lo channels COUT .. 2 COUT-1) and, when cl_hi is given, also
// channels-last [slice][H * W][COUT] (the input of the tensor-core input-gradient
// convolution, staged in shared memory and stored as contiguous 16-byte words);
// per (slice, block of 256 pixels, channel) the sum of delta over the block's
// pixels (the bias gradient's terms: each warp in a fixed butterfly, then the
// warps in order).  CTA = (block of 256 pixels, slice), one pixel per thread.
constexpr int kSplitPix = 256;
template <int COUT>
__global__ void __launch_bounds__(256) dn_dsplit_kernel(const float* __restrict__ d,
                                                        const __nv_bfloat16* __restrict__ mask, int64_t HW,
                                                        __nv_bfloat16* __restrict__ out, __nv_bfloat16* __restrict__ cl_hi,
                                                        __nv_bfloat16* __restrict__ cl_lo, float* __restrict__ bpart) {
    constexpr int NW = COUT > 1 ? COUT / 2 : 1;                 // 32-bit words per pixel and term
    __shared__ float red[8][COUT];
    __shared__ __align__(16) uint32_t stage[2][COUT > 1 ? kSplitPix : 1][NW + (COUT > 1 ? 4 : 0)];
    const int b = blockIdx.y;
    const int64_t p0 = (int64_t)blockIdx.x * kSplitPix, p = p0 + threadIdx.x;
    const bool in = p < HW;
    // every channel's loads first (all in flight together), then the split
    float v[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) v[co] = in ? __ldg(d + ((int64_t)b * COUT + co) * HW + p) : 0.0f;
    if (mask != nullptr && in) {
        unsigned short m[COUT];
#pragma unroll
        for (int co = 0; co < COUT; ++co)
            m[co] = __ldg(reinterpret_cast<const unsigned short*>(mask) + ((int64_t)b * COUT + co) * HW + p);
#pragma unroll
        for (int co = 0; co < COUT; ++co)
            if (!(__uint_as_float((uint32_t)m[co] << 16) > 0.0f)) v[co] = 0.0f;
    }
#pragma unroll
    for (int co = 0; co < COUT; ++co) {
        if (in) {
            const __nv_bfloat16 hi = __float2bfloat16_rn(v[co]);
            const __nv_bfloat16 lo = __float2bfloat16_rn(v[co] - __bfloat162float(hi));
            out[((int64_t)b * 2 * COUT + co) * HW + p] = hi;
            out[((int64_t)b * 2 * COUT + COUT + co) * HW + p] = lo;
            if constexpr (COUT > 1) {
                reinterpret_cast<__nv_bfloat16*>(stage[0][threadIdx.x])[co] = hi;
                reinterpret_cast<__nv_bfloat16*>(stage[1][threadIdx.x])[co] = lo;
            }
        }
    }
    // bias terms: the warp's 32 pixels in a fixed butterfly, then the 8 warps in order
#pragma unroll
    for (int co = 0; co < COUT; ++co) {
        float t = v[co];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][co] = t;
    }
    __syncthreads();
    if constexpr (COUT > 1) {
        if (cl_hi != nullptr) {
            // the block's pixels are contiguous in the channels-last arrays: 16-byte words in order
            const int64_t npx = HW - p0 < kSplitPix ? HW - p0 : kSplitPix;
            constexpr int Q = NW / 4;                                  // 16-byte words per pixel
            for (int t = threadIdx.x; t < 2 * npx * Q; t += 256) {
                const int term = t / (int)(npx * Q), r = t - term * (int)(npx * Q);
                const int px = r / Q, q = r - px * Q;
                const uint4 w = *reinterpret_cast<const uint4*>(&stage[term][px][4 * q]);
                __nv_bfloat16* dst = term == 0 ? cl_hi : cl_lo;
                *reinterpret_cast<uint4*>(dst + ((int64_t)b * HW + p0 + px) * COUT + 8 * q) = w;
            }
        }
    }
    if (threadIdx.x < COUT) {
        float s = 0.0f;
        for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
        bpart[((int64_t)b * gridDim.x + blockIdx.x) * COUT + threadIdx.x] = s;
    }
}

// x-shifted copies of a layer input (bf16 [slice][CIN][H][W]) for the GEMM's B
// operand: out[slice][kx * CINP + c][y][x] = in[slice][c][y][x + kx - 1], zero
// outside the image and for c >= CIN.  One thread per (slice, c < CINP, y, group
// of 8 columns; W a multiple of 8): one 16-byte load, its two neighbours, three
// 16-byte stores.
template <int CIN, int CINP>
__global__ void __launch_bounds__(256) dn_shift3_kernel(const __nv_bfloat16* __restrict__ in, int B, int H, int W,
                                                        __nv_bfloat16* __restrict__ out) {
    const int64_t HW = (int64_t)H * W;
    const int G = W / 8;
    const int64_t n = (int64_t)B * CINP * H * G;
    const uint16_t* src = reinterpret_cast<const uint16_t*>(in);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int gx = (int)(i % G);
        const int64_t r = i / G;                 // (b, c, y)
        const int y = (int)(r % H);
        const int64_t bc = r / H;
        const int c = (int)(bc % CINP), b = (int)(bc / CINP);
        const int x0 = gx * 8;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        uint32_t left = 0u, right = 0u;
        if (c < CIN) {
            const int64_t row = ((int64_t)b * CIN + c) * HW + (int64_t)y * W;
            const uint4 v = *reinterpret_cast<const uint4*>(src + row + x0);
            w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
            if (x0 > 0) left = (uint32_t)src[row + x0 - 1] << 16;   // in the high half, as element 2q - 1 of a word
            if (x0 + 8 < W) right = src[row + x0 + 8];
        }
        // kx = 0: element j is in[x0 + j - 1]; kx = 2: in[x0 + j + 1]
        uint32_t s0[4], s2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t prev = q == 0 ? left : w[q - 1];
            const uint32_t next = q == 3 ? right : w[q + 1];
            s0[q] = __byte_perm(prev, w[q], 0x5432);   // (high half of prev, low half of w[q])
            s2[q] = __byte_perm(w[q], next, 0x5432);   // (high half of w[q], low half of next)
        }
        const int64_t o = (int64_t)b * 3 * CINP * HW + (int64_t)y * W + x0;
        *reinterpret_cast<uint4*>(out + o + (int64_t)c * HW) = make_uint4(s0[0], s0[1], s0[2], s0[3]);
        *reinterpret_cast<uint4*>(out + o + (int64_t)(CINP + c) * HW) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4*>(out + o + (int64_t)(2 * CINP + c) * HW) = make_uint4(s2[0], s2[1], s2[2], s2[3]);
    }
}

// The GEMM on tcgen05, persistent over units (slice, block of up to 32 rows).
// Per image row y of a unit, one stage holds A(y) = the 2 COUT delta rows of
// that image row (64 pixels, 128-byte rows, 128-byte swizzle; the tile's other
// rows up to M = 128 stay zero) and B(y) = the 3 CINP shifted input rows of
// image row y; rows y0 - 1 and y0 + R are loaded too (TMA zero fill outside
// the image).  For A(y) and each ky, one MMA with B(y + ky - 1) (N = 3 CINP)
// per 16 pixels adds into TMEM columns [ky * 3 CINP, (ky + 1) * 3 CINP): column
// ky * 3 CINP + kx * CINP + ci of row co is dW[co][ci][ky][kx] (rows >= COUT: the
// lo terms).  The accumulator spans all of the CTA's units; at the end the
// CTA writes its 2 COUT rows to part[cta].  Warp 0 (one thread) loads, warp 1
// (one thread) issues the MMAs and frees each stage once the MMAs that read it
// are done; all four warps drain the accumulator.  Every wait is bounded.
constexpr int kWgThreads = 128;
constexpr int kWgStages = 6;
constexpr int kWgRows = 32;
template <int CINP, int COUT>
struct WgCfg {
    static constexpr int kNB = 3 * CINP;                         // B rows per image row: 48 or 96
    static constexpr int kABytes = 128 * 128;                    // A tile, M = 128 rows of 128 bytes
    static constexpr uint32_t kALoad = 2 * COUT * 128;           // bytes of A the copies write
    static constexpr uint32_t kBBytes = kNB * 128;
    static constexpr int kStage = kABytes + (int)kBBytes;        // a multiple of 1024
    static constexpr uint32_t kCols = 9 * CINP;                  // accumulator columns: 144 or 288
    static constexpr uint32_t kTmemCols = kCols > 256 ? 512 : 256;
    static constexpr size_t kSmem = 1024 + (size_t)kWgStages * kStage + 256;
};

template <int CINP, int COUT>
__global__ void __launch_bounds__(kWgThreads, 1) dn_wgrad_tc_kernel(const __grid_constant__ CUtensorMap a_map,
                                                                    const __grid_constant__ CUtensorMap b_map, int H,
                                                                    int n_slices, float* __restrict__ part,
                                                                    unsigned int* status,
                                                                    unsigned long long timeout_ns) {
    using C = WgCfg<CINP, COUT>;
    constexpr int S = kWgStages;
    extern __shared__ uint8_t smem_wg[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_wg) + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + (size_t)S * C::kStage);
    uint64_t* empty = full + S;
    uint64_t* done = empty + S;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* any_flag = abort_flag + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R = H < kWgRows ? H : kWgRows;
    const int nrb = (H + R - 1) / R, n_units = nrb * n_slices;

    // rows 2 COUT .. 127 of every A tile stay zero (the copies write rows below)
    for (int s = 0; s < S; ++s) {
        uint4* a = reinterpret_cast<uint4*>(sm + (size_t)s * C::kStage + C::kALoad);
        for (int i = tid; i < (int)((C::kABytes - C::kALoad) / 16); i += kWgThreads) a[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    fence_proxy_async_smem();
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        *any_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, C::kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------- producer
        uint32_t g = 0;   // stage items issued
        bool ok = true;
        for (int u = blockIdx.x; ok && u < n_units; u += gridDim.x) {
            const int b = u / nrb, y0 = (u - b * nrb) * R;
            const int rows = min(R, H - y0);
            for (int k = 0; k <= rows + 1; ++k, ++g) {
                const int s = (int)(g % S);
                if (!mbar_wait_bounded(&empty[s], ((g / S) & 1u) ^ 1u, abort_flag, status, timeout_ns)) {
                    ok = false;
                    break;
                }
                const bool with_a = k >= 1 && k <= rows;
                mbar_arrive_expect_tx(&full[s], C::kBBytes + (with_a ? C::kALoad : 0u));
                uint8_t* st = sm + (size_t)s * C::kStage;
                tma_load_4d(st + C::kABytes, &b_map, &full[s], 0, 0, y0 - 1 + k, b);
                if (with_a) tma_load_4d(st, &a_map, &full[s], 0, 0, y0 - 1 + k, b);
            }
        }
        if (!ok)   // copies still in flight land before the CTA ends
            for (uint32_t j = g > (uint32_t)S ? g - S : 0u; j < g; ++j)
                mbar_wait_bounded(&full[j % S], (j / S) & 1u, nullptr, nullptr, timeout_ns);
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------------------- MMA issuer
        constexpr uint32_t idesc = idesc_f32acc<true>(128, C::kNB);
        uint32_t g = 0, waited = 0;
        bool ok = true, any = false;
        for (int u = blockIdx.x; ok && u < n_units; u += gridDim.x) {
            const int b = u / nrb, y0 = (u - b * nrb) * R;
            const int rows = min(R, H - y0);
            const uint32_t g0 = g;
            for (int k = 1; ok && k <= rows; ++k) {
                while (waited <= g0 + (uint32_t)k + 1u) {
                    if (!mbar_wait_bounded(&full[waited % S], (waited / S) & 1u, abort_flag, status, timeout_ns)) {
                        ok = false;
                        break;
                    }
                    ++waited;
                }
                if (!ok) break;
                tc_fence_after();
                const uint64_t ad = sdesc_kmajor_sw128(smem_u32(sm + (size_t)((g0 + k) % S) * C::kStage));
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)   // 16 pixels (32 bytes of each 128-byte row) per MMA
#pragma unroll
                    for (int ky = 0; ky < 3; ++ky) {
                        const uint32_t item = g0 + (uint32_t)(k - 1 + ky);
                        const uint64_t bd =
                            sdesc_kmajor_sw128(smem_u32(sm + (size_t)(item % S) * C::kStage + C::kABytes));
                        umma_f32<true>(tmem_base + (uint32_t)(ky * C::kNB), ad + (uint64_t)(2 * ks),
                                       bd + (uint64_t)(2 * ks), idesc, (any || ks > 0) ? 1u : 0u);
                    }
                any = true;
                umma_commit(&empty[(g0 + k - 1) % S]);
            }
            if (!ok) break;
            umma_commit(&empty[(g0 + rows) % S]);
            umma_commit(&empty[(g0 + rows + 1) % S]);
            g = g0 + rows + 2;
        }
        *any_flag = any ? 1 : 0;
        if (any) umma_commit(done);
        else mbar_arrive(done);
    }
    // ------------------------------------------------------------ all warps: drain
    __syncwarp();
    const bool fin = mbar_wait_bounded(done, 0, nullptr, status, timeout_ns);
    tc_fence_after();
    if (fin && !*abort_flag && 32 * warp < 2 * COUT) {
        const int row = 32 * warp + lane;
        float* out = part + ((size_t)blockIdx.x * 2 * COUT + row) * C::kCols;
        const bool any = *any_flag != 0;
#pragma unroll 1
        for (uint32_t c0 = 0; c0 < C::kCols; c0 += 16) {
            uint32_t r[16];
            if (any) {
                tmem_ld_32x32b_x16(tmem_base + ((uint32_t)(32 * warp) << 16) + c0, r);
                tmem_ld_wait();
            }
            if (row < 2 * COUT)
#pragma unroll
                for (int j = 0; j < 16; ++j) out[c0 + j] = any ? __uint_as_float(r[j]) : 0.0f;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, C::kTmemCols);
    }
}

// Bias gradient: CTA co sums bpart[i][co] over i, thread t the terms
// i = t, t + 256, ... in order, then the threads in a fixed tree.
template <int COUT>
__global__ void __launch_bounds__(256) dn_bias_reduce_kernel(const float* __restrict__ bpart, int nb,
                                                             float* __restrict__ grad_bias) {
    __shared__ float red[256];
    const int co = blockIdx.x;
    float s = 0.0f;
    for (int i = threadIdx.x; i < nb; i += 256) s += bpart[(size_t)i * COUT + co];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) grad_bias[co] = red[0];
}

// dW[co][ci][tap] = sum over CTAs in order of the hi and lo rows of column
// tap * CINP + ci (the bias gradient: dn_bias_reduce_kernel).
template <int CIN, int CINP, int COUT>
__global__ void dn_wgrad_tc_reduce_kernel(const float* __restrict__ part, int nparts, float* __restrict__ grad) {
    constexpr int kCols = 9 * CINP;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= COUT * CIN * 9) return;
    const int co = k / (CIN * 9), ci = (k / 9) % CIN, tap = k % 9;
    const int col = tap * CINP + ci;
    float s = 0.0f;
    for (int i = 0; i < nparts; ++i) {
        const float* p = part + (size_t)i * 2 * COUT * kCols;
        s += p[(size_t)co * kCols + col] + p[(size_t)(COUT + co) * kCols + col];
    }
    grad[k] = s;
}

// grad[k] = sum over CTAs of part[cta][k], CTAs in order
__global__ void dn_reduce_parts_kernel(const float* __restrict__ part, int nparts, int n, float* __restrict__ grad) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float s = 0.0f;
    for (int i = 0; i < nparts; ++i) s += part[(int64_t)i * n + k];
    grad[k] = s;
}

// ------------------------------------------------------------------ loss
// dY = 2 (y - s t) / count; per-block sums of (y - s t)^2 in float64.
__global__ void dn_mse_kernel(const float* __restrict__ y, const float* __restrict__ t,
                              const float* __restrict__ scale, int64_t n, float* __restrict__ dy,
                              double* __restrict__ part) {
    __shared__ double red[256];
    const float s = *scale;
    const float inv = 2.0f / (float)n;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = y[i] - t[i] * s;
        dy[i] = e * inv;
        acc += (double)e * (double)e;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void dn_loss_kernel(const double* __restrict__ part, int nparts, int64_t n, float* __restrict__ loss) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t = 0.0;
    for (int i = 0; i < nparts; ++i) t += part[i];
    *loss = (float)(t / (double)n);
}

// out[i] = y[i] / s
__global__ void dn_unscale_kernel(const float* __restrict__ y, const float* __restrict__ scale, int64_t n,
                                  float* __restrict__ out) {
    const float s = *scale;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = y[i] / s;
}

// ------------------------------------------------------------------ Adam
// b1, b2 and their complements 1 - b1, 1 - b2 come rounded separately (1 - 0.999f
// in float32 is 1.3e-5 away from 0.001).
__global__ void dn_adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                               const float* __restrict__ g, int n, float lr, float b1, float omb1, float b2,
                               float omb2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + omb1 * gi;
    const float vi = b2 * v[i] + omb2 * (gi * gi);
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

template <int CIN, int COUT, int MODE>
cudaError_t conv(const void* in, const __nv_bfloat16* mask, const float* w, const float* bias,
                 const __nv_bfloat16* x0, void* out, int B, int H, int W, cudaStream_t st) {
    const size_t smem = sizeof(float) * ((size_t)CIN * (kTH + 2) * (kTW + 2) + (size_t)CIN * 9 * COUT);
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        e = cudaFuncSetAttribute(dn_conv_kernel<CIN, COUT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    dim3 grid((unsigned)((W + kTW - 1) / kTW), (unsigned)((H + kTH - 1) / kTH), (unsigned)B);
    dn_conv_kernel<CIN, COUT, MODE><<<grid, kConvThreads, smem, st>>>(in, mask, w, bias, x0, out, H, W);
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t wgrad(const __nv_bfloat16* in, const float* d, const __nv_bfloat16* mask, int B, int H, int W,
                  int nparts, float* part, float* grad, cudaStream_t st) {
    constexpr int NT = ((CIN * 9 + 31) / 32) * 32;
    const size_t smem = sizeof(float) * ((size_t)CIN * (kTH + 2) * (kTW + 2) + (size_t)kTH * kTW * COUT);
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        e = cudaFuncSetAttribute(dn_wgrad_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    const int per = (B + nparts - 1) / nparts;
    const int used = (B + per - 1) / per;
    dn_wgrad_kernel<CIN, COUT><<<used, NT, smem, st>>>(in, d, mask, B, H, W, per, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    constexpr int n = COUT * CIN * 9 + COUT;
    dn_reduce_parts_kernel<<<(n + 255) / 256, 256, 0, st>>>(part, used, n, grad);
    return cudaGetLastError();
}

// Input gradient of a hidden layer on the tensor cores: g = conv(delta_hi +
// delta_lo; flipped weights wt [tap][32][32]), FP32 channels-first.
cudaError_t conv_tc_bwd(const __nv_bfloat16* d_hi, const __nv_bfloat16* d_lo, const __nv_bfloat16* wt, float* g,
                        int B, int H, int W, int sm_count, unsigned int* status, unsigned long long timeout_ns,
                        cudaStream_t st) {
    const int64_t HW = (int64_t)H * W;
    const int R = tc_rows(W);
    const uint64_t dims[4] = {32, (uint64_t)W, (uint64_t)H, (uint64_t)B};
    const uint64_t str[3] = {64, (uint64_t)W * 64, (uint64_t)HW * 64};
    const uint32_t box[4] = {32, (uint32_t)W, (uint32_t)(R + 2), 1};
    const uint64_t wdims[3] = {32, 32, 9}, wstr[2] = {64, 64 * 32};
    const uint32_t wbox[3] = {32, 32, 9};
    CUtensorMap hi_map, lo_map, w_map;
    if (!make_bf16_map_sw64(&hi_map, d_hi, 4, dims, str, box) || !make_bf16_map_sw64(&lo_map, d_lo, 4, dims, str, box) ||
        !make_bf16_map_sw64(&w_map, wt, 3, wdims, wstr, wbox))
        return cudaErrorInvalidValue;
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const size_t smem = tc_smem(W);
    if (!attr[dev]) {
        const int smax = (int)(tc_smem(32) > tc_smem(128) ? tc_smem(32) : tc_smem(128));
        e = cudaFuncSetAttribute(dn_conv_tc_kernel<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    const int64_t units = (int64_t)((H + R - 1) / R) * B;
    const unsigned grid = (unsigned)(units < sm_count ? units : sm_count);
    dn_conv_tc_kernel<32, true><<<grid, kTcThreadsP, smem, st>>>(hi_map, lo_map, w_map, nullptr, nullptr, nullptr,
                                                                 nullptr, g, H, W, B, status, timeout_ns);
    return cudaGetLastError();
}

// Weight gradient of one layer on the tensor cores (images 64 pixels wide):
// delta split, shifted input copies, the GEMM, the fixed-order reduction.
struct WgBuffers {
    __nv_bfloat16* dsplit;
    __nv_bfloat16* cl_hi;   // channels-last split of delta (null: not wanted)
    __nv_bfloat16* cl_lo;
    __nv_bfloat16* shifted;
    float* part;
    float* bpart;
};
template <int CIN, int CINP, int COUT>
cudaError_t wgrad_tc(const __nv_bfloat16* in, const float* d, const __nv_bfloat16* mask, int B, int H, int W,
                     const WgBuffers& wb, float* grad, int sm_count, unsigned int* status,
                     unsigned long long timeout_ns, cudaStream_t st) {
    using C = WgCfg<CINP, COUT>;
    if (W != 64) return cudaErrorInvalidValue;
    const int64_t HW = (int64_t)H * W;
    const int nblk = (int)((HW + kSplitPix - 1) / kSplitPix);
    dn_dsplit_kernel<COUT><<<dim3((unsigned)nblk, (unsigned)B), 256, 0, st>>>(d, mask, HW, wb.dsplit, wb.cl_hi,
                                                                               wb.cl_lo, wb.bpart);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nshift = (int64_t)B * CINP * HW / 8;
    const int64_t sblocks = (nshift + 255) / 256 < 8 * (int64_t)sm_count ? (nshift + 255) / 256 : 8 * (int64_t)sm_count;
    dn_shift3_kernel<CIN, CINP><<<(unsigned)sblocks, 256, 0, st>>>(in, B, H, W, wb.shifted);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    CUtensorMap amap, bmap;
    const uint64_t adims[4] = {(uint64_t)W, (uint64_t)(2 * COUT), (uint64_t)H, (uint64_t)B};
    const uint64_t astr[3] = {(uint64_t)HW * 2, (uint64_t)W * 2, (uint64_t)(2 * COUT) * HW * 2};
    const uint32_t abox[4] = {64, (uint32_t)(2 * COUT), 1, 1};
    const uint64_t bdims[4] = {(uint64_t)W, (uint64_t)C::kNB, (uint64_t)H, (uint64_t)B};
    const uint64_t bstr[3] = {(uint64_t)HW * 2, (uint64_t)W * 2, (uint64_t)C::kNB * HW * 2};
    const uint32_t bbox[4] = {64, (uint32_t)C::kNB, 1, 1};
    if (!make_bf16_map_sw128(&amap, wb.dsplit, 4, adims, astr, abox) ||
        !make_bf16_map_sw128(&bmap, wb.shifted, 4, bdims, bstr, bbox))
        return cudaErrorInvalidValue;
    static bool attr[64] = {};
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        e = cudaFuncSetAttribute(dn_wgrad_tc_kernel<CINP, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)C::kSmem);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    const int R = H < kWgRows ? H : kWgRows;
    const int64_t units = (int64_t)B * ((H + R - 1) / R);
    int grid = sm_count < kWgMaxCtas ? sm_count : kWgMaxCtas;
    if (units < grid) grid = (int)units;
    dn_wgrad_tc_kernel<CINP, COUT><<<grid, kWgThreads, C::kSmem, st>>>(amap, bmap, H, B, wb.part, status, timeout_ns);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    constexpr int n = COUT * CIN * 9;
    dn_wgrad_tc_reduce_kernel<CIN, CINP, COUT><<<(n + 255) / 256, 256, 0, st>>>(wb.part, grid, grad);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dn_bias_reduce_kernel<COUT><<<COUT, 256, 0, st>>>(wb.bpart, B * nblk, grad + n);
    return cudaGetLastError();
}

}  // namespace

// Parameter offsets in the model blob.
constexpr int64_t kW0 = 0, kB0 = kW0 + 32 * 9 * 9, kW1 = kB0 + 32, kB1 = kW1 + 32 * 32 * 9, kW2 = kB1 + 32,
                  kB2 = kW2 + 32 * 32 * 9, kW3 = kB2 + 32, kB3 = kW3 + 32 * 9;
static_assert(kB3 + 1 == kDenoiserParams, "model blob layout");

DenoiseLayout denoise_layout(int ha, int wa, int hb, int wb, bool training) {
    DenoiseLayout L{};
    const int64_t B = (int64_t)hb * wb, HW = (int64_t)ha * wa;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 255) / 256 * 256;
        return at;
    };
    L.scale = take(sizeof(float));
    L.sums = take(sizeof(double) * kSumBlocks);
    L.x0 = take(2 * (size_t)(B * 9 * HW));
    L.a1 = take(2 * (size_t)(B * 32 * HW));
    L.a2 = take(2 * (size_t)(B * 32 * HW));
    L.a3 = take(2 * (size_t)(B * 32 * HW));
    L.y = take(4 * (size_t)(B * HW));
    L.tc = (wa == 32 || wa == 64 || wa == 128) && B <= 65535 ? 1 : 0;
    if (L.tc) {
        L.xc = take(64 * (size_t)(B * HW));
        L.c1 = take(64 * (size_t)(B * HW));
        L.c2 = take(64 * (size_t)(B * HW));
        L.wt = take(2 * (size_t)(3 * 9 * 32 * 32 + 9 * 16 * 32));
    }
    if (training) {
        L.dy = take(4 * (size_t)(B * HW));
        L.d_hi = take(4 * (size_t)(B * 32 * HW));
        L.d_lo = take(4 * (size_t)(B * 32 * HW));
        L.part = take(sizeof(float) * (size_t)kDenoiseParts * (32 * 32 * 9 + 32));
        L.wg = wa == 64 && B <= 65535 ? 1 : 0;
        if (L.wg) {
            L.dsplit = take(2 * (size_t)(B * 64 * HW));
            L.shifted = take(2 * (size_t)(B * 96 * HW));
            L.wgpart = take(sizeof(float) * (size_t)kWgMaxCtas * 64 * 288);
            L.bpart = take(sizeof(float) * (size_t)B * ((HW + 255) / 256) * 32);
            L.dcl_hi = take(2 * (size_t)(B * 32 * HW));
            L.dcl_lo = take(2 * (size_t)(B * 32 * HW));
            L.wtb = take(2 * (size_t)(2 * 9 * 32 * 32));
        }
    }
    L.bytes = o;
    return L;
}

namespace {
// The network on the tensor cores (scale already known): stacked input in both
// layouts, layers 0..2 (a1, a2, a3 channels-first for the backward pass when
// keep_cf; channels-last copies for the next layer, layer 2's into the input's
// buffer) and the last layer into y.
cudaError_t forward_tc(const float* model, const float* gamma_in, const float* scale, int ha, int wa, int hb,
                       int wb, uint8_t* ws, const DenoiseLayout& L, bool keep_cf, unsigned int* status,
                       unsigned long long timeout_ns, cudaStream_t st) {
    const int B = hb * wb;
    const int64_t HW = (int64_t)ha * wa;
    auto* x0 = reinterpret_cast<__nv_bfloat16*>(ws + L.x0);
    auto* xc = reinterpret_cast<__nv_bfloat16*>(ws + L.xc);
    auto* c1 = reinterpret_cast<__nv_bfloat16*>(ws + L.c1);
    auto* c2 = reinterpret_cast<__nv_bfloat16*>(ws + L.c2);
    auto* wt = reinterpret_cast<__nv_bfloat16*>(ws + L.wt);
    float* y = reinterpret_cast<float*>(ws + L.y);
    __nv_bfloat16* acf[3] = {keep_cf ? reinterpret_cast<__nv_bfloat16*>(ws + L.a1) : nullptr,
                             keep_cf ? reinterpret_cast<__nv_bfloat16*>(ws + L.a2) : nullptr,
                             keep_cf ? reinterpret_cast<__nv_bfloat16*>(ws + L.a3) : nullptr};
    const __nv_bfloat16* ins[4] = {xc, c1, c2, xc};
    __nv_bfloat16* outs_cl[3] = {c1, c2, xc};
    const float* biases[4] = {model + kB0, model + kB1, model + kB2, model + kB3};
    const int64_t n_pix = (int64_t)B * HW;
    dn_stack_both_kernel<<<(unsigned)((n_pix + 255) / 256 < 4096 ? (n_pix + 255) / 256 : 4096), 256, 0, st>>>(
        gamma_in, scale, hb, wb, HW, n_pix, x0, xc);
    dn_wprep_kernel<<<(3 * 9 * 32 * 32 + 9 * 16 * 32 + 255) / 256, 256, 0, st>>>(model, kW0, kW1, kW2, kW3, wt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    static bool attr[64] = {};
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const int smax = (int)(tc_smem(32) > tc_smem(128) ? tc_smem(32) : tc_smem(128));
    if (!attr[dev]) {
        if ((e = cudaFuncSetAttribute(dn_conv_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax)) !=
                cudaSuccess ||
            (e = cudaFuncSetAttribute(dn_conv_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax)) !=
                cudaSuccess)
            return e;
        attr[dev] = true;
    }
    const size_t smem = tc_smem(wa);
    const int R = tc_rows(wa);
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int64_t units = (int64_t)((ha + R - 1) / R) * B;
    const dim3 grid((unsigned)(units < sms ? units : sms));
    const uint64_t dims[4] = {32, (uint64_t)wa, (uint64_t)ha, (uint64_t)B};
    const uint64_t str[3] = {64, (uint64_t)wa * 64, (uint64_t)HW * 64};
    const uint32_t box[4] = {32, (uint32_t)wa, (uint32_t)(R + 2), 1};
    for (int l = 0; l < 4; ++l) {
        const int nout = l < 3 ? 32 : 16;
        const uint64_t wdims[3] = {32, (uint64_t)nout, 9}, wstr[2] = {64, 64 * (uint64_t)nout};
        const uint32_t wbox[3] = {32, (uint32_t)nout, 9};
        CUtensorMap in_map, w_map;
        if (!make_bf16_map_sw64(&in_map, ins[l], 4, dims, str, box) ||
            !make_bf16_map_sw64(&w_map, wt + (size_t)l * 9 * 32 * 32, 3, wdims, wstr, wbox))
            return cudaErrorInvalidValue;
        if (l < 3)
            dn_conv_tc_kernel<32><<<grid, kTcThreadsP, smem, st>>>(in_map, in_map, w_map, biases[l], acf[l], outs_cl[l],
                                                                   nullptr, nullptr, ha, wa, B, status, timeout_ns);
        else
            dn_conv_tc_kernel<16><<<grid, kTcThreadsP, smem, st>>>(in_map, in_map, w_map, biases[l], nullptr, nullptr, x0, y,
                                                                   ha, wa, B, status, timeout_ns);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}
}  // namespace

cudaError_t denoise_forward(const float* model, const float* gamma_in, int ha, int wa, int hb, int wb,
                            uint8_t* ws, const DenoiseLayout& L, bool keep_cf, unsigned int* status,
                            unsigned long long timeout_ns, cudaStream_t st) {
    const int B = hb * wb;
    const int64_t HW = (int64_t)ha * wa, n = (int64_t)B * HW;
    float* scale = reinterpret_cast<float*>(ws + L.scale);
    double* sums = reinterpret_cast<double*>(ws + L.sums);
    auto* x0 = reinterpret_cast<__nv_bfloat16*>(ws + L.x0);
    auto* a1 = reinterpret_cast<__nv_bfloat16*>(ws + L.a1);
    auto* a2 = reinterpret_cast<__nv_bfloat16*>(ws + L.a2);
    auto* a3 = reinterpret_cast<__nv_bfloat16*>(ws + L.a3);
    float* y = reinterpret_cast<float*>(ws + L.y);
    dn_sumsq_kernel<<<kSumBlocks, 256, 0, st>>>(gamma_in, n, sums);
    dn_scale_kernel<<<1, 32, 0, st>>>(sums, kSumBlocks, n, scale);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (L.tc) return forward_tc(model, gamma_in, scale, ha, wa, hb, wb, ws, L, keep_cf, status, timeout_ns, st);
    dn_stack_kernel<<<dim3((unsigned)((HW + 255) / 256 < 64 ? (HW + 255) / 256 : 64), 9, (unsigned)B), 256, 0, st>>>(
        gamma_in, scale, hb, wb, HW, x0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = conv<9, 32, kFwdHidden>(x0, nullptr, model + kW0, model + kB0, nullptr, a1, B, ha, wa, st)) != cudaSuccess) return e;
    if ((e = conv<32, 32, kFwdHidden>(a1, nullptr, model + kW1, model + kB1, nullptr, a2, B, ha, wa, st)) != cudaSuccess) return e;
    if ((e = conv<32, 32, kFwdHidden>(a2, nullptr, model + kW2, model + kB2, nullptr, a3, B, ha, wa, st)) != cudaSuccess) return e;
    return conv<32, 1, kFwdLast>(a3, nullptr, model + kW3, model + kB3, x0, y, B, ha, wa, st);
}

cudaError_t denoise_output(const uint8_t* ws, const DenoiseLayout& L, int64_t n, float* gamma_out, cudaStream_t st) {
    dn_unscale_kernel<<<1024, 256, 0, st>>>(reinterpret_cast<const float*>(ws + L.y),
                                            reinterpret_cast<const float*>(ws + L.scale), n, gamma_out);
    return cudaGetLastError();
}

cudaError_t denoise_backward(const float* model, const float* gamma_target, int ha, int wa, int hb, int wb,
                             uint8_t* ws, const DenoiseLayout& L, float* grad, float* loss, int sm_count,
                             unsigned int* status, unsigned long long timeout_ns, cudaStream_t st) {
    const int B = hb * wb;
    const int64_t HW = (int64_t)ha * wa, n = (int64_t)B * HW;
    const float* scale = reinterpret_cast<const float*>(ws + L.scale);
    double* sums = reinterpret_cast<double*>(ws + L.sums);
    auto* x0 = reinterpret_cast<const __nv_bfloat16*>(ws + L.x0);
    auto* a1 = reinterpret_cast<const __nv_bfloat16*>(ws + L.a1);
    auto* a2 = reinterpret_cast<const __nv_bfloat16*>(ws + L.a2);
    auto* a3 = reinterpret_cast<const __nv_bfloat16*>(ws + L.a3);
    const float* y = reinterpret_cast<const float*>(ws + L.y);
    float* dy = reinterpret_cast<float*>(ws + L.dy);
    float* dhi = reinterpret_cast<float*>(ws + L.d_hi);
    float* dlo = reinterpret_cast<float*>(ws + L.d_lo);
    float* part = reinterpret_cast<float*>(ws + L.part);
    dn_mse_kernel<<<kSumBlocks, 256, 0, st>>>(y, gamma_target, scale, n, dy, sums);
    dn_loss_kernel<<<1, 32, 0, st>>>(sums, kSumBlocks, n, loss);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    WgBuffers wgb{L.wg ? reinterpret_cast<__nv_bfloat16*>(ws + L.dsplit) : nullptr, nullptr, nullptr,
                  L.wg ? reinterpret_cast<__nv_bfloat16*>(ws + L.shifted) : nullptr,
                  L.wg ? reinterpret_cast<float*>(ws + L.wgpart) : nullptr,
                  L.wg ? reinterpret_cast<float*>(ws + L.bpart) : nullptr};
    __nv_bfloat16* dcl_hi = L.wg ? reinterpret_cast<__nv_bfloat16*>(ws + L.dcl_hi) : nullptr;
    __nv_bfloat16* dcl_lo = L.wg ? reinterpret_cast<__nv_bfloat16*>(ws + L.dcl_lo) : nullptr;
    __nv_bfloat16* wtb = L.wg ? reinterpret_cast<__nv_bfloat16*>(ws + L.wtb) : nullptr;
    if (L.wg) {
        dn_wprep_bwd_kernel<<<(2 * 9 * 32 * 32 + 255) / 256, 256, 0, st>>>(model, kW1, kW2, wtb);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // layer 3 (32 -> 1): d at its output = dy
    if (L.wg) e = wgrad_tc<32, 32, 1>(a3, dy, nullptr, B, ha, wa, wgb, grad + kW3, sm_count, status, timeout_ns, st);
    else e = wgrad<32, 1>(a3, dy, nullptr, B, ha, wa, kDenoiseParts, part, grad + kW3, st);
    if (e != cudaSuccess) return e;
    if ((e = conv<1, 32, kBwdData>(dy, nullptr, model + kW3, nullptr, nullptr, dhi, B, ha, wa, st)) != cudaSuccess) return e;
    // layer 2: d at its output = dhi masked by a3
    if (L.wg) {   // the split of delta also feeds the tensor-core input gradient
        wgb.cl_hi = dcl_hi;
        wgb.cl_lo = dcl_lo;
        e = wgrad_tc<32, 32, 32>(a2, dhi, a3, B, ha, wa, wgb, grad + kW2, sm_count, status, timeout_ns, st);
        if (e == cudaSuccess)
            e = conv_tc_bwd(dcl_hi, dcl_lo, wtb + 9 * 32 * 32, dlo, B, ha, wa, sm_count, status, timeout_ns, st);
    } else {
        e = wgrad<32, 32>(a2, dhi, a3, B, ha, wa, kDenoiseParts, part, grad + kW2, st);
        if (e == cudaSuccess) e = conv<32, 32, kBwdData>(dhi, a3, model + kW2, nullptr, nullptr, dlo, B, ha, wa, st);
    }
    if (e != cudaSuccess) return e;
    // layer 1: d at its output = dlo masked by a2
    if (L.wg) {
        e = wgrad_tc<32, 32, 32>(a1, dlo, a2, B, ha, wa, wgb, grad + kW1, sm_count, status, timeout_ns, st);
        if (e == cudaSuccess) e = conv_tc_bwd(dcl_hi, dcl_lo, wtb, dhi, B, ha, wa, sm_count, status, timeout_ns, st);
        wgb.cl_hi = wgb.cl_lo = nullptr;
    } else {
        e = wgrad<32, 32>(a1, dlo, a2, B, ha, wa, kDenoiseParts, part, grad + kW1, st);
        if (e == cudaSuccess) e = conv<32, 32, kBwdData>(dlo, a2, model + kW1, nullptr, nullptr, dhi, B, ha, wa, st);
    }
    if (e != cudaSuccess) return e;
    // layer 0: d at its output = dhi masked by a1
    if (L.wg) return wgrad_tc<9, 16, 32>(x0, dhi, a1, B, ha, wa, wgb, grad + kW0, sm_count, status, timeout_ns, st);
    return wgrad<9, 32>(x0, dhi, a1, B, ha, wa, kDenoiseParts, part, grad + kW0, st);
}

cudaError_t denoise_adam(float* model, float* m, float* v, const float* grad, int64_t step, float lr,
                         cudaStream_t st) {
    const float c1 = (float)(1.0 - pow(0.9, (double)step)), c2 = (float)(1.0 - pow(0.999, (double)step));
    dn_adam_kernel<<<(kDenoiserParams + 255) / 256, 256, 0, st>>>(model, m, v, grad, kDenoiserParams, lr, 0.9f, 0.1f,
                                                                    0.999f, 0.001f, 1e-8f, c1, c2);
    return cudaGetLastError();
}

}  // namespace cpi
