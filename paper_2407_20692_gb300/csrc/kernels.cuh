// Host-side declarations shared by the library's translation units: kernel
// parameter blocks and launchers.  Nothing here is part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "gamma_div.cuh"

namespace cpi {

// Status bits recorded by kernels in the per-device status word.
constexpr unsigned int kStatusTimeoutBit = 1u;

// One detector image's frames as the kernels see them (validated copy of cpi_frames).
struct FramesDev {
    const uint8_t* data;
    int32_t bits, height, width, x0, y0;
    int64_t row_stride, frame_stride;
    int32_t bit_order;
};

// ------------------------------------------------------------------ ingest
// Frames -> K-major tensor-core operands [M][kstride] and marginal sums.
// kBf16: values as BF16 (any bit depth); else 1-bit values as FP4 E2M1, two per byte.
constexpr int kIngestPixels = 32;                 // pixels per CTA
constexpr int kIngestRowBytes = 256;              // BF16 operand bytes per pixel per CTA (E2M1: half)
inline int ingest_frames_per_cta(bool bf16) { return bf16 ? 128 : 256; }

// vmax (BF16 path, may be null): the largest A and B value seen is raised into
// vmax[0] and vmax[1] (the caller zeroes them first).
cudaError_t launch_ingest(bool bf16, const FramesDev& a, const FramesDev& b, int64_t n_frames,
                          int64_t kstride_bytes, uint8_t* op_a, uint8_t* op_b, int64_t* s_a,
                          int64_t* s_b, uint32_t* vmax, cudaStream_t st);

// ------------------------------------------------------------------ moments
// One raw-moment problem: S_ab of one (A, B) pair, split into work units of
// (frame chunk, 128 x BLOCK_N output tile).
struct MomentsProblem {
    int32_t* partial;        // [n_chunks][M][N] exact partial sums (uint32 bit patterns)
    int32_t M, N;            // A pixels (rows), B pixels (columns)
    int32_t k_blocks;        // K blocks of 128 bytes per operand row
    int32_t kb_per_chunk;    // K blocks per frame chunk (one partial slot each)
    int32_t n_chunks, tiles_m, tiles_n;
    int32_t unit_begin;      // first unit of this problem in the launch
    const uint32_t* vmax;    // BF16 path: largest A and B value of the call's frames (written by
                             // ingest), which set the exact FP32 segment length
    int32_t add_partial;     // 1: add the sums into the partial slots (uint32, wrapping never
                             // reached: binary frames, fewer than 2^32 per slot) instead of storing
};

// A persistent launch over the units of up to K problems (K = 1 for a single
// correlation, kMaxGroup for a batch).  Passed as a __grid_constant__ kernel
// parameter, so the TMA descriptors live in parameter space.
constexpr int kMaxGroup = 64;
template <int K>
struct MomentsLaunch {
    CUtensorMap map_a[K];
    CUtensorMap map_b[K];
    MomentsProblem prob[K];
    int32_t n_problems, n_units;
    unsigned int* status;
    unsigned long long timeout_ns;
};

struct MomentsShape {
    int block_n;             // N tile
    int k_per_block;         // elements per K block (128 bytes)
    int stages;
    size_t smem_bytes;
};
// block_n: the output tile's width, 256 (single correlations) or 128.
MomentsShape moments_shape(bool bf16, int block_n = 256);

cudaError_t launch_moments(bool bf16, int block_n, const MomentsLaunch<1>& L, int sm_count, cudaStream_t st);
cudaError_t launch_moments_group(bool bf16, int block_n, const MomentsLaunch<kMaxGroup>& L, int sm_count,
                                 cudaStream_t st);

// ------------------------------------------------------------------ fold / finalize
cudaError_t launch_fold(const int32_t* partial, int n_chunks, int64_t M, int64_t N,
                        int64_t* s_ab, int accumulate, int write_sab, const int64_t* s_a,
                        const int64_t* s_b, int64_t n_frames, double* gamma, float* gamma_f32,
                        cudaStream_t st, int wide = 0);
// wide != 0: the numerator N S_ab - S_a S_b is formed in 128 bits (sums from
// accumulating calls, which the per-call overflow check does not bound).

// ------------------------------------------------------------------ refocus
constexpr int kRefocusMaxPlanesPerLaunch = 128;
struct PlaneBlock {
    double alpha[kRefocusMaxPlanesPerLaunch];
    double beta[kRefocusMaxPlanesPerLaunch];
};
// Planes with |alpha| or |beta| above this are rejected (coordinates are formed
// in 32.32 fixed point).
constexpr double kRefocusMaxCoef = 1.0e6;
// Shapes the refocusing kernels take: wa <= 512 and hb small enough for the y
// taps of one output row to fit a CTA (hb <= 12800).
bool refocus_supported(int ha, int wa, int hb, int wb);
// Workspace bytes: the x-stage images of up to kRefocusMaxPlanesPerLaunch planes
// ([planes][hb][ha][wa] floats), plus a row-padded copy of Gamma when its rows
// do not meet the staging alignment.  0 if unsupported.
size_t refocus_ws_bytes(int ha, int wa, int hb, int wb, int n_planes);
// Kernel launches of one refocusing call.
int refocus_launches(int ha, int wa, int n_planes);
// Whole refocusing of gamma_f32 (slice-major [hb*wb][ha*wa]) into out
// ([n_planes][ha][wa]); alpha, beta: host arrays of n_planes coefficients.
cudaError_t refocus_run(const float* gamma_f32, int ha, int wa, int hb, int wb, const double* alpha,
                        const double* beta, int n_planes, float* out, void* workspace, int sm_count,
                        unsigned int* status, unsigned long long timeout_ns, cudaStream_t st);
// Tiled tensor map over a float32 array of rank 2 or 3 (no swizzle); dims
// innermost first, strides in bytes for dims 1..rank-1.  False if the driver
// rejects it.
bool make_f32_map(CUtensorMap* m, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                  const uint32_t* box);

// ------------------------------------------------------------------ 4-D refocus
constexpr int kRefocus4dChunk = 64;        // planes per launch chunk (at most)
struct Plane4Block {
    double c[kRefocus4dChunk][4];          // alpha, beta, gamma, delta
};
struct Refocus4dLayout {                   // byte offsets in the workspace
    int chunk;                             // planes per chunk
    int64_t stride;                        // elements per coordinate table
    size_t tables, c_hi, c_lo, bytes;
};
Refocus4dLayout refocus4d_layout(int ha, int wa, int hb, int wb, int n_planes);
bool refocus4d_box_fits(int wa, int wb);
// planes of one chunk (np <= layout.chunk); out = [np][ha][wa]
cudaError_t launch_refocus4d_chunk(const float* gamma_f32, int ha, int wa, int hb, int wb, const Plane4Block& coef,
                                   int np, uint8_t* ws, const Refocus4dLayout& L, float* out, cudaStream_t st);

// ------------------------------------------------------------------ denoiser
constexpr int kDenoiserParams = 21409;    // model blob floats
constexpr int kDenoiseParts = 456;        // CTAs of a weight-gradient pass (fixed-order partials; 3 x 152 SMs)
struct DenoiseLayout {                    // byte offsets in the workspace
    size_t scale, sums, x0, a1, a2, a3, y, dy, d_hi, d_lo, part;
    // tensor-core forward (widths 32, 64, 128): channels-last copies of x (padded
    // to 32 channels), a1 and a2, and the bf16 weights of layers 0..2; tc = 0 if
    // the width does not allow it
    int tc;
    size_t xc, c1, c2, wt;
    // tensor-core weight gradients (training, width 64): the layer's output
    // gradient as two bf16 terms [slice][2 Cout][H][W], x-shifted copies of the
    // layer input [slice][3 Cin'][H][W] (Cin' = 16 or 32), per-CTA partial sums
    // and per-block bias sums; wg = 0 if the width does not allow it
    int wg;
    size_t dsplit, shifted, wgpart, bpart;
    // and the input gradients of layers 2 and 1 on the tensor cores: the split
    // delta channels-last (hi, lo) and the flipped bf16 weights of layers 1, 2
    size_t dcl_hi, dcl_lo, wtb, bytes;
};
constexpr int kWgMaxCtas = 152 * 2;       // CTAs of a tensor-core weight-gradient pass (partial slots)
// Tiled tensor map over a bfloat16 array of rank 3 or 4 with 64-byte swizzle
// (box innermost extent 64 bytes); dims innermost first, strides in bytes for
// dims 1..rank-1.  False if the driver rejects it.
bool make_bf16_map_sw64(CUtensorMap* m, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                        const uint32_t* box);
// As make_bf16_map_sw64 with 128-byte swizzle (box innermost extent 128 bytes).
bool make_bf16_map_sw128(CUtensorMap* m, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                         const uint32_t* box);
DenoiseLayout denoise_layout(int ha, int wa, int hb, int wb, bool training);
// scale, stacked input, activations and y of the network on gamma_in (keep_cf:
// also the channels-first activations the backward pass reads; status,
// timeout_ns: the bounded waits of the tensor-core layers)
cudaError_t denoise_forward(const float* model, const float* gamma_in, int ha, int wa, int hb, int wb,
                            uint8_t* ws, const DenoiseLayout& L, bool keep_cf, unsigned int* status,
                            unsigned long long timeout_ns, cudaStream_t st);
cudaError_t denoise_output(const uint8_t* ws, const DenoiseLayout& L, int64_t n, float* gamma_out,
                           cudaStream_t st);
// after denoise_forward: loss and gradient of the model blob
cudaError_t denoise_backward(const float* model, const float* gamma_target, int ha, int wa, int hb, int wb,
                             uint8_t* ws, const DenoiseLayout& L, float* grad, float* loss, int sm_count,
                             unsigned int* status, unsigned long long timeout_ns, cudaStream_t st);
cudaError_t denoise_adam(float* model, float* m, float* v, const float* grad, int64_t step, float lr,
                         cudaStream_t st);

// ------------------------------------------------------------------ self test
cudaError_t launch_wait_selftest(unsigned int* status, unsigned long long timeout_ns,
                                 cudaStream_t st);

}  // namespace cpi
