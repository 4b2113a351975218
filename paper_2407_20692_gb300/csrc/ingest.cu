// Step a1/a3: frames -> tensor-core operands and marginal sums.
//
// The frames arrive frame-major (all pixels of frame i, then frame i+1, ...),
// packed one bit per pixel (Section 2 of the paper) or one byte per pixel.  The
// raw-moment contraction sums over frames, so each operand row must hold one
// pixel's values over consecutive frames (K-major).  One CTA transposes a tile
// of 32 pixels x 256 output bytes through shared memory:
//   - 1-bit frames -> FP8 E4M3 bytes (0x00 / 0x38 = 1.0), 256 frames per CTA;
//   - any frames   -> BF16 (integers 0..255 are exact), 128 frames per CTA.
// Frames at or beyond n_frames are written as 0, so every operand row is padded
// to a whole number of CTA tiles.  The same pass adds the marginal sums
// S_a = sum_i A_i (Eq. (1), second term) with exact int64 atomics.
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace cpi {
namespace {

__device__ __forceinline__ uint32_t load_pixel(const FramesDev& d, const uint8_t* base, int sh,
                                               int64_t f) {
    const uint8_t v = __ldg(base + f * d.frame_stride);
    return d.bits == 8 ? (uint32_t)v : ((uint32_t)v >> sh) & 1u;
}

template <bool kBf16>
__global__ void __launch_bounds__(256) ingest_kernel(FramesDev A, FramesDev B, int64_t n_frames,
                                                     int64_t kstride_bytes, uint8_t* op_a,
                                                     uint8_t* op_b, int64_t* s_a, int64_t* s_b,
                                                     int tiles_a, uint32_t* vmax) {
    constexpr int kFramesPerWarp = kBf16 ? 16 : 32;   // 32 operand bytes per pixel per warp
    const bool is_a = (int)blockIdx.x < tiles_a;
    const FramesDev d = is_a ? A : B;
    const int tile = is_a ? (int)blockIdx.x : (int)blockIdx.x - tiles_a;
    uint8_t* op = is_a ? op_a : op_b;
    int64_t* s = is_a ? s_a : s_b;
    const int64_t M = (int64_t)d.height * d.width;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    __shared__ __align__(16) uint8_t tile_s[kIngestPixels][kIngestRowBytes + 16];
    __shared__ long long part[8][32];
    __shared__ uint32_t wmax[8];

    const int64_t p = (int64_t)tile * kIngestPixels + lane;
    const bool valid = p < M;
    int64_t e = 0;
    if (valid) {
        const int64_t y = p / d.width, x = p - y * d.width;
        e = (d.y0 + y) * d.row_stride + d.x0 + x;
    }
    const uint8_t* base = d.data + (d.bits == 8 ? e : (e >> 3));
    int sh = (int)(e & 7);
    if (d.bit_order) sh = 7 - sh;

    const int64_t f0 = (int64_t)blockIdx.y * (kFramesPerWarp * 8) + warp * kFramesPerWarp;
    long long sum = 0;
    uint32_t w[8];
    uint32_t mx = 0;
    if constexpr (kBf16) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t lo = 0, hi = 0;
            const int64_t f = f0 + 2 * j;
            if (valid && f < n_frames) lo = load_pixel(d, base, sh, f);
            if (valid && f + 1 < n_frames) hi = load_pixel(d, base, sh, f + 1);
            sum += lo + hi;
            mx = max(mx, max(lo, hi));
            const uint32_t blo = __bfloat16_as_ushort(__float2bfloat16_rn((float)lo));
            const uint32_t bhi = __bfloat16_as_ushort(__float2bfloat16_rn((float)hi));
            w[j] = blo | (bhi << 16);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t word = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t f = f0 + 4 * j + q;
                uint32_t v = 0;
                if (valid && f < n_frames) v = load_pixel(d, base, sh, f);
                sum += v;
                word |= (v ? 0x38u : 0u) << (8 * q);   // E4M3 1.0 = 0x38
            }
            w[j] = word;
        }
    }
    uint4* dst = reinterpret_cast<uint4*>(&tile_s[lane][warp * 32]);
    dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
    dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
    part[warp][lane] = sum;
    if constexpr (kBf16) {
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0) wmax[warp] = mx;
    }
    __syncthreads();
    if (kBf16 && vmax != nullptr && threadIdx.x == 0) {
        uint32_t m = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) m = max(m, wmax[k]);
        uint32_t* slot = vmax + (is_a ? 0 : 1);
        // read first: the atomic is needed only while the recorded maximum grows
        if (m > *reinterpret_cast<volatile uint32_t*>(slot)) atomicMax(slot, m);
    }

    // 32 rows x 256 bytes = 512 chunks of 16 bytes; consecutive threads write
    // consecutive chunks of one operand row.
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int idx = it * 256 + threadIdx.x;
        const int row = idx >> 4, chunk = idx & 15;
        const int64_t pp = (int64_t)tile * kIngestPixels + row;
        if (pp < M) {
            const uint4 v = *reinterpret_cast<const uint4*>(&tile_s[row][chunk * 16]);
            *reinterpret_cast<uint4*>(op + pp * kstride_bytes + (int64_t)blockIdx.y * kIngestRowBytes +
                                      chunk * 16) = v;
        }
    }
    if (warp == 0 && valid) {
        long long t = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += part[k][lane];
        if (t) atomicAdd(reinterpret_cast<unsigned long long*>(s + p), (unsigned long long)t);
    }
}

// 32 x 32 bit-matrix transpose across a warp: lane i holds row i on entry
// (bit j = column j) and column i on exit (bit j = row j).  Five rounds of
// block swaps (16, 8, 4, 2, 1).
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t w, int lane) {
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const int s = 16 >> r;
        const uint32_t m = masks[r];
        const uint32_t t = __shfl_xor_sync(0xffffffffu, w, s);
        w = (lane & s) ? ((w & ~m) | ((t >> s) & m)) : ((w & m) | ((t << s) & ~m));
    }
    return w;
}

// Binary frames whose region rows are a multiple of 32 pixels wide, with
// 4-byte aligned frames.  CTA = 32 consecutive region pixels (within one row) x
// 1024 frames; warp w takes, in each of 4 rounds, frames f0 + 256r + 32w .. +31,
// one frame per lane.  All 8 word loads are issued first; then each lane
// funnel-shifts out the 32 pixel bits of its frame, the warp transposes the four
// 32 x 32 bit blocks together (lane j then holds pixel j's bits over 32 frames),
// and each bit becomes one E4M3 byte (0x38 = 1.0): 4 bits -> 4 bytes by one
// multiply that spreads them 8 bits apart.  The bytes are staged in shared
// memory and written as whole operand-row segments with coalesced stores.
constexpr int kBitsRounds = 4;
__global__ void __launch_bounds__(256) ingest_bits_kernel(FramesDev A, FramesDev B, int64_t n_frames,
                                                          int64_t kstride_bytes, uint8_t* op_a,
                                                          uint8_t* op_b, int64_t* s_a, int64_t* s_b,
                                                          int tiles_a) {
    const bool is_a = (int)blockIdx.x < tiles_a;
    const FramesDev d = is_a ? A : B;
    const int tile = is_a ? (int)blockIdx.x : (int)blockIdx.x - tiles_a;
    uint8_t* op = is_a ? op_a : op_b;
    int64_t* s = is_a ? s_a : s_b;
    const int64_t M = (int64_t)d.height * d.width;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ long long part[8][32];
    __shared__ __align__(16) uint8_t stile[32][256 * kBitsRounds + 16];

    const int64_t p0 = (int64_t)tile * 32;               // first pixel; the 32 share one row
    const int64_t y = p0 / d.width, x = p0 - y * d.width;
    const int64_t e0 = (d.y0 + y) * d.row_stride + d.x0 + x;   // bit offset inside a frame
    const int sh = (int)(e0 & 31);
    const int64_t fcta = (int64_t)blockIdx.y * (256 * kBitsRounds);
    uint32_t lo[kBitsRounds], hi[kBitsRounds];
#pragma unroll
    for (int r = 0; r < kBitsRounds; ++r) {
        const int64_t f = fcta + r * 256 + warp * 32 + lane;
        lo[r] = hi[r] = 0u;
        if (f < n_frames) {
            const uint32_t* w = reinterpret_cast<const uint32_t*>(d.data + f * d.frame_stride) + (e0 >> 5);
            lo[r] = __ldg(w);
            if (sh) hi[r] = __ldg(w + 1);
        }
    }
    const int64_t p = p0 + lane;
    uint32_t col[kBitsRounds];
#pragma unroll
    for (int r = 0; r < kBitsRounds; ++r) {
        uint32_t l = lo[r], h = hi[r];
        if (d.bit_order) {   // MSB-first bytes: reverse the bits of every byte first
            l = __byte_perm(__brev(l), 0, 0x0123);
            h = __byte_perm(__brev(h), 0, 0x0123);
        }
        col[r] = __funnelshift_r(l, h, sh);
    }
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        const int sw = 16 >> t;
        const uint32_t m = masks[t];
        uint32_t xx[kBitsRounds];
#pragma unroll
        for (int r = 0; r < kBitsRounds; ++r) xx[r] = __shfl_xor_sync(0xffffffffu, col[r], sw);
#pragma unroll
        for (int r = 0; r < kBitsRounds; ++r)
            col[r] = (lane & sw) ? ((col[r] & ~m) | ((xx[r] >> sw) & m)) : ((col[r] & m) | ((xx[r] << sw) & ~m));
    }
    int cnt = 0;
#pragma unroll
    for (int r = 0; r < kBitsRounds; ++r) {
        cnt += __popc(col[r]);
        uint32_t o[8];
#pragma unroll
        for (int qq = 0; qq < 8; ++qq) {
            const uint32_t nib = (col[r] >> (4 * qq)) & 0xFu;
            o[qq] = ((nib * 0x00204081u) & 0x01010101u) * 0x38u;
        }
        uint4* dst = reinterpret_cast<uint4*>(&stile[lane][r * 256 + warp * 32]);
        dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
        dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
    }
    __syncthreads();
    {
        const int64_t cols = kstride_bytes - fcta < 1024 ? kstride_bytes - fcta : 1024;
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int idx = it * 256 + threadIdx.x;
            const int rr = idx >> 6, c16 = idx & 63;
            const int64_t pp = p0 + rr;
            if (pp < M && c16 * 16 < cols)
                *reinterpret_cast<uint4*>(op + pp * kstride_bytes + fcta + c16 * 16) =
                    *reinterpret_cast<const uint4*>(&stile[rr][c16 * 16]);
        }
    }
    part[warp][lane] = cnt;
    __syncthreads();
    if (warp == 0 && p < M) {
        long long t = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += part[k][lane];
        if (t) atomicAdd(reinterpret_cast<unsigned long long*>(s + p), (unsigned long long)t);
    }
}

}  // namespace

// Conditions of the word-load path for binary frames.
static bool bits_fast_ok(const FramesDev& d) {
    return d.bits == 1 && d.width % 32 == 0 && d.frame_stride % 4 == 0 &&
           reinterpret_cast<uintptr_t>(d.data) % 4 == 0;
}
cudaError_t launch_ingest(bool bf16, const FramesDev& a, const FramesDev& b, int64_t n_frames,
                          int64_t kstride_bytes, uint8_t* op_a, uint8_t* op_b, int64_t* s_a,
                          int64_t* s_b, uint32_t* vmax, cudaStream_t st) {
    const int64_t Ma = (int64_t)a.height * a.width, Mb = (int64_t)b.height * b.width;
    const int tiles_a = (int)((Ma + kIngestPixels - 1) / kIngestPixels);
    const int tiles_b = (int)((Mb + kIngestPixels - 1) / kIngestPixels);
    const int64_t frame_tiles = kstride_bytes / kIngestRowBytes;
    if (frame_tiles > 65535) {
        // grid.y limit: split the frame range over several launches
        for (int64_t t0 = 0; t0 < frame_tiles; t0 += 65535) {
            const int64_t nt = frame_tiles - t0 < 65535 ? frame_tiles - t0 : 65535;
            const int64_t fpc = ingest_frames_per_cta(bf16);
            FramesDev a2 = a, b2 = b;
            a2.data = a.data + t0 * fpc * a.frame_stride;
            b2.data = b.data + t0 * fpc * b.frame_stride;
            const int64_t rem = n_frames - t0 * fpc;
            dim3 grid(tiles_a + tiles_b, (unsigned)nt);
            if (bf16)
                ingest_kernel<true><<<grid, 256, 0, st>>>(a2, b2, rem, kstride_bytes,
                                                          op_a + t0 * kIngestRowBytes,
                                                          op_b + t0 * kIngestRowBytes, s_a, s_b,
                                                          tiles_a, vmax);
            else
                ingest_kernel<false><<<grid, 256, 0, st>>>(a2, b2, rem, kstride_bytes,
                                                           op_a + t0 * kIngestRowBytes,
                                                           op_b + t0 * kIngestRowBytes, s_a, s_b,
                                                           tiles_a, nullptr);
        }
        return cudaGetLastError();
    }
    dim3 grid(tiles_a + tiles_b, (unsigned)frame_tiles);
    if (!bf16 && bits_fast_ok(a) && bits_fast_ok(b)) {
        const int64_t gy = (kstride_bytes + 256 * kBitsRounds - 1) / (256 * kBitsRounds);
        if (gy > 65535) return cudaErrorInvalidValue;
        ingest_bits_kernel<<<dim3(tiles_a + tiles_b, (unsigned)gy), 256, 0, st>>>(
            a, b, n_frames, kstride_bytes, op_a, op_b, s_a, s_b, tiles_a);
        return cudaGetLastError();
    }
    if (bf16)
        ingest_kernel<true><<<grid, 256, 0, st>>>(a, b, n_frames, kstride_bytes, op_a, op_b, s_a,
                                                  s_b, tiles_a, vmax);
    else
        ingest_kernel<false><<<grid, 256, 0, st>>>(a, b, n_frames, kstride_bytes, op_a, op_b, s_a,
                                                   s_b, tiles_a, nullptr);
    return cudaGetLastError();
}

}  // namespace cpi
