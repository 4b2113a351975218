// Step a1/a3: frames -> tensor-core operands and marginal sums.
//
// The frames arrive frame-major (all pixels of frame i, then frame i+1, ...),
// packed one bit per pixel (Section 2 of the paper) or one byte per pixel.  The
// raw-moment contraction sums over frames, so each operand row must hold one
// pixel's values over consecutive frames (K-major):
//   - 1-bit frames whose region rows are whole 32-pixel words apart ->
//     FP4 E2M1 values packed two per byte (0x0 / 0x2 = 1.0; frame 2j in the low
//     nibble of byte j), ingest_bits_kernel: a block of frames staged word-wise
//     in shared memory, transposed 32 x 32 bits per warp;
//   - 8-bit frames with 4-pixel aligned regions -> BF16 (integers 0..255 are
//     exact), ingest_u8x4_kernel: one CTA per tile of 128 pixels x 128 frames;
//   - any other frames -> BF16 (1-bit frames that do not meet the first case as
//     packed E2M1), one CTA per tile of 32 pixels x 128 (BF16) or 256 (E2M1)
//     frames.
// The raw-moment GEMM loads the packed E2M1 rows with a tensor map of 16 x 4-bit
// groups, which spreads each 8-byte group over 16 bytes of shared memory: the
// layout tcgen05 kind::f8f6f4 reads 4-bit operands in.  A binary operand row is
// so half as many bytes in HBM and L2 as an 8-bit one would be.
// Frames at or beyond n_frames are written as 0, so every operand row is padded
// to a whole number of CTA tiles.  The same pass adds the marginal sums
// S_a = sum_i A_i (Eq. (1), second term) with exact int64 atomics.

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
            // BF16 of v < 2^8 without the conversion pipe: (2^23 + v) - 2^23 = v exactly,
            // and its upper half is BF16(v)
            const float flo = __uint_as_float(0x4B000000u | lo) - 8388608.0f;
            const float fhi = __uint_as_float(0x4B000000u | hi) - 8388608.0f;
            w[j] = __byte_perm(__float_as_uint(flo), __float_as_uint(fhi), 0x7632u);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t word = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int64_t f = f0 + 8 * j + q;
                uint32_t v = 0;
                if (valid && f < n_frames) v = load_pixel(d, base, sh, f);
                sum += v;
                word |= (v ? 0x2u : 0u) << (4 * q);   // E2M1 1.0 = 0x2, frame 2k in the low nibble
            }
            w[j] = word;
        }
    }
    if constexpr (kBf16) {
        uint4* dst = reinterpret_cast<uint4*>(&tile_s[lane][warp * 32]);
        dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
        dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
    } else {
        *reinterpret_cast<uint4*>(&tile_s[lane][warp * 16]) = make_uint4(w[0], w[1], w[2], w[3]);
    }
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

    // 32 rows x 256 bytes (BF16) or 128 bytes (E2M1) in chunks of 16 bytes;
    // consecutive threads write consecutive chunks of one operand row.
    constexpr int kRowOut = kBf16 ? kIngestRowBytes : kIngestRowBytes / 2;
    constexpr int kChunks = kRowOut / 16;
#pragma unroll
    for (int it = 0; it < kIngestPixels * kChunks / 256; ++it) {
        const int idx = it * 256 + threadIdx.x;
        const int row = idx / kChunks, chunk = idx % kChunks;
        const int64_t pp = (int64_t)tile * kIngestPixels + row;
        if (pp < M) {
            const uint4 v = *reinterpret_cast<const uint4*>(&tile_s[row][chunk * 16]);
            *reinterpret_cast<uint4*>(op + pp * kstride_bytes + (int64_t)blockIdx.y * kRowOut + chunk * 16) = v;
        }
    }
    if (warp == 0 && valid) {
        long long t = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += part[k][lane];
        if (t) atomicAdd(reinterpret_cast<unsigned long long*>(s + p), (unsigned long long)t);
    }
}

// 8-bit frames whose regions are 4-pixel aligned (width, x0, row and frame
// strides multiples of 4 bytes): CTA = 128 pixels x 128 frames.  Lane l of warp
// w loads pixels 4l .. 4l + 3 of the tile (one 4-byte word, so a warp reads 128
// contiguous bytes of a frame row) for frames 16w .. 16w + 15, all 16 loads in
// flight.  BF16 of a byte v without the conversion pipe: the float with bits
// 0x4B000000 | v is 2^23 + v, minus 2^23 is v exactly, and v < 2^8 leaves the low
// 16 bits of its float zero, so its upper half is BF16(v) exactly.  Each lane
// writes its pixels' 32-byte row segments to a shared tile whose 16-byte chunks
// are XOR-swizzled by pixel / 4 (the 8 lanes of one store phase hit 8 distinct
// chunks), and the tile leaves as whole 256-byte operand rows.
constexpr int kX4Pixels = 128;
constexpr int kX4Frames = 128;                           // 256 bytes of BF16 per operand row
static_assert(kX4Frames * 2 == kIngestRowBytes, "same operand row blocks as ingest_kernel");

__device__ __forceinline__ uint32_t x4_prmt(uint32_t a, uint32_t b, uint32_t sel) {
    return __byte_perm(a, b, sel);
}

__global__ void __launch_bounds__(256) ingest_u8x4_kernel(FramesDev A, FramesDev B, int64_t n_frames,
                                                          int64_t kstride_bytes, uint8_t* op_a, uint8_t* op_b,
                                                          int64_t* s_a, int64_t* s_b, int tiles_a, uint32_t* vmax) {
    __shared__ __align__(16) uint8_t tile_s[kX4Pixels * kX4Frames * 2];   // [pixel][16 chunks of 16 B], swizzled
    __shared__ uint32_t part[8][kX4Pixels];
    __shared__ uint32_t wmax[8];
    const bool is_a = (int)blockIdx.x < tiles_a;
    const FramesDev d = is_a ? A : B;
    const int tile = is_a ? (int)blockIdx.x : (int)blockIdx.x - tiles_a;
    uint8_t* op = is_a ? op_a : op_b;
    int64_t* s = is_a ? s_a : s_b;
    const int64_t M = (int64_t)d.height * d.width;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    const int64_t p = (int64_t)tile * kX4Pixels + 4 * lane;   // first of the lane's 4 pixels (same image row)
    const bool valid = p < M;
    const uint8_t* base = d.data;
    if (valid) {
        const int64_t y = p / d.width, x = p - y * d.width;
        base += (d.y0 + y) * d.row_stride + d.x0 + x;
    }
    const int64_t f0 = (int64_t)blockIdx.y * kX4Frames + warp * 16;
    uint32_t v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j)
        v[j] = (valid && f0 + j < n_frames) ? __ldg(reinterpret_cast<const uint32_t*>(base + (f0 + j) * d.frame_stride))
                                            : 0u;
    // marginal sums: bytes 0, 2 and 1, 3 in 16-bit lanes (16 x 255 < 2^16)
    uint32_t s02 = 0, s13 = 0, mx4 = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        s02 += v[j] & 0x00FF00FFu;
        s13 += (v[j] >> 8) & 0x00FF00FFu;
        mx4 = __vmaxu4(mx4, v[j]);
    }
    const uint32_t pix_sum[4] = {s02 & 0xFFFFu, s13 & 0xFFFFu, s02 >> 16, s13 >> 16};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        // 16 frames of pixel 4 lane + q: 8 words of two BF16 values, as two 16-byte chunks
        uint32_t w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            // 0x4B0000vv for frames 2j and 2j + 1 (byte q of each word)
            const uint32_t lo = x4_prmt(v[2 * j], 0x4B000000u, 0x7440u + (uint32_t)q);
            const uint32_t hi = x4_prmt(v[2 * j + 1], 0x4B000000u, 0x7440u + (uint32_t)q);
            const float flo = __uint_as_float(lo) - 8388608.0f, fhi = __uint_as_float(hi) - 8388608.0f;
            w[j] = x4_prmt(__float_as_uint(flo), __float_as_uint(fhi), 0x7632u);
        }
        const int row = 4 * lane + q, swz = lane & 7;
        uint4* dst = reinterpret_cast<uint4*>(tile_s + row * (kX4Frames * 2));
        dst[(2 * warp) ^ swz] = make_uint4(w[0], w[1], w[2], w[3]);
        dst[(2 * warp + 1) ^ swz] = make_uint4(w[4], w[5], w[6], w[7]);
        part[warp][row] = pix_sum[q];
    }
    uint32_t m = max(max(mx4 & 0xFFu, (mx4 >> 8) & 0xFFu), max((mx4 >> 16) & 0xFFu, mx4 >> 24));
    m = __reduce_max_sync(0xffffffffu, m);
    if (lane == 0) wmax[warp] = m;
    __syncthreads();
    if (vmax != nullptr && threadIdx.x == 0) {
        uint32_t mm = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) mm = max(mm, wmax[k]);
        uint32_t* slot = vmax + (is_a ? 0 : 1);
        if (mm > *reinterpret_cast<volatile uint32_t*>(slot)) atomicMax(slot, mm);
    }
    // 128 rows x 16 chunks; 16 consecutive threads write one 256-byte operand row
#pragma unroll
    for (int it = 0; it < kX4Pixels * 16 / 256; ++it) {
        const int idx = it * 256 + threadIdx.x;
        const int row = idx >> 4, c = idx & 15;
        const int64_t pp = (int64_t)tile * kX4Pixels + row;
        if (pp < M) {
            const uint4 val = reinterpret_cast<const uint4*>(tile_s + row * (kX4Frames * 2))[c ^ ((row >> 2) & 7)];
            *reinterpret_cast<uint4*>(op + pp * kstride_bytes + (int64_t)blockIdx.y * (kX4Frames * 2) + c * 16) = val;
        }
    }
    if (threadIdx.x < kX4Pixels) {
        const int64_t pp = (int64_t)tile * kX4Pixels + threadIdx.x;
        if (pp < M) {
            uint32_t t = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) t += part[k][threadIdx.x];
            if (t) atomicAdd(reinterpret_cast<unsigned long long*>(s + pp), (unsigned long long)t);
        }
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
// 4-byte aligned frames.  CTA = (region, chunk of kWC frame words) x block of
// kFB frames.  Words w0 .. w0 + kWC of every frame of the block are loaded with
// coalesced 4-byte loads into shared memory, in rows of kWP words (kWP odd: a
// warp reading one word of 32 frames touches 32 banks).  Each warp then takes
// whole 32-pixel tiles of the region whose first word lies in the chunk: per 32
// frames, lane i funnel-shifts its frame's 32 pixel bits out of two words, the
// warp transposes the 32 x 32 bit block (lane j then holds pixel j over the 32
// frames), and each bit becomes one E2M1 nibble (0x2 = 1.0; 8 bits -> 8 nibbles
// by three shift-or-mask steps).  The tile's 32 operand rows of kFB / 2 bytes
// are staged per warp and stored as whole 64-byte row pieces; one int64 atomic
// per pixel adds the block's count to the marginal sum.
constexpr int kFB = 128;                 // frames per CTA
constexpr int kWC = 64;                  // frame words per chunk
constexpr int kWP = kWC + 1;             // shared row pitch in words (odd)
constexpr int kStageRow = kFB / 2 + 16;  // staged operand row (E2M1, two frames per byte), bytes
constexpr size_t kBitsSmem = sizeof(uint32_t) * kFB * kWP + (size_t)8 * 32 * kStageRow;
static_assert(kWP % 2 == 1, "odd pitch");

__host__ __device__ inline int64_t floor_div(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// First and last frame word a region's pixels occupy.
__host__ __device__ inline int64_t region_first_word(const FramesDev& d) {
    return ((int64_t)d.y0 * d.row_stride + d.x0) >> 5;
}
__host__ __device__ inline int64_t region_last_word(const FramesDev& d) {
    return ((int64_t)(d.y0 + d.height - 1) * d.row_stride + d.x0 + d.width - 1) >> 5;
}

__global__ void __launch_bounds__(256) ingest_bits_kernel(FramesDev A, FramesDev B, int64_t n_frames, int64_t f_base,
                                                          int64_t kstride_bytes, uint8_t* op_a, uint8_t* op_b,
                                                          int64_t* s_a, int64_t* s_b, int chunks_a) {
    extern __shared__ __align__(16) uint8_t smem_bits[];
    uint32_t* S = reinterpret_cast<uint32_t*>(smem_bits);                       // [kFB][kWP]
    const bool is_a = (int)blockIdx.x < chunks_a;
    const FramesDev d = is_a ? A : B;
    const int chunk = is_a ? (int)blockIdx.x : (int)blockIdx.x - chunks_a;
    uint8_t* op = is_a ? op_a : op_b;
    int64_t* s = is_a ? s_a : s_b;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t* st = smem_bits + sizeof(uint32_t) * kFB * kWP + (size_t)warp * 32 * kStageRow;

    const int64_t w0 = region_first_word(d) + (int64_t)chunk * kWC;
    const int64_t words_per_frame = d.frame_stride >> 2;
    const int64_t f0 = f_base + (int64_t)blockIdx.y * kFB;
    // asynchronous 4-byte copies (all of a thread's loads in flight at once);
    // words past the frames or past a frame's end are zero-filled
    // (warp w copies frames w, w + 8, ...; lane l words l and l + 32, lane 0 also word 64)
    static_assert(kWC == 64, "two words per lane plus one");
    for (int fr = warp; fr < kFB; fr += 8) {
        const int64_t f = f0 + fr;
        const uint32_t* fbase = reinterpret_cast<const uint32_t*>(d.data + (f < n_frames ? f : 0) * d.frame_stride) + w0;
        const uint32_t sbase = static_cast<uint32_t>(__cvta_generic_to_shared(S + fr * kWP));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int w = k < 2 ? lane + 32 * k : 64;
            if (k == 2 && lane != 0) break;
            const bool in = f < n_frames && w0 + w < words_per_frame;
            const uint32_t* src = in ? fbase + w : reinterpret_cast<const uint32_t*>(d.data);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sbase + 4u * (uint32_t)w), "l"(src),
                         "r"(in ? 4 : 0)
                         : "memory");
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();

    // rows with a tile whose first bit e0 = (y0 + y) rs + x0 + 32 xt lies in the chunk
    const int ntx = d.width >> 5;
    const int64_t rs = d.row_stride, lo_bit = w0 << 5, hi_bit = (w0 + kWC) << 5;
    int64_t ylo = -floor_div(-(lo_bit - d.x0 - 32 * (int64_t)(ntx - 1)), rs) - d.y0;
    int64_t yhi = floor_div(hi_bit - 1 - d.x0, rs) - d.y0;
    if (ylo < 0) ylo = 0;
    if (yhi > d.height - 1) yhi = d.height - 1;
    const int64_t n_items = yhi >= ylo ? (yhi - ylo + 1) * ntx : 0;
    for (int64_t t = warp; t < n_items; t += 8) {
        const int64_t y = ylo + t / ntx;
        const int xt = (int)(t - (t / ntx) * ntx);
        const int64_t e0 = (d.y0 + y) * rs + d.x0 + 32 * (int64_t)xt;
        if (e0 < lo_bit || e0 >= hi_bit) continue;             // warp-uniform
        const int wl = (int)((e0 >> 5) - w0), sh = (int)(e0 & 31);
        int cnt = 0;
#pragma unroll
        for (int g = 0; g < kFB / 32; ++g) {
            const uint32_t* row = S + (g * 32 + lane) * kWP + wl;
            uint32_t lo = row[0], hi = sh ? row[1] : 0u;
            if (d.bit_order) {   // MSB-first bytes: reverse the bits of every byte first
                lo = __byte_perm(__brev(lo), 0, 0x0123);
                hi = __byte_perm(__brev(hi), 0, 0x0123);
            }
            const uint32_t col = warp_transpose32(__funnelshift_r(lo, hi, sh), lane);
            cnt += __popc(col);
            uint32_t o[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {   // frames 8k .. 8k + 7 -> nibbles 0 .. 7 of word k
                uint32_t x = (col >> (8 * k)) & 0xFFu;
                x = (x | (x << 12)) & 0x000F000Fu;
                x = (x | (x << 6)) & 0x03030303u;
                x = (x | (x << 3)) & 0x11111111u;
                o[k] = x << 1;
            }
            *reinterpret_cast<uint4*>(st + lane * kStageRow + g * 16) = make_uint4(o[0], o[1], o[2], o[3]);
        }
        __syncwarp();
        const int64_t p0 = y * d.width + 32 * (int64_t)xt;
#pragma unroll
        for (int k = 0; k < 32 * (kFB / 2) / 16 / 32; ++k) {
            const int idx = k * 32 + lane, r = idx / (kFB / 32), c16 = idx % (kFB / 32);
            *reinterpret_cast<uint4*>(op + (p0 + r) * kstride_bytes + f0 / 2 + c16 * 16) =
                *reinterpret_cast<const uint4*>(st + r * kStageRow + c16 * 16);
        }
        __syncwarp();
        if (cnt) atomicAdd(reinterpret_cast<unsigned long long*>(s + p0 + lane), (unsigned long long)cnt);
    }
}

}  // namespace

// Conditions of the word-load path for binary frames.
static bool bits_fast_ok(const FramesDev& d) {
    return d.bits == 1 && d.width % 32 == 0 && d.frame_stride % 4 == 0 &&
           reinterpret_cast<uintptr_t>(d.data) % 4 == 0;
}
// Conditions of the 4-pixel path for 8-bit frames.
static bool u8x4_ok(const FramesDev& d) {
    return d.bits == 8 && d.width % 4 == 0 && d.x0 % 4 == 0 && d.row_stride % 4 == 0 && d.frame_stride % 4 == 0 &&
           reinterpret_cast<uintptr_t>(d.data) % 4 == 0;
}
cudaError_t launch_ingest(bool bf16, const FramesDev& a, const FramesDev& b, int64_t n_frames,
                          int64_t kstride_bytes, uint8_t* op_a, uint8_t* op_b, int64_t* s_a,
                          int64_t* s_b, uint32_t* vmax, cudaStream_t st) {
    const int64_t Ma = (int64_t)a.height * a.width, Mb = (int64_t)b.height * b.width;
    const int tiles_a = (int)((Ma + kIngestPixels - 1) / kIngestPixels);
    const int tiles_b = (int)((Mb + kIngestPixels - 1) / kIngestPixels);
    if (!bf16 && bits_fast_ok(a) && bits_fast_ok(b) && (2 * kstride_bytes) % kFB == 0) {
        static bool attr[64] = {};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (!attr[dev]) {
            e = cudaFuncSetAttribute(ingest_bits_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBitsSmem);
            if (e != cudaSuccess) return e;
            attr[dev] = true;
        }
        const int chunks_a = (int)((region_last_word(a) - region_first_word(a)) / kWC + 1);
        const int chunks_b = (int)((region_last_word(b) - region_first_word(b)) / kWC + 1);
        const int64_t blocks = 2 * kstride_bytes / kFB;   // two E2M1 frames per byte
        for (int64_t y0 = 0; y0 < blocks; y0 += 65535) {   // grid.y limit
            const int64_t ny = blocks - y0 < 65535 ? blocks - y0 : 65535;
            ingest_bits_kernel<<<dim3((unsigned)(chunks_a + chunks_b), (unsigned)ny), 256, kBitsSmem, st>>>(
                a, b, n_frames, y0 * kFB, kstride_bytes, op_a, op_b, s_a, s_b, chunks_a);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const int64_t row_out = bf16 ? kIngestRowBytes : kIngestRowBytes / 2;   // operand bytes per CTA row
    const int64_t frame_tiles = kstride_bytes / row_out;
    if (bf16 && u8x4_ok(a) && u8x4_ok(b)) {
        const int xa = (int)((Ma + kX4Pixels - 1) / kX4Pixels), xb = (int)((Mb + kX4Pixels - 1) / kX4Pixels);
        for (int64_t t0 = 0; t0 < frame_tiles; t0 += 65535) {   // grid.y limit
            const int64_t nt = frame_tiles - t0 < 65535 ? frame_tiles - t0 : 65535;
            FramesDev a2 = a, b2 = b;
            a2.data = a.data + t0 * kX4Frames * a.frame_stride;
            b2.data = b.data + t0 * kX4Frames * b.frame_stride;
            ingest_u8x4_kernel<<<dim3((unsigned)(xa + xb), (unsigned)nt), 256, 0, st>>>(
                a2, b2, n_frames - t0 * kX4Frames, kstride_bytes, op_a + t0 * kIngestRowBytes,
                op_b + t0 * kIngestRowBytes, s_a, s_b, xa, vmax);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
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
                ingest_kernel<true><<<grid, 256, 0, st>>>(a2, b2, rem, kstride_bytes, op_a + t0 * row_out,
                                                          op_b + t0 * row_out, s_a, s_b, tiles_a, vmax);
            else
                ingest_kernel<false><<<grid, 256, 0, st>>>(a2, b2, rem, kstride_bytes, op_a + t0 * row_out,
                                                           op_b + t0 * row_out, s_a, s_b, tiles_a, nullptr);
        }
        return cudaGetLastError();
    }
    dim3 grid(tiles_a + tiles_b, (unsigned)frame_tiles);
    if (bf16)
        ingest_kernel<true><<<grid, 256, 0, st>>>(a, b, n_frames, kstride_bytes, op_a, op_b, s_a,
                                                  s_b, tiles_a, vmax);
    else
        ingest_kernel<false><<<grid, 256, 0, st>>>(a, b, n_frames, kstride_bytes, op_a, op_b, s_a,
                                                   s_b, tiles_a, nullptr);
    return cudaGetLastError();
}

}  // namespace cpi
