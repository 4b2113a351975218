// Step a5: refocusing (Section "CPI algorithm", item 2; Section 4.1, "Refocusing
// Optimization").  For plane (alpha, beta) and spatial output pixel (r, c):
//     out(r, c) = sum over angular pixels (br, bc) of
//                 Gamma~_(br,bc)( alpha*(r - cya) + beta*sy*(br - cyb) + cya,
//                                 alpha*(c - cxa) + beta*sx*(bc - cxb) + cxa )
// where Gamma~_b interpolates the spatial image Gamma[.][b] bilinearly (taps
// outside the grid read 0), cxa = (wa-1)/2, cxb = (wb-1)/2, sx = wa/wb, and
// likewise for rows.
//
// The sample point separates: its column depends only on (c, bc) and its row
// only on (r, br).  So for one plane and one angular row br the kernel first
// interpolates along x and sums over the angular columns,
//     U(y, c) = sum_bc  wx0(c,bc) S_(br,bc)(y, xo) + wx1(c,bc) S_(br,bc)(y, xo+1),
// then interpolates U along y:
//     out(r, c) += wy0(r,br) U(yo, c) + wy1(r,br) U(yo+1, c),
// which reads each staged slice value twice instead of four times.
//
// Coordinates are computed on the fly inside the kernel (the point of Section
// 4.1) in 32.32 fixed point: u = A + B with A = alpha*(j - c_a) + c_a per
// output column (row) and B = beta*s*(b - c_b) per angular column (row), each
// rounded once from FP64.  The fraction is rounded to 24 bits, so both weights
// (1 - f, f) are exact FP32 numbers and sum to exactly 1.  Sums are FP32 with
// Kahan compensation across pairs of angular columns; the partial image of each
// angular row is written in FP32 and the rows are added in a fixed order
// (Kahan-compensated) by a second kernel, so the result is deterministic.
//
// Layout: Gamma arrives slice-major, float [Mb][Ma]; slice b is one contiguous
// spatial image, staged into shared memory by TMA (see the pipelined kernel).
//
// This file is compiled without FMA contraction: the Kahan steps depend on the
// written rounding order; the products use explicit fmaf.
#include <cstring>

#include "kernels.cuh"
#include "ptx.cuh"

namespace cpi {
namespace {

constexpr int kBox = 256;        // elements per 1-D TMA box
constexpr int kUPad = 2;         // zero rows above and below each U image

// ------------------------------------------------------------ coordinates
__device__ __forceinline__ long long fix32(double v) { return __double2ll_rn(v * 4294967296.0); }

struct Frac {
    int i;      // floor of the coordinate
    float f;    // fraction, a multiple of 2^-24 in [0, 1)
};
__device__ __forceinline__ Frac split_fix(long long u) {
    const long long u24 = (u + 128) >> 8;      // round the 32-bit fraction to 24 bits
    return {(int)(u24 >> 24), (float)(int)(u24 & 0xFFFFFF) * 0x1p-24f};
}

// Taps of one axis in an unpadded row of n values: read columns off and off+1
// with weights w0, w1.  Taps outside [0, n) get weight 0 and are moved onto
// in-grid columns, so no read leaves the staged slice.
struct __align__(16) STap {
    int off;
    float w0, w1;
    int unused;
};
__device__ __forceinline__ STap slice_tap(long long u, int n) {
    const Frac q = split_fix(u);
    const float w1 = q.f, w0 = 1.0f - q.f;
    if (q.i >= 0 && q.i <= n - 2) return {q.i, w0, w1, 0};
    if (q.i == -1) return {0, w1, 0.0f, 0};                       // only column 0 inside
    if (q.i == n - 1) return n >= 2 ? STap{n - 2, 0.0f, w0, 0} : STap{0, w0, 0.0f, 0};
    return {0, 0.0f, 0.0f, 0};
}

// Taps of one axis in a buffer with kUPad zero rows (columns) on both sides:
// out-of-grid taps read the zero border.
struct PTap {
    int off;
    float w0, w1;
};
__device__ __forceinline__ PTap padded_tap(long long u, int n) {
    const Frac q = split_fix(u);
    return {min(max(q.i, -kUPad), n) + kUPad, 1.0f - q.f, q.f};
}

__device__ __forceinline__ void kahan_add(float& acc, float& cmp, float v) {
    const float y = v - cmp;
    const float t = acc + y;
    cmp = (t - acc) - y;
    acc = t;
}

__device__ __forceinline__ void tma_load_1d(void* dst, const CUtensorMap* m, uint64_t* bar, int32_t x) {
    asm volatile(
        "cp.async.bulk.tensor.1d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(smem_u32(bar)), "r"(x)
        : "memory");
}

// ------------------------------------------------------------ pipelined kernel
// Persistent: one CTA of kThreads per SM walks the work units blockIdx.x,
// blockIdx.x + gridDim.x, ...  A unit is (angular row br, block of PB planes);
// units are ordered br-major, so CTAs running at the same time stage the same
// slices (L2 reuse) and, as the grid is a multiple of the plane-block count in
// the common case, a CTA keeps its plane block from unit to unit.
//
// Slices (br, bc) of the CTA's units stream through kStages shared-memory
// buffers, one TMA copy (group) each, completion counted on full[stage].  The
// last warp to finish with a buffer (a shared counter per stage) issues the copy
// of the slice kStages further on into it, so no thread ever waits for a free
// buffer.  Staging: a 2-D box of (wa4 + 8) x R*NK rows from column -4, wa4 = wa
// rounded up to a multiple of 4 (columns outside 0 .. wa-1 come back as zeros:
// the out-of-grid taps), when wa4 + 8 <= 256 and R*NK <= 256; rows past the
// slice's ha are the next slice's (or zeros past Gamma's end).  A Gamma whose
// rows are not 16-byte multiples is first copied with its rows padded to wa4
// floats (refocus_repack_kernel).  Wider slices: 1-D boxes of 256 elements from
// the 16-byte boundary at or below the slice (which then sits 0-3 elements in).
//
// Thread t owns column c = t % wa and rows rp + R*k, k < NK (row_split below).
// For each step of NSTEP staged slices it reads the x taps of a group of 2 or 4
// planes (from a per-plane-block table when it fits in shared memory, else
// computes them), then, rows outer and planes inner, adds the step's slices with
// fused multiply-adds and Kahan-adds the sum into its U values.  After the
// unit's last slice each plane's U image in turn goes to shared memory and is
// interpolated along y; this angular row's contribution to each output pixel is
// written to partial[br][plane][pixel].
//
// Every wait is bounded (the device status word records a time out).  A slice
// that never arrives stops every thread at that same slice, so no barrier is
// left half-entered.
constexpr int kThreads = 512;
constexpr int kMaxStages = 4;
constexpr int kPadL = 4;         // zero columns left of a 2-D staged row (TMA x start -4)
constexpr int kPadR = 4;

// Rows of the spatial image per thread: NK = ceil(ha / floor(kThreads / wa)),
// the threads of one column split the rows into R = ceil(ha / NK) row sets
// (thread row rp takes rows rp, rp + R, ...).  Every thread runs NK rows; the
// R * NK - ha (< NK) rows past the image are staged too (the next slice's rows,
// or zeros past Gamma's end) and their sums are dropped.
struct RowSplit {
    int R, NK;
};
__host__ __device__ inline RowSplit row_split(int ha, int wa) {
    const int r0 = kThreads / wa;
    const int nk = (ha + r0 - 1) / r0;
    return {(ha + nk - 1) / nk, nk};
}

template <bool kPad>
struct XTab;
template <>
struct XTab<true> {    // 2-D staged rows with zero borders: w0 = 1 - w1
    int off;
    float w1;
};
template <>
struct XTab<false> {   // unpadded rows: both weights (edge taps moved in-grid)
    STap t;
};

template <bool kPad>
__device__ __forceinline__ XTab<kPad> make_xtab(long long u, int wa, int sh) {
    if constexpr (kPad) {
        const Frac q = split_fix(u);
        return {min(max(q.i, -2), wa) + kPadL, q.f};
    } else {
        STap t = slice_tap(u, wa);
        t.off += sh;
        return {t};
    }
}

template <bool kPad>
__device__ __forceinline__ void read_xtab(const XTab<kPad>* e, int& off, float& w0, float& w1) {
    if constexpr (kPad) {
        const float2 v = *reinterpret_cast<const float2*>(e);
        off = __float_as_int(v.x);
        w1 = v.y;
        w0 = 1.0f - v.y;
    } else {
        const float4 v = *reinterpret_cast<const float4*>(e);
        off = __float_as_int(v.x);
        w0 = v.y;
        w1 = v.z;
    }
}

template <int KR, int PB, int NSTEP, int kST, bool kPad, bool kTable, int kWA, int kHA>
__global__ void __launch_bounds__(kThreads, 1) refocus_pipe_kernel(const __grid_constant__ CUtensorMap tm,
                                                                   const RefocusGeom geo, const PlaneBlock pl,
                                                                   float* __restrict__ partial) {
    static_assert(NSTEP == 1 || NSTEP == 2, "one or two slices per step");
    constexpr int NW = kThreads / 32;
    const int kStages = kST ? kST : geo.stages;        // 2..kMaxStages, > NSTEP
    extern __shared__ __align__(128) float sm_raw[];
    const int ha = kWA ? kHA : geo.ha, wa = kWA ? kWA : geo.wa, hb = geo.hb, wb = geo.wb;
    const int Ma = ha * wa;
    const int WS = kPad ? ((wa + 3) & ~3) + kPadL + kPadR : wa;     // staged row stride
    const int slice_f = geo.slice_f;                   // floats per stage buffer (multiple of 32)
    uint8_t* p = reinterpret_cast<uint8_t*>(
        sm_raw + (((128u - (static_cast<uint32_t>(__cvta_generic_to_shared(sm_raw)) & 127u)) & 127u) >> 2));
    float* const buf0 = reinterpret_cast<float*>(p);
    p += sizeof(float) * (size_t)kStages * slice_f;
    XTab<kPad>* const xtab = reinterpret_cast<XTab<kPad>*>(p);   // [PB][wb][wa] when kTable
    if (kTable) p += sizeof(XTab<kPad>) * (size_t)PB * wb * wa;
    PTap* const yt = reinterpret_cast<PTap*>(p);                  // [PB][ha]
    p += (sizeof(PTap) * (size_t)PB * ha + 15) & ~(size_t)15;
    long long* const ax = reinterpret_cast<long long*>(p);        // [PB][wa]
    p += sizeof(long long) * (size_t)PB * wa;
    long long* const bx = reinterpret_cast<long long*>(p);        // [PB][wb]
    p += sizeof(long long) * (size_t)PB * wb;
    float* const U = reinterpret_cast<float*>(p);                 // [ha + 2*kUPad][wa], one plane at a time
    __shared__ __align__(8) uint64_t full[kMaxStages];
    __shared__ unsigned int relcnt[kMaxStages];

    const int tid = threadIdx.x, lane = tid & 31;
    const int n_pb = (geo.n_planes + PB - 1) / PB;
    const int n_units = hb * n_pb;
    const int n_mine = blockIdx.x < n_units ? (n_units - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const uint32_t total_sl = (uint32_t)n_mine * (uint32_t)wb;
    const double cxa = 0.5 * (double)(wa - 1), cya = 0.5 * (double)(ha - 1);
    const double cxb = 0.5 * (double)(wb - 1), cyb = 0.5 * (double)(hb - 1);
    const double sx = (double)wa / (double)wb, sy = (double)ha / (double)hb;
    const RowSplit rs = row_split(ha, wa);
    const int BH = rs.R * rs.NK;                       // staged rows per slice (>= ha)
    const uint32_t stage_bytes = (uint32_t)(kPad ? BH * WS * sizeof(float) : geo.boxes * kBox * sizeof(float));

    // slice q of this CTA (q-th slice of its unit sequence) -> stage q % kStages
    auto issue = [&](uint32_t q) {
        const int s = (int)(q % kStages);
        const int k = (int)(q / (uint32_t)wb), bc = (int)(q - (uint32_t)k * wb);
        const int u = blockIdx.x + k * gridDim.x;
        const int br = u / n_pb;
        mbar_arrive_expect_tx(&full[s], stage_bytes);
        float* dst = buf0 + (size_t)s * slice_f;
        if constexpr (kPad) {
            tma_load_2d(dst, &tm, &full[s], -kPadL, (br * wb + bc) * ha);
        } else {
            const long long e = (long long)(br * wb + bc) * Ma;
            const int32_t x0 = (int32_t)(e & ~3ll);
            for (int b = 0; b < geo.boxes; ++b) tma_load_1d(dst + b * kBox, &tm, &full[s], x0 + b * kBox);
        }
    };

    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&full[i], 1);
            relcnt[i] = 0;
        }
        fence_barrier_init();
    }
    for (int i = tid; i < 2 * kUPad * wa; i += kThreads) {   // zero border rows of U
        const int row = i / wa, x = i - row * wa;
        U[(row < kUPad ? row : ha + row) * wa + x] = 0.0f;
    }
    __syncthreads();
    if (tid == 0)
        for (uint32_t q = 0; q < (uint32_t)kStages && q < total_sl; ++q) issue(q);

    const int R = rs.R, NK = rs.NK;
    constexpr int kWdiv = kWA > 0 ? kWA : 1;
    constexpr bool kFull = kWA > 0 && kThreads % kWdiv == 0 && kHA == KR * (kThreads / kWdiv);
    constexpr int kRStep = (kThreads / kWdiv) * (((kWA + 3) & ~3) + (kPad ? kPadL + kPadR : 0));
    const int c = tid % wa, rp = tid / wa;
    const bool active = kFull || rp < R;
    // rows of the image this thread owns (the U writes); it computes NK rows
    const int nk = kFull ? KR : (active ? max(0, min(KR, (ha - rp + R - 1) / R)) : 0);
    const int rstep = R * WS;
    uint32_t g = 0;          // slices of this CTA consumed so far
    int cs = 0;              // stage of slice g
    uint32_t cp = 0;         // phase parity of slice g in its stage
    int cur_pb = -1;
    for (int k = 0; k < n_mine; ++k) {
        const int u = blockIdx.x + k * gridDim.x;
        const int br = u / n_pb, pblk = u - br * n_pb, p0 = pblk * PB;
        const int np = min(PB, geo.n_planes - p0);
        if (pblk != cur_pb) {   // uniform: fixed-point x coordinates of this plane block
            for (int i = tid; i < np * wa; i += kThreads) {
                const int j = i / wa, x = i - j * wa;
                ax[i] = fix32(pl.alpha[p0 + j] * ((double)x - cxa) + cxa);
            }
            for (int i = tid; i < np * wb; i += kThreads) {
                const int j = i / wb, b = i - j * wb;
                bx[i] = fix32((pl.beta[p0 + j] * sx) * ((double)b - cxb));
            }
            __syncthreads();
            if constexpr (kTable) {   // thread (rp, c) fills column c of table rows rp, rp + r0, ...
                const int r0 = kThreads / wa;
                if (rp < r0) {
                    for (int j = 0; j < np; ++j) {
                        const long long axj = ax[j * wa + c];
                        for (int b = rp; b < wb; b += r0)
                            xtab[(j * wb + b) * wa + c] = make_xtab<kPad>(axj + bx[j * wb + b], wa, 0);
                    }
                }
                __syncthreads();
            }
            cur_pb = pblk;
        }
        // Two slices per step: the step's sum (four fused multiply-adds) is
        // Kahan-added into U.  One slice per step: each slice's sum is.
        float Ua[PB][KR], Uc[PB][KR];
#pragma unroll
        for (int j = 0; j < PB; ++j)
#pragma unroll
            for (int kk = 0; kk < KR; ++kk) Ua[j][kk] = Uc[j][kk] = 0.0f;
        for (int bc0 = 0; bc0 < wb; bc0 += NSTEP) {
            const int nsl = min(NSTEP, wb - bc0);
            // stages and phase parities of this step's slices g and g + 1
            const int s0 = cs, s1 = cs + 1 == kStages ? 0 : cs + 1;
            const uint32_t p1 = s1 == 0 ? cp ^ 1u : cp;
            bool ok = mbar_wait_bounded(&full[s0], cp, nullptr, geo.status, geo.timeout_ns);
            if (NSTEP == 2 && nsl == 2)
                ok = ok && mbar_wait_bounded(&full[s1], p1, nullptr, geo.status, geo.timeout_ns);
            if (!ok) {   // every thread stops at this same slice
                if (tid == 0)
                    for (uint32_t q = g; q < g + kStages && q < total_sl; ++q)
                        mbar_wait_bounded(&full[q % kStages], (q / kStages) & 1u, nullptr, nullptr, geo.timeout_ns);
                return;
            }
            if (nk > 0) {
                // 1-D staging: the slice starts sh elements into its buffer
                const int sh0 = kPad ? 0 : (int)(((long long)(br * wb + bc0) * Ma) & 3);
                const int sh1 = kPad ? 0 : (int)(((long long)(br * wb + bc0 + 1) * Ma) & 3);
                const float* S0 = buf0 + (size_t)s0 * slice_f + rp * WS + sh0;
                const float* S1 = buf0 + (size_t)s1 * slice_f + rp * WS + sh1;
                // rows outer, planes inner (groups of 2 or 4 planes with their
                // taps in registers); planes past the block's last take its taps
                // and rows past the image are computed from staged data, both
                // dropped at the U writes
                constexpr int PG = KR >= 8 ? (PB < 2 ? PB : 2) : (PB < 4 ? PB : 4);
                const bool two = NSTEP == 2 && nsl == 2;
#pragma unroll
                for (int g0 = 0; g0 < PB; g0 += PG) {
                    const float* qa[PG];
                    const float* qb[PG];
                    float a0[PG], a1[PG], b0[PG], b1[PG];
#pragma unroll
                    for (int jj = 0; jj < PG; ++jj) {
                        const int j = min(g0 + jj, np - 1);
                        int oa, ob = 0;
                        b0[jj] = 0.0f;
                        b1[jj] = 0.0f;
                        if constexpr (kTable) {
                            read_xtab<kPad>(&xtab[(j * wb + bc0) * wa + c], oa, a0[jj], a1[jj]);
                            if (two) read_xtab<kPad>(&xtab[(j * wb + bc0 + 1) * wa + c], ob, b0[jj], b1[jj]);
                        } else {
                            const XTab<kPad> ta = make_xtab<kPad>(ax[j * wa + c] + bx[j * wb + bc0], wa, 0);
                            read_xtab<kPad>(&ta, oa, a0[jj], a1[jj]);
                            if (two) {
                                const XTab<kPad> tb = make_xtab<kPad>(ax[j * wa + c] + bx[j * wb + bc0 + 1], wa, 0);
                                read_xtab<kPad>(&tb, ob, b0[jj], b1[jj]);
                            }
                        }
                        qa[jj] = S0 + oa;
                        qb[jj] = S1 + ob;
                    }
                    if (two) {
#pragma unroll
                        for (int kk = 0; kk < KR; ++kk) {
                            if (kFull || kk < NK) {
                                const int o = kWA ? kk * kRStep : kk * rstep;
#pragma unroll
                                for (int jj = 0; jj < PG; ++jj) {
                                    float t = __fmaf_rn(a1[jj], qa[jj][o + 1], a0[jj] * qa[jj][o]);
                                    t = __fmaf_rn(b1[jj], qb[jj][o + 1], __fmaf_rn(b0[jj], qb[jj][o], t));
                                    kahan_add(Ua[g0 + jj][kk], Uc[g0 + jj][kk], t);
                                }
                            }
                        }
                    } else {
#pragma unroll
                        for (int kk = 0; kk < KR; ++kk) {
                            if (kFull || kk < NK) {
                                const int o = kWA ? kk * kRStep : kk * rstep;
#pragma unroll
                                for (int jj = 0; jj < PG; ++jj) {
                                    const float t = __fmaf_rn(a1[jj], qa[jj][o + 1], a0[jj] * qa[jj][o]);
                                    kahan_add(Ua[g0 + jj][kk], Uc[g0 + jj][kk], t);
                                }
                            }
                        }
                    }
                }
            }
            // release the step's buffers; the last warp to do so refills them
            __syncwarp();
            if (lane == 0) {
                for (int i = 0; i < nsl; ++i) {
                    const uint32_t q = g + i;
                    const int s = i == 0 ? s0 : s1;
                    __threadfence_block();
                    if (atomicAdd(&relcnt[s], 1u) == NW - 1) {
                        relcnt[s] = 0;
                        __threadfence_block();
                        if (q + kStages < total_sl) {
                            fence_proxy_async_smem();
                            issue(q + kStages);
                        }
                    }
                }
            }
            g += nsl;
            cs = nsl == 2 ? s1 : s0;
            cp = nsl == 2 ? p1 : cp;
            if (++cs == kStages) {
                cs = 0;
                cp ^= 1u;
            }
        }

        // y-interpolation of this angular row, one plane at a time through U
        __syncthreads();   // the previous unit's U and y taps are no longer read
        for (int i = tid; i < np * ha; i += kThreads) {
            const int j = i / ha, r = i - j * ha;
            const long long uy = fix32(pl.alpha[p0 + j] * ((double)r - cya) + cya) +
                                 fix32((pl.beta[p0 + j] * sy) * ((double)br - cyb));
            PTap t = padded_tap(uy, ha);
            t.off *= wa;
            yt[i] = t;
        }
#pragma unroll
        for (int j = 0; j < PB; ++j) {
            if (j < np) {
                if (j > 0) __syncthreads();   // U of the previous plane is no longer read
#pragma unroll
                for (int kk = 0; kk < KR; ++kk)
                    if (kFull || kk < nk) U[(rp + R * kk + kUPad) * wa + c] = Ua[j][kk] - Uc[j][kk];
                __syncthreads();
                float* dst = partial + ((int64_t)br * geo.total_planes + geo.plane_offset + p0 + j) * Ma;
#pragma unroll
                for (int kk = 0; kk < KR; ++kk) {
                    if (kFull || kk < nk) {
                        const int r = rp + R * kk;
                        const PTap ty = yt[j * ha + r];
                        const float v0 = U[ty.off + c], v1 = U[ty.off + wa + c];
                        dst[(int64_t)r * wa + c] = __fmaf_rn(ty.w1, v1, ty.w0 * v0);
                    }
                }
            }
        }
    }
}

// ------------------------------------------------------------ repack
// Row pitch change for 2-D staging: dst[r * pitch + c] = src[r * wa + c] for the
// rows of every slice (the pitch's extra columns are left as they are; the
// tensor map's width is wa, so the copy reads them back as zeros).
__global__ void __launch_bounds__(256) refocus_repack_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                                             int64_t n, int wa, int pitch) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / wa;
        dst[r * pitch + (i - r * wa)] = src[i];
    }
}

// ------------------------------------------------------------ direct kernel
// Fallback for spatial images too large for the pipelined kernel's registers:
// CTA = (range of angular pixels, plane, band of output rows); each angular
// pixel's slice is staged with a zero border and its 4 taps read per output.
constexpr int kDirectThreads = 512;
template <int KR>
__global__ void __launch_bounds__(kDirectThreads) refocus_direct_kernel(const float* __restrict__ gamma,
                                                                        const RefocusGeom geo,
                                                                        const PlaneBlock pl,
                                                                        float* __restrict__ partial) {
    extern __shared__ __align__(16) float sm[];
    const int ha = geo.ha, wa = geo.wa, hb = geo.hb, wb = geo.wb;
    const int W2 = wa + 2 * kUPad;
    const int64_t Ma = (int64_t)ha * wa;
    float* slice = sm;                                                   // (ha + 4) x (wa + 4)
    PTap* xt = reinterpret_cast<PTap*>(slice + (ha + 2 * kUPad) * W2);   // [wa]
    PTap* yt = xt + wa;                                                  // [ha]
    const int tid = threadIdx.x;
    const int R = kDirectThreads / wa;
    const int c = tid % wa, rp = tid / wa;
    const bool active = rp < R;
    const int row0 = blockIdx.z * (R * KR);
    const int p = blockIdx.y;
    const double al = pl.alpha[p], be = pl.beta[p];
    const double sx = (double)wa / (double)wb, sy = (double)ha / (double)hb;
    const double cxa = 0.5 * (double)(wa - 1), cya = 0.5 * (double)(ha - 1);
    const double cxb = 0.5 * (double)(wb - 1), cyb = 0.5 * (double)(hb - 1);

    for (int i = tid; i < (ha + 2 * kUPad) * W2; i += kDirectThreads) slice[i] = 0.0f;
    float acc[KR], cmp[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k) acc[k] = cmp[k] = 0.0f;
    const int nb = hb * wb;
    const int b_begin = blockIdx.x * geo.b_per_range;
    const int b_end = min(b_begin + geo.b_per_range, nb);
    for (int b = b_begin; b < b_end; ++b) {
        __syncthreads();
        const float* src = gamma + (int64_t)b * Ma;
        if (active)
            for (int r = rp; r < ha; r += R) slice[(r + kUPad) * W2 + c + kUPad] = __ldg(src + (int64_t)r * wa + c);
        const int br = b / wb, bc = b - br * wb;
        for (int j = tid; j < wa + ha; j += kDirectThreads) {
            if (j < wa) {
                xt[j] = padded_tap(fix32(al * ((double)j - cxa) + cxa) + fix32((be * sx) * ((double)bc - cxb)), wa);
            } else {
                const int r = j - wa;
                PTap t = padded_tap(fix32(al * ((double)r - cya) + cya) + fix32((be * sy) * ((double)br - cyb)), ha);
                t.off *= W2;
                yt[r] = t;
            }
        }
        __syncthreads();
        if (active) {
            const PTap tx = xt[c];
#pragma unroll
            for (int k = 0; k < KR; ++k) {
                const int r = row0 + rp + R * k;
                if (r < ha) {
                    const PTap ty = yt[r];
                    const int base = ty.off + tx.off;
                    const float v00 = slice[base], v01 = slice[base + 1];
                    const float v10 = slice[base + W2], v11 = slice[base + W2 + 1];
                    const float top = __fmaf_rn(tx.w1, v01, tx.w0 * v00);
                    const float bot = __fmaf_rn(tx.w1, v11, tx.w0 * v10);
                    kahan_add(acc[k], cmp[k], __fmaf_rn(ty.w1, bot, ty.w0 * top));
                }
            }
        }
    }
    if (!active) return;
    float* dst = partial + ((int64_t)blockIdx.x * geo.total_planes + geo.plane_offset + p) * Ma;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
        const int r = row0 + rp + R * k;
        if (r < ha) dst[(int64_t)r * wa + c] = acc[k] - cmp[k];
    }
}

// Sum of the per-range partial images in a fixed order, Kahan-compensated in
// FP32 (error <= 2 * 2^-24 of the summed magnitudes, to first order).
__global__ void refocus_reduce_kernel(const float* __restrict__ partial, int n_ranges,
                                      int64_t per_range, float* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < per_range;
         i += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.0f, cmp = 0.0f;
        int r = 0;
        for (; r + 8 <= n_ranges; r += 8) {   // 8 loads in flight, then the adds in order
            float v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = __ldg(partial + (int64_t)(r + k) * per_range + i);
#pragma unroll
            for (int k = 0; k < 8; ++k) kahan_add(acc, cmp, v[k]);
        }
        for (; r < n_ranges; ++r) kahan_add(acc, cmp, __ldg(partial + (int64_t)r * per_range + i));
        out[i] = acc - cmp;
    }
}

template <typename K>
cudaError_t set_smem_attr(K kernel, int slot) {
    static bool done[64][64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || slot < 0 || slot >= 64) return cudaErrorInvalidValue;
    if (!done[slot][dev]) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e != cudaSuccess) return e;
        done[slot][dev] = true;
    }
    return cudaSuccess;
}

constexpr size_t kSmemCap = 220 * 1024;

// 1-D staging: 256-element boxes covering the slice from the 16-byte boundary
// at or below its start (and one value past it when wa == 1).
int box_rows(int ha, int wa) {
    const RowSplit rs = row_split(ha, wa);
    return rs.R * rs.NK;
}

int pipe_boxes(int ha, int wa) {
    const int64_t ma = (int64_t)box_rows(ha, wa) * wa;
    const int64_t lead = (ma % 4 == 0) ? 0 : 3;
    const int64_t tail = (wa == 1) ? 1 : 0;
    return (int)((lead + ma + tail + kBox - 1) / kBox);
}

struct PipeCfg {
    bool pad;      // 2-D padded staging (else 1-D boxes)
    bool table;    // per-plane-block x-tap table in shared memory
    int pb, nstep, stages, kr;
};

int pitch4(int wa) { return (wa + 3) & ~3; }

bool pad_staging(int ha, int wa) { return pitch4(wa) + kPadL + kPadR <= 256 && box_rows(ha, wa) <= 256; }

int slice_floats(int ha, int wa, bool pad) {
    return pad ? ((box_rows(ha, wa) * (pitch4(wa) + kPadL + kPadR) + 31) & ~31) : pipe_boxes(ha, wa) * kBox;
}

size_t pipe_smem(int ha, int wa, int wb, const PipeCfg& c) {
    size_t b = 128 + sizeof(float) * (size_t)c.stages * slice_floats(ha, wa, c.pad);
    if (c.table) b += (c.pad ? sizeof(XTab<true>) : sizeof(XTab<false>)) * (size_t)c.pb * wb * wa;
    b += (sizeof(PTap) * (size_t)c.pb * ha + 15) & ~(size_t)15;
    b += sizeof(long long) * (size_t)c.pb * (wa + wb);
    b += sizeof(float) * (size_t)(ha + 2 * kUPad) * wa;
    return b;
}

int rows_per_thread(int ha, int wa) { return wa <= kThreads ? row_split(ha, wa).NK : 1 << 30; }

template <int KR, int PB, int NSTEP, int kST, bool kPad, bool kTable, int kWA = 0, int kHA = 0>
cudaError_t launch_pipe(const CUtensorMap* tm, const RefocusGeom& geo, const PlaneBlock& pl, float* partial,
                        size_t smem, int grid, cudaStream_t st, int slot) {
    auto kern = refocus_pipe_kernel<KR, PB, NSTEP, kST, kPad, kTable, kWA, kHA>;
    cudaError_t e = set_smem_attr(kern, slot);
    if (e != cudaSuccess) return e;
    kern<<<grid, kThreads, smem, st>>>(*tm, geo, pl, partial);
    return cudaGetLastError();
}

template <int KR>
cudaError_t launch_direct(const float* g, const RefocusGeom& geo, const PlaneBlock& pl,
                          float* partial, int zchunks, size_t smem, cudaStream_t st, int slot) {
    cudaError_t e = set_smem_attr(refocus_direct_kernel<KR>, slot);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)geo.n_ranges, (unsigned)geo.n_planes, (unsigned)zchunks);
    refocus_direct_kernel<KR><<<grid, kDirectThreads, smem, st>>>(g, geo, pl, partial);
    return cudaGetLastError();
}

// Kernel choice for an image shape.
struct RefocusVariant {
    bool pipe;     // pipelined kernel (else direct)
    PipeCfg cfg;
};

RefocusVariant refocus_variant(int ha, int wa, int wb) {
    RefocusVariant v{false, {false, false, 1, 1, 2, 1}};
    if (wa > kThreads) return v;
    const bool pad = pad_staging(ha, wa);
    const int rows = rows_per_thread(ha, wa);
    // candidates in order of preference; the first whose rows per thread and
    // shared memory fit is used
    const int kr8 = rows <= 1 ? 1 : rows <= 2 ? 2 : 4;
    const PipeCfg cands[] = {
        {pad, true, 8, 2, 4, kr8},                                  // <= 4 rows: 8 planes per unit
        {pad, true, 4, 2, 4, 8},                                    // <= 8 rows: 4 planes per unit
        {pad, true, 2, 2, 4, 16}, {pad, false, 2, 2, 4, 16},        // <= 16 rows: 2 planes per unit
        {pad, true, 2, 2, 3, 16}, {pad, false, 2, 2, 3, 16},
        {pad, true, 1, 2, 4, 32}, {pad, false, 1, 2, 4, 32},        // <= 32 rows: 1 plane per unit
        {pad, true, 1, 2, 3, 32}, {pad, false, 1, 2, 3, 32},
        {pad, false, 1, 1, 2, 32},                                  // one slice per step, 2 stages
    };
    for (const PipeCfg& c : cands) {
        if (rows > c.kr) continue;
        if (c.pb == 8 && rows > 4) continue;
        if (pipe_smem(ha, wa, wb, c) <= kSmemCap) return {true, c};
    }
    return v;
}

template <bool kPad>
cudaError_t launch_pipe_cfg(const PipeCfg& c, const CUtensorMap* tm, const RefocusGeom& geo, const PlaneBlock& pl,
                            float* partial, size_t smem, int grid, cudaStream_t st) {
    const int base = kPad ? 0 : 20;
    if (c.pb == 8) {
        if constexpr (kPad) {   // compile-time shape of a common square detector size
            if (geo.wa == 32 && geo.ha == 32)
                return launch_pipe<2, 8, 2, 4, true, true, 32, 32>(tm, geo, pl, partial, smem, grid, st, base + 0);
        }
        switch (c.kr) {
            case 1: return launch_pipe<1, 8, 2, 4, kPad, true>(tm, geo, pl, partial, smem, grid, st, base + 1);
            case 2: return launch_pipe<2, 8, 2, 4, kPad, true>(tm, geo, pl, partial, smem, grid, st, base + 2);
            default: return launch_pipe<4, 8, 2, 4, kPad, true>(tm, geo, pl, partial, smem, grid, st, base + 3);
        }
    }
    if (c.pb == 4) {
        if constexpr (kPad) {
            if (geo.wa == 64 && geo.ha == 64)
                return launch_pipe<8, 4, 2, 4, true, true, 64, 64>(tm, geo, pl, partial, smem, grid, st, base + 4);
        }
        return launch_pipe<8, 4, 2, 4, kPad, true>(tm, geo, pl, partial, smem, grid, st, base + 5);
    }
    if (c.pb == 2)
        return c.table ? launch_pipe<16, 2, 2, 0, kPad, true>(tm, geo, pl, partial, smem, grid, st, base + 6)
                       : launch_pipe<16, 2, 2, 0, kPad, false>(tm, geo, pl, partial, smem, grid, st, base + 7);
    if (c.nstep == 2)
        return c.table ? launch_pipe<32, 1, 2, 0, kPad, true>(tm, geo, pl, partial, smem, grid, st, base + 8)
                       : launch_pipe<32, 1, 2, 0, kPad, false>(tm, geo, pl, partial, smem, grid, st, base + 9);
    return launch_pipe<32, 1, 1, 2, kPad, false>(tm, geo, pl, partial, smem, grid, st, base + 10);
}

}  // namespace

bool refocus_pipelined(int ha, int wa, int wb) { return refocus_variant(ha, wa, wb).pipe; }

int refocus_staging(int ha, int wa, int wb) {
    const RefocusVariant v = refocus_variant(ha, wa, wb);
    if (!v.pipe) return 0;
    return v.cfg.pad ? 2 : 1;
}

int refocus_box_rows(int ha, int wa) { return box_rows(ha, wa); }

int refocus_pitch(int ha, int wa, int wb) {
    return refocus_staging(ha, wa, wb) == 2 && wa % 4 != 0 ? pitch4(wa) : 0;
}

cudaError_t launch_refocus_repack(const float* gamma_f32, float* dst, int64_t rows, int wa, int pitch,
                                  int sm_count, cudaStream_t st) {
    const int64_t n = rows * wa;
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = 8 * (int64_t)sm_count;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    refocus_repack_kernel<<<(unsigned)blocks, 256, 0, st>>>(gamma_f32, dst, n, wa, pitch);
    return cudaGetLastError();
}

size_t refocus_smem_bytes(int ha, int wa, int wb) {
    const RefocusVariant v = refocus_variant(ha, wa, wb);
    if (v.pipe) return pipe_smem(ha, wa, wb, v.cfg);
    return sizeof(float) * (size_t)(ha + 2 * kUPad) * (wa + 2 * kUPad) + sizeof(PTap) * ((size_t)wa + ha);
}

int refocus_ranges(int ha, int wa, int hb, int wb, int n_planes, int sm_count) {
    // pipelined kernel: one range per angular row; direct kernel: ranges of
    // angular pixels sized to fill the GPU
    if (refocus_pipelined(ha, wa, wb)) return hb;
    const int units = hb * wb;
    int target = (4 * sm_count + n_planes - 1) / (n_planes > 0 ? n_planes : 1);
    if (target < 1) target = 1;
    if (target > units) target = units;
    const int per = (units + target - 1) / target;
    return (units + per - 1) / per;
}

int refocus_range_size(int ha, int wa, int hb, int wb, int n_ranges) {
    if (refocus_pipelined(ha, wa, wb)) return 1;
    return (hb * wb + n_ranges - 1) / n_ranges;
}

cudaError_t launch_refocus(const float* gamma_f32, const CUtensorMap* tm, const RefocusGeom& geo_in,
                           const PlaneBlock& pl, float* partial, int sm_count, cudaStream_t st) {
    const size_t smem = refocus_smem_bytes(geo_in.ha, geo_in.wa, geo_in.wb);
    const RefocusVariant v = refocus_variant(geo_in.ha, geo_in.wa, geo_in.wb);
    RefocusGeom geo = geo_in;
    if (v.pipe) {
        if (tm == nullptr) return cudaErrorInvalidValue;
        geo.boxes = pipe_boxes(geo.ha, geo.wa);
        geo.slice_f = slice_floats(geo.ha, geo.wa, v.cfg.pad);
        geo.stages = v.cfg.stages;
        const int units = geo.hb * ((geo.n_planes + v.cfg.pb - 1) / v.cfg.pb);
        const int grid = units < sm_count ? units : sm_count;
        return v.cfg.pad ? launch_pipe_cfg<true>(v.cfg, tm, geo, pl, partial, smem, grid, st)
                         : launch_pipe_cfg<false>(v.cfg, tm, geo, pl, partial, smem, grid, st);
    }
    const int R = kDirectThreads / geo.wa;
    int kr = 1;
    while (kr < 16 && R * kr < geo.ha) kr *= 2;
    const int zchunks = (geo.ha + R * kr - 1) / (R * kr);
    switch (kr) {
        case 1: return launch_direct<1>(gamma_f32, geo, pl, partial, zchunks, smem, st, 40);
        case 2: return launch_direct<2>(gamma_f32, geo, pl, partial, zchunks, smem, st, 41);
        case 4: return launch_direct<4>(gamma_f32, geo, pl, partial, zchunks, smem, st, 42);
        case 8: return launch_direct<8>(gamma_f32, geo, pl, partial, zchunks, smem, st, 43);
        default: return launch_direct<16>(gamma_f32, geo, pl, partial, zchunks, smem, st, 44);
    }
}

cudaError_t launch_refocus_reduce(const float* partial, int n_ranges, int64_t per_range,
                                  float* out, cudaStream_t st) {
    int64_t blocks = (per_range + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    refocus_reduce_kernel<<<(unsigned)blocks, 256, 0, st>>>(partial, n_ranges, per_range, out);
    return cudaGetLastError();
}

}  // namespace cpi
