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
// only on (r, br).  So the refocusing runs as two stages:
//   x stage:  U_(p,br)(y, c) = sum_bc  wx0 S_(br,bc)(y, xo) + wx1 S_(br,bc)(y, xo + 1)
//             (every slice value staged once is used by a block of planes);
//   y stage:  out_p(r, c) = sum_br  wy0 U_(p,br)(yo, c) + wy1 U_(p,br)(yo + 1, c).
// The x stage holds almost all the work (P * Ma * Mb samples of two taps); the y
// stage has a factor wb less and reads U once from memory.
//
// Coordinates are computed on the fly inside the kernels (the point of Section
// 4.1) in 32.32 fixed point.  x stage: u = A(c) + B(bc), A = alpha*(c - cxa) + cxa
// rounded once from FP64 per output column, B stepped from angular column to
// angular column by the fixed-point increment beta*sx (error below wb * 2^-33
// pixels).  y stage: both parts rounded once from FP64.  The fraction is rounded
// to 24 bits, so both weights (1 - f, f) are exact FP32 numbers that sum to 1.
// Sums are FP32: the two slices of a step are combined with fused multiply-adds
// and the step sums Kahan-added into U; the y stage Kahan-adds over the angular
// rows in a fixed order, so the result is deterministic.
//
// Layout: Gamma arrives slice-major, float [Mb][Ma]; slice b is one contiguous
// spatial image, of which the x stage stages bands of rows by TMA.
//
// This file is compiled without FMA contraction: the Kahan steps depend on the
// written rounding order; the products use explicit fmaf.
#include <cstring>

#include "kernels.cuh"
#include "ptx.cuh"

namespace cpi {
namespace {

// ------------------------------------------------------------ coordinates
__device__ __forceinline__ long long fix32(double v) { return __double2ll_rn(v * 4294967296.0); }

__device__ __forceinline__ void kahan_add(float& acc, float& cmp, float v) {
    const float y = v - cmp;
    const float t = acc + y;
    cmp = (t - acc) - y;
    acc = t;
}

// Two FP32 lanes in one 64-bit register pair, for the packed f32x2 instructions
// of sm_100+ (each lane is an ordinary IEEE round-to-nearest FP32 operation).
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpk2(f32x2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// kahan_add on both lanes
__device__ __forceinline__ void kahan_add2(f32x2& acc, f32x2& cmp, f32x2 v) {
    const f32x2 y = sub2(v, cmp);
    const f32x2 t = add2(acc, y);
    cmp = sub2(sub2(t, acc), y);
    acc = t;
}

// Taps of one axis from a 32.32 fixed-point coordinate: integer part i and the
// fraction rounded to 24 bits; taps outside [0, n) get weight 0 and are moved
// onto in-grid rows, so no read leaves the image.
struct YTap {
    int o0, o1;         // element offsets of the two rows (row * wa)
    float w0, w1;
};
__device__ __forceinline__ YTap y_tap(long long u, int n, int wa) {
    const long long u24 = (u + 128) >> 8;
    const int i = (int)(u24 >> 24);
    const float f = (float)(int)(u24 & 0xFFFFFF) * 0x1p-24f;
    const bool v0 = i >= 0 && i < n, v1 = i + 1 >= 0 && i + 1 < n;
    const int r0 = min(max(i, 0), n - 1), r1 = min(max(i + 1, 0), n - 1);
    return {r0 * wa, r1 * wa, v0 ? 1.0f - f : 0.0f, v1 ? f : 0.0f};
}

// ------------------------------------------------------------ x stage
// Persistent: one CTA of kBandThreads per SM walks the work units blockIdx.x,
// blockIdx.x + gridDim.x, ...  A unit is (angular row br, block of PB planes,
// band of BH = R * KR rows of the spatial image); units are ordered br-major, so
// the CTAs running at one time stage the slices of the same angular row (L2
// reuse).  Each unit streams the wb slices (br, 0 .. wb-1) of its band through
// `stages` shared-memory buffers, one TMA copy each, completion counted on
// full[stage]; the last warp to finish with a buffer (a shared counter per
// stage) issues the copy of the slice `stages` further on into it, so no thread
// ever waits for a free buffer.
//
// Staging: the band's rows with WS floats per row, a zero border of pad_l
// columns on the left and at least pad_l on the right (the columns outside
// 0 .. wa-1 arrive as TMA out-of-bounds fill: taps outside the grid read
// zeros, no test in the loop).  wa <= 248: a 2-D box {WS, BH} from column -4;
// wider rows: a 3-D view of each row as 16-float chunks, box {16, WS/16, BH}
// from chunk -1 (pad 16).  Rows past the slice's ha are the next slice's (or
// zero fill past Gamma's end); their sums are dropped.
//
// Thread t owns column c = t % cwt and rows rp * KR .. rp * KR + KR - 1 of the
// band (rp = t / cwt < R).  For each step of two slices it forms the x taps of
// its column for the PB planes (fixed point, in registers), then, rows outer
// and planes inner, adds the step's two samples with fused multiply-adds and
// Kahan-adds the sum into U.  After the unit's last slice it writes U for its
// rows: ubuf[plane][br][row][c].
//
// Every wait is bounded (the device status word records a time out).  A slice
// that never arrives stops every thread at that same slice.
constexpr int kBandThreads = 512;
constexpr int kBandMaxStages = 8;

struct BandGeom {
    int32_t ha, wa, hb, wb;
    int32_t n_planes;          // planes of this launch
    int32_t cwt, R, BH;        // column threads, row sets, band rows (R * KR)
    int32_t n_bands, n_pb;     // bands per image, plane blocks
    int32_t pad_l;             // zero columns left of a staged row (4 or 16)
    int32_t mode3d;            // 3-D chunked staging (rows wider than 248)
    int32_t stages;            // stage buffers (<= kBandMaxStages)
    uint32_t stage_bytes;      // BH * WS * 4
    const long long* xcol;     // [n_planes][kBandThreads]: column part of each column thread's x coordinate
    const long long* xang;     // [n_planes][2]: angular part at bc = 0, and its step per angular column
    unsigned int* status;
    unsigned long long timeout_ns;
};

// Fixed-point x coordinates of a launch's planes (32.32, each rounded once from
// FP64): xcol[p][c] = fix(alpha (c - cxa) + cxa) + the 24-bit rounding bias and
// the staging pad, for every column thread c; xang[p] = {fix(beta sx (0 - cxb)),
// fix(beta sx)}.
__global__ void __launch_bounds__(256) refocus_xtables_kernel(const PlaneBlock pl, int n_planes, int wa, int wb,
                                                              int pad_l, long long* __restrict__ xcol,
                                                              long long* __restrict__ xang) {
    const double cxa = 0.5 * (double)(wa - 1), cxb = 0.5 * (double)(wb - 1);
    const double sx = (double)wa / (double)wb;
    const long long bias = 128ll + ((long long)pad_l << 32);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_planes * kBandThreads; i += gridDim.x * blockDim.x) {
        const int p = i / kBandThreads, c = i - p * kBandThreads;
        xcol[i] = fix32(pl.alpha[p] * ((double)c - cxa) + cxa) + bias;
        if (c == 0) {
            const double bs = pl.beta[p] * sx;
            xang[2 * p] = fix32(bs * (0.0 - cxb));
            xang[2 * p + 1] = fix32(bs);
        }
    }
}

// PT planes per thread: a unit holds PB = PT planes, so every staged value
// serves PB planes while each thread keeps the sums of all of them.
template <int WS, int KR, int PT>
__global__ void __launch_bounds__(kBandThreads, 1) refocus_band_kernel(const __grid_constant__ CUtensorMap tm,
                                                                           const BandGeom g, const PlaneBlock pl,
                                                                           float* __restrict__ ubuf) {
    constexpr int NW = kBandThreads / 32;
    constexpr int PB = PT;
    static_assert(PT % 2 == 0, "planes are processed in pairs");
    extern __shared__ __align__(128) float sm_raw[];
    float* const buf0 =
        sm_raw + (((128u - (static_cast<uint32_t>(__cvta_generic_to_shared(sm_raw)) & 127u)) & 127u) >> 2);
    __shared__ __align__(8) uint64_t full[kBandMaxStages];
    __shared__ unsigned int relcnt[kBandMaxStages];

    const int ha = g.ha, wa = g.wa, hb = g.hb, wb = g.wb;
    const int stages = g.stages;
    const int slice_f = (g.BH * WS + 31) & ~31;    // floats per stage buffer (128-byte multiple)
    const int tid = threadIdx.x, lane = tid & 31;
    const int c = tid % g.cwt, rp = tid / g.cwt;
    const bool active = rp < g.R;
    const int per_br = g.n_pb * g.n_bands;
    const int n_units = hb * per_br;
    const int n_mine = (int)blockIdx.x < n_units ? (n_units - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const uint32_t total_sl = (uint32_t)n_mine * (uint32_t)wb;

    // slice q of this CTA (q-th slice of its unit sequence) -> stage q % stages
    auto issue = [&](uint32_t q) {
        const int s = (int)(q % (uint32_t)stages);
        const int k = (int)(q / (uint32_t)wb), bc = (int)(q - (uint32_t)k * wb);
        const int u = (int)blockIdx.x + k * (int)gridDim.x;
        const int br = u / per_br, band = (u - br * per_br) % g.n_bands;
        const int y = (br * wb + bc) * ha + band * g.BH;
        mbar_arrive_expect_tx(&full[s], g.stage_bytes);
        float* dst = buf0 + (size_t)s * slice_f;
        if (g.mode3d) tma_load_3d(dst, &tm, &full[s], 0, -1, y);
        else tma_load_2d(dst, &tm, &full[s], -4, y);
    };

    if (tid == 0) {
        for (int i = 0; i < stages; ++i) {
            mbar_init(&full[i], 1);
            relcnt[i] = 0;
        }
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0)
        for (uint32_t q = 0; q < (uint32_t)stages && q < total_sl; ++q) issue(q);

    const int lo_b = g.pad_l - 2, hi_b = g.pad_l + wa;    // clamp of a tap's staged column
    uint32_t gs = 0;      // slices of this CTA consumed so far
    int cs = 0;           // stage of slice gs
    uint32_t cp = 0;      // phase parity of slice gs in its stage
    for (int k = 0; k < n_mine; ++k) {
        const int u = (int)blockIdx.x + k * (int)gridDim.x;
        const int br = u / per_br, rest = u - br * per_br;
        const int pblk = rest / g.n_bands, band = rest - pblk * g.n_bands;
        const int p0 = pblk * PB;
        const int np = min(PB, g.n_planes - p0);
        // running coordinate of this column at angular column bc (from bc = 0):
        // the column's part (with the 24-bit rounding bias and the staging pad)
        // plus the angular part, stepped by dB per angular column
        long long X[PT], dB[PT];
#pragma unroll
        for (int j = 0; j < PT; ++j) {
            const int pj = p0 + min(j, np - 1);
            X[j] = __ldg(g.xcol + (size_t)pj * kBandThreads + c) + __ldg(g.xang + 2 * pj);
            dB[j] = __ldg(g.xang + 2 * pj + 1);
        }
        // sums of plane pairs (2q, 2q + 1) in the two lanes of a packed register
        f32x2 U[PT / 2][KR], C[PT / 2][KR];
#pragma unroll
        for (int q = 0; q < PT / 2; ++q)
#pragma unroll
            for (int kk = 0; kk < KR; ++kk) U[q][kk] = C[q][kk] = 0ull;
        for (int bc0 = 0; bc0 < wb; bc0 += 2) {
            const int nsl = min(2, wb - bc0);
            const int s0 = cs, s1 = cs + 1 == stages ? 0 : cs + 1;
            const uint32_t p1 = s1 == 0 ? cp ^ 1u : cp;
            bool ok = mbar_wait_bounded(&full[s0], cp, nullptr, g.status, g.timeout_ns);
            if (nsl == 2) ok = ok && mbar_wait_bounded(&full[s1], p1, nullptr, g.status, g.timeout_ns);
            if (!ok) {   // every thread stops at this same slice
                if (tid == 0)
                    for (uint32_t q = gs; q < gs + (uint32_t)stages && q < total_sl; ++q)
                        mbar_wait_bounded(&full[q % (uint32_t)stages], (q / (uint32_t)stages) & 1u, nullptr, nullptr,
                                          g.timeout_ns);
                return;
            }
            if (active) {
                const float* S0 = buf0 + (size_t)s0 * slice_f + rp * KR * WS;
                const float* S1 = buf0 + (size_t)s1 * slice_f + rp * KR * WS;
                const f32x2 one2 = pk2(1.0f, 1.0f);
                // one plane pair at a time: its taps live in registers while its
                // rows are summed (lane l of every packed value: plane 2q + l)
#pragma unroll
                for (int q = 0; q < PT / 2; ++q) {
                    const float* pa[2];
                    const float* pb[2];
                    float fa[2], fb[2];
#pragma unroll
                    for (int l = 0; l < 2; ++l) {
                        const int j = 2 * q + l;
                        const long long ua = X[j];
                        const long long ub = ua + dB[j];
                        X[j] = ub + dB[j];
                        pa[l] = S0 + min(max((int)(ua >> 32), lo_b), hi_b);
                        fa[l] = (float)((uint32_t)ua >> 8) * 0x1p-24f;
                        pb[l] = S1 + min(max((int)(ub >> 32), lo_b), hi_b);
                        fb[l] = (float)((uint32_t)ub >> 8) * 0x1p-24f;
                    }
                    const f32x2 a1 = pk2(fa[0], fa[1]), b1 = pk2(fb[0], fb[1]);
                    const f32x2 a0 = sub2(one2, a1), b0 = sub2(one2, b1);
                    if (nsl == 2) {
#pragma unroll
                        for (int kk = 0; kk < KR; ++kk) {
                            const int o = kk * WS;
                            const f32x2 va0 = pk2(pa[0][o], pa[1][o]), va1 = pk2(pa[0][o + 1], pa[1][o + 1]);
                            const f32x2 vb0 = pk2(pb[0][o], pb[1][o]), vb1 = pk2(pb[0][o + 1], pb[1][o + 1]);
                            f32x2 t = fma2(a1, va1, mul2(a0, va0));
                            t = fma2(b1, vb1, fma2(b0, vb0, t));
                            kahan_add2(U[q][kk], C[q][kk], t);
                        }
                    } else {
#pragma unroll
                        for (int kk = 0; kk < KR; ++kk) {
                            const int o = kk * WS;
                            const f32x2 va0 = pk2(pa[0][o], pa[1][o]), va1 = pk2(pa[0][o + 1], pa[1][o + 1]);
                            kahan_add2(U[q][kk], C[q][kk], fma2(a1, va1, mul2(a0, va0)));
                        }
                    }
                }
            }
            // release the step's buffers; the last warp to do so refills them
            __syncwarp();
            if (lane == 0) {
                for (int i = 0; i < nsl; ++i) {
                    const uint32_t q = gs + i;
                    const int s = i == 0 ? s0 : s1;
                    __threadfence_block();
                    if (atomicAdd(&relcnt[s], 1u) == NW - 1) {
                        relcnt[s] = 0;
                        __threadfence_block();
                        if (q + stages < total_sl) {
                            fence_proxy_async_smem();
                            issue(q + stages);
                        }
                    }
                }
            }
            gs += nsl;
            cs = nsl == 2 ? s1 : s0;
            cp = nsl == 2 ? p1 : cp;
            if (++cs == stages) {
                cs = 0;
                cp ^= 1u;
            }
        }
        // this angular row's x-interpolated images for the unit's planes and rows
        if (active && c < wa) {
            const int64_t Ma = (int64_t)ha * wa;
#pragma unroll
            for (int q = 0; q < PT / 2; ++q) {
#pragma unroll
                for (int kk = 0; kk < KR; ++kk) {
                    const int row = band * g.BH + rp * KR + kk;
                    float v[2];
                    unpk2(sub2(U[q][kk], C[q][kk]), v[0], v[1]);
#pragma unroll
                    for (int l = 0; l < 2; ++l) {
                        const int j = 2 * q + l;
                        if (j < np && row < ha)
                            ubuf[((int64_t)(p0 + j) * hb + br) * Ma + (int64_t)row * wa + c] = v[l];
                    }
                }
            }
        }
    }
}

// ------------------------------------------------------------ y stage
// out[p][r][c] = sum over br of wy0 U[p][br][yo][c] + wy1 U[p][br][yo + 1][c],
// Kahan-added over br in order.  CTA = (RB output rows, plane); the y taps of its
// rows for every angular row are formed first (FP64 -> 32.32 fixed point) into
// shared memory.  Rows whose width is a multiple of 4 are read as 16-byte
// vectors (four adjacent outputs per thread).
constexpr int kYThreads = 256;
struct YGeom {
    int32_t ha, wa, hb, RB;
    int32_t plane_offset;      // index of this launch's first plane in `out`
};

__global__ void __launch_bounds__(kYThreads) refocus_ystage_kernel(const float* __restrict__ ubuf, const YGeom g,
                                                                   const PlaneBlock pl, float* __restrict__ out) {
    extern __shared__ __align__(16) YTap ytab[];     // [RB][hb]
    const int ha = g.ha, wa = g.wa, hb = g.hb, RB = g.RB;
    const int p = blockIdx.y;
    const int r0 = blockIdx.x * RB;
    const double al = pl.alpha[p], be = pl.beta[p];
    const double cya = 0.5 * (double)(ha - 1), cyb = 0.5 * (double)(hb - 1);
    const double sy = (double)ha / (double)hb;
    for (int i = threadIdx.x; i < RB * hb; i += kYThreads) {
        const int rr = i / hb, br = i - rr * hb;
        const long long uy = fix32(al * ((double)(r0 + rr) - cya) + cya) + fix32((be * sy) * ((double)br - cyb));
        ytab[i] = y_tap(uy, ha, wa);
    }
    __syncthreads();
    const int64_t Ma = (int64_t)ha * wa;
    const float* src = ubuf + (int64_t)p * hb * Ma;
    if ((wa & 3) == 0) {   // four adjacent columns per thread, 16-byte loads
        const int wq = wa >> 2;
        for (int idx = threadIdx.x; idx < RB * wq; idx += kYThreads) {
            const int rr = idx / wq, c = (idx - rr * wq) * 4;
            const int r = r0 + rr;
            if (r >= ha) continue;
            const YTap* t = ytab + rr * hb;
            float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f}, cmp[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            const float* s = src + c;
#pragma unroll 4
            for (int br = 0; br < hb; ++br) {
                const YTap y = t[br];
                const float4 v0 = __ldg(reinterpret_cast<const float4*>(s + y.o0));
                const float4 v1 = __ldg(reinterpret_cast<const float4*>(s + y.o1));
                kahan_add(acc[0], cmp[0], __fmaf_rn(y.w1, v1.x, y.w0 * v0.x));
                kahan_add(acc[1], cmp[1], __fmaf_rn(y.w1, v1.y, y.w0 * v0.y));
                kahan_add(acc[2], cmp[2], __fmaf_rn(y.w1, v1.z, y.w0 * v0.z));
                kahan_add(acc[3], cmp[3], __fmaf_rn(y.w1, v1.w, y.w0 * v0.w));
                s += Ma;
            }
            float* o = out + ((int64_t)(g.plane_offset + p) * ha + r) * wa + c;
#pragma unroll
            for (int k = 0; k < 4; ++k) o[k] = acc[k] - cmp[k];
        }
        return;
    }
    for (int idx = threadIdx.x; idx < RB * wa; idx += kYThreads) {
        const int rr = idx / wa, c = idx - rr * wa;
        const int r = r0 + rr;
        if (r >= ha) continue;
        const YTap* t = ytab + rr * hb;
        float acc = 0.0f, cmp = 0.0f;
        const float* s = src + c;
#pragma unroll 4
        for (int br = 0; br < hb; ++br) {
            const YTap y = t[br];
            const float v0 = __ldg(s + y.o0), v1 = __ldg(s + y.o1);
            kahan_add(acc, cmp, __fmaf_rn(y.w1, v1, y.w0 * v0));
            s += Ma;
        }
        out[((int64_t)(g.plane_offset + p) * ha + r) * wa + c] = acc - cmp;
    }
}

// ------------------------------------------------------------ repack
// dst[r * pitch + c] = src[r * wa + c] for c < wa and 0 for wa <= c < pitch:
// rows padded to a multiple of 4 (2-D staging) or 16 floats (3-D staging).
__global__ void __launch_bounds__(256) refocus_repack_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                                             int64_t rows, int wa, int pitch) {
    const int64_t n = rows * pitch;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / pitch;
        const int c = (int)(i - r * pitch);
        dst[i] = c < wa ? src[r * wa + c] : 0.0f;
    }
}

// ------------------------------------------------------------ host planning
constexpr size_t kSmemCap = 220 * 1024;
constexpr int kMaxBandWidth = 512;

// Staged row pitch classes (compile-time strides): 2-D staging for rows up to
// 248 wide, 3-D chunked staging up to 512.
constexpr int kWS2d[] = {40, 72, 104, 136, 200, 256};
constexpr int kWS3d[] = {288, 416, 544};

struct BandPlan {
    bool ok;
    int WS, KR, PB;
    int cwt, R, BH, n_bands, pad_l, mode3d, stages;
    int pitch;              // row pitch (floats) of the Gamma copy the tensor map reads; 0: Gamma itself
    size_t smem;
};

BandPlan band_plan(int ha, int wa) {
    BandPlan b{};
    if (wa < 1 || wa > kMaxBandWidth || ha < 1) return b;
    b.cwt = 32 * ((wa + 31) / 32);
    b.R = kBandThreads / b.cwt;
    if (wa <= 248) {
        const int need = ((wa + 3) & ~3) + 8;
        for (int ws : kWS2d)
            if (ws >= need) {
                b.WS = ws;
                break;
            }
        b.pad_l = 4;
        b.mode3d = 0;
        b.pitch = wa % 4 == 0 ? 0 : (wa + 3) & ~3;
    } else {
        const int p16 = (wa + 15) & ~15;
        for (int ws : kWS3d)
            if (ws >= p16 + 32) {
                b.WS = ws;
                break;
            }
        b.pad_l = 16;
        b.mode3d = 1;
        b.pitch = wa % 16 == 0 ? 0 : p16;
    }
    if (b.WS == 0) return b;
    b.KR = 8;
    b.PB = 4;
    if (b.WS == 40 && ha <= 2 * b.R) {   // short, narrow images: fewer rows per thread, more planes
        b.KR = 2;
        b.PB = 8;
    }
    b.BH = b.R * b.KR;
    b.n_bands = (ha + b.BH - 1) / b.BH;
    const size_t stage_bytes = (((size_t)b.BH * b.WS + 31) & ~(size_t)31) * sizeof(float);
    int st = (int)((200 * 1024) / stage_bytes);
    b.stages = st > kBandMaxStages ? kBandMaxStages : st;
    if (b.stages < 3) return b;
    b.smem = 128 + (size_t)b.stages * stage_bytes;
    b.ok = true;
    return b;
}

template <typename K>
cudaError_t set_smem_attr(K kernel, int slot, size_t bytes) {
    static bool done[64][64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || slot < 0 || slot >= 64) return cudaErrorInvalidValue;
    if (!done[slot][dev]) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        done[slot][dev] = true;
    }
    return cudaSuccess;
}

template <int WS, int KR, int PT>
cudaError_t launch_band_t(const CUtensorMap* tm, const BandGeom& g, const PlaneBlock& pl, float* ubuf, size_t smem,
                          int grid, cudaStream_t st, int slot) {
    auto kern = refocus_band_kernel<WS, KR, PT>;
    cudaError_t e = set_smem_attr(kern, slot, kSmemCap);
    if (e != cudaSuccess) return e;
    kern<<<grid, kBandThreads, smem, st>>>(*tm, g, pl, ubuf);
    return cudaGetLastError();
}

cudaError_t launch_band(const BandPlan& b, const CUtensorMap* tm, const BandGeom& g, const PlaneBlock& pl,
                        float* ubuf, int grid, cudaStream_t st) {
    if (b.KR == 2) return launch_band_t<40, 2, 8>(tm, g, pl, ubuf, b.smem, grid, st, 0);
    switch (b.WS) {
        case 40: return launch_band_t<40, 8, 4>(tm, g, pl, ubuf, b.smem, grid, st, 1);
        case 72: return launch_band_t<72, 8, 4>(tm, g, pl, ubuf, b.smem, grid, st, 2);
        case 104: return launch_band_t<104, 8, 4>(tm, g, pl, ubuf, b.smem, grid, st, 3);
        case 136: return launch_band_t<136, 8, 4>(tm, g, pl, ubuf, b.smem, grid, st, 4);
        case 200: return launch_band_t<200, 8, 4>(tm, g, pl, ubuf, b.smem, grid, st, 5);
        case 256: return launch_band_t<256, 8, 4>(tm, g, pl, ubuf, b.smem, grid, st, 6);
        case 288: return launch_band_t<288, 8, 4>(tm, g, pl, ubuf, b.smem, grid, st, 7);
        case 416: return launch_band_t<416, 8, 4>(tm, g, pl, ubuf, b.smem, grid, st, 8);
        case 544: return launch_band_t<544, 8, 4>(tm, g, pl, ubuf, b.smem, grid, st, 9);
        default: return cudaErrorInvalidValue;
    }
}

// Output rows per y-stage CTA: its y taps (rows x hb entries) fit in 200 KiB.
int y_rows_per_cta(int hb) {
    int rb = (int)((200 * 1024) / ((size_t)hb * sizeof(YTap)));
    if (rb > 8) rb = 8;
    return rb;
}

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// x-coordinate tables of one launch (at the end of the workspace)
size_t xtables_bytes() {
    return round256((size_t)kRefocusMaxPlanesPerLaunch * kBandThreads * sizeof(long long)) +
           round256((size_t)kRefocusMaxPlanesPerLaunch * 2 * sizeof(long long));
}

}  // namespace

bool refocus_supported(int ha, int wa, int hb, int wb) {
    if (ha < 1 || wa < 1 || hb < 1 || wb < 1 || wa > kMaxBandWidth) return false;
    if ((int64_t)hb * wb * ha >= ((int64_t)1 << 31) - 1024) return false;   // TMA row coordinates are int32
    return band_plan(ha, wa).ok && y_rows_per_cta(hb) >= 1;
}

size_t refocus_ws_bytes(int ha, int wa, int hb, int wb, int n_planes) {
    if (!refocus_supported(ha, wa, hb, wb) || n_planes < 1) return 0;
    const size_t Ma = (size_t)ha * wa, Mb = (size_t)hb * wb;
    const BandPlan b = band_plan(ha, wa);
    const int per_launch = n_planes < kRefocusMaxPlanesPerLaunch ? n_planes : kRefocusMaxPlanesPerLaunch;
    size_t bytes = round256((size_t)per_launch * hb * Ma * sizeof(float));
    if (b.pitch) bytes += round256(Mb * ha * (size_t)b.pitch * sizeof(float));
    return bytes + xtables_bytes();
}

int refocus_launches(int ha, int wa, int n_planes) {
    const int chunks = (n_planes + kRefocusMaxPlanesPerLaunch - 1) / kRefocusMaxPlanesPerLaunch;
    return 3 * chunks + (band_plan(ha, wa).pitch ? 1 : 0);
}

cudaError_t refocus_run(const float* gamma_f32, int ha, int wa, int hb, int wb, const double* alpha,
                        const double* beta, int n_planes, float* out, void* workspace, int sm_count,
                        unsigned int* status, unsigned long long timeout_ns, cudaStream_t st) {
    const int64_t Ma = (int64_t)ha * wa, Mb = (int64_t)hb * wb;
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    PlaneBlock pb;
    const BandPlan b = band_plan(ha, wa);
    {
        if (!b.ok) return cudaErrorInvalidValue;
        const int per_launch = n_planes < kRefocusMaxPlanesPerLaunch ? n_planes : kRefocusMaxPlanesPerLaunch;
        float* ubuf = reinterpret_cast<float*>(ws);
        const float* src = gamma_f32;
        int pitch = wa;
        if (b.pitch) {
            float* copy = reinterpret_cast<float*>(ws + round256((size_t)per_launch * hb * Ma * sizeof(float)));
            const int64_t rows = Mb * ha;
            int64_t blocks = (rows * b.pitch + 255) / 256;
            if (blocks > 8 * (int64_t)sm_count) blocks = 8 * (int64_t)sm_count;
            refocus_repack_kernel<<<(unsigned)blocks, 256, 0, st>>>(gamma_f32, copy, rows, wa, b.pitch);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            src = copy;
            pitch = b.pitch;
        }
        CUtensorMap tm;
        if (!b.mode3d) {
            const uint64_t dims[2] = {(uint64_t)wa, (uint64_t)(Mb * ha)};
            const uint64_t strides[1] = {(uint64_t)pitch * sizeof(float)};
            const uint32_t box[2] = {(uint32_t)b.WS, (uint32_t)b.BH};
            if (!make_f32_map(&tm, src, 2, dims, strides, box)) return cudaErrorInvalidValue;
        } else {
            const uint64_t dims[3] = {16, (uint64_t)(pitch / 16), (uint64_t)(Mb * ha)};
            const uint64_t strides[2] = {16 * sizeof(float), (uint64_t)pitch * sizeof(float)};
            const uint32_t box[3] = {16, (uint32_t)(b.WS / 16), (uint32_t)b.BH};
            if (!make_f32_map(&tm, src, 3, dims, strides, box)) return cudaErrorInvalidValue;
        }
        const int RB = y_rows_per_cta(hb);
        size_t tab_off = round256((size_t)per_launch * hb * Ma * sizeof(float));
        if (b.pitch) tab_off += round256(Mb * ha * (size_t)b.pitch * sizeof(float));
        long long* xcol = reinterpret_cast<long long*>(ws + tab_off);
        long long* xang = reinterpret_cast<long long*>(
            ws + tab_off + round256((size_t)kRefocusMaxPlanesPerLaunch * kBandThreads * sizeof(long long)));
        for (int p0 = 0; p0 < n_planes; p0 += kRefocusMaxPlanesPerLaunch) {
            const int np = n_planes - p0 < kRefocusMaxPlanesPerLaunch ? n_planes - p0 : kRefocusMaxPlanesPerLaunch;
            std::memset(&pb, 0, sizeof(pb));
            for (int i = 0; i < np; ++i) {
                pb.alpha[i] = alpha[p0 + i];
                pb.beta[i] = beta[p0 + i];
            }
            BandGeom g{};
            g.ha = ha;
            g.wa = wa;
            g.hb = hb;
            g.wb = wb;
            g.n_planes = np;
            g.cwt = b.cwt;
            g.R = b.R;
            g.BH = b.BH;
            g.n_bands = b.n_bands;
            g.n_pb = (np + b.PB - 1) / b.PB;
            g.pad_l = b.pad_l;
            g.mode3d = b.mode3d;
            g.stages = b.stages;
            g.stage_bytes = (uint32_t)((size_t)b.BH * b.WS * sizeof(float));
            g.xcol = xcol;
            g.xang = xang;
            g.status = status;
            g.timeout_ns = timeout_ns;
            refocus_xtables_kernel<<<(unsigned)((np * kBandThreads + 255) / 256), 256, 0, st>>>(pb, np, wa, wb, b.pad_l,
                                                                                               xcol, xang);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            const int64_t units = (int64_t)hb * g.n_pb * g.n_bands;
            const int grid = units < sm_count ? (int)units : sm_count;
            e = launch_band(b, &tm, g, pb, ubuf, grid, st);
            if (e != cudaSuccess) return e;
            YGeom y{ha, wa, hb, RB, p0};
            const size_t ysmem = (size_t)RB * hb * sizeof(YTap);
            e = set_smem_attr(refocus_ystage_kernel, 20, kSmemCap);
            if (e != cudaSuccess) return e;
            refocus_ystage_kernel<<<dim3((unsigned)((ha + RB - 1) / RB), (unsigned)np), kYThreads, ysmem, st>>>(
                ubuf, y, pb, out);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

}  // namespace cpi
