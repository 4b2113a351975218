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
// Interpolation coordinates are computed on the fly inside the kernel (the
// point of Section 4.1), per slice for the W_a columns and per angular row for
// the H_a rows, in double-float arithmetic on the FP32 pipe (~48-bit
// significands; GB300's FP64 pipe is a small fraction of its FP32 rate).  All
// sums are Kahan-compensated FP32; the partial image of each angular row is
// written in FP32 and the rows are added in a fixed order (Kahan-compensated)
// by a second kernel, so the result is deterministic.
//
// Layout: Gamma arrives slice-major, float [Mb][Ma]; slice b is one contiguous
// spatial image, staged into shared memory with cp.async (double-buffered),
// with zero columns on both sides so that out-of-grid taps read 0.
//
// This file is compiled without FMA contraction: the double-float and Kahan
// steps depend on the written rounding order; the products use explicit fmaf.
#include <cstring>

#include "kernels.cuh"
#include "ptx.cuh"

namespace cpi {
namespace {

constexpr int kThreads = 512;
constexpr int kPadL = 4;      // zero columns left of the interior (keeps 16-byte alignment)
constexpr int kPadR = 4;
constexpr int kSepPlanes = 2;  // planes per CTA of the separable kernel
constexpr int kSepStages = 3;  // staged slices (TMA pipeline depth)

// ------------------------------------------------------------ double-float helpers
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ DF df_split(double v) {
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}
// (a.hi + a.lo) * x for a small exactly representable x
__device__ __forceinline__ DF df_mul(DF a, float x) {
    const float p = a.hi * x;
    float e = __fmaf_rn(a.hi, x, -p);
    e = __fmaf_rn(a.lo, x, e);
    return two_sum(p, e);
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const DF s = two_sum(a.hi, b.hi);
    return two_sum(s.hi, s.lo + (a.lo + b.lo));
}

// Bilinear tap of one axis: u = (scale * j_centred + shift * b_centred) + centre.
// Returns the padded offset of the first tap and both weights (zero weights when
// neither tap lies inside [0, n)).
struct Tap {
    int off;
    float w0, w1;
};
__device__ __forceinline__ Tap axis_tap(DF scale, float jc, DF shift, float bcen, float centre,
                                        int n, int pad) {
    const DF u = df_add(df_add(df_mul(scale, jc), df_mul(shift, bcen)), DF{centre, 0.0f});
    float f0 = floorf(u.hi);
    float fr = (u.hi - f0) + u.lo;
    if (fr < 0.0f) {
        f0 -= 1.0f;
        fr += 1.0f;
    } else if (fr >= 1.0f) {
        f0 += 1.0f;
        fr -= 1.0f;
    }
    Tap t{pad - 1, 0.0f, 0.0f};
    if (f0 >= -1.0f && f0 <= (float)(n - 1)) {
        t.off = (int)f0 + pad;
        t.w0 = 1.0f - fr;
        t.w1 = fr;
    }
    return t;
}

__device__ __forceinline__ void kahan_add(float& acc, float& cmp, float v) {
    const float y = v - cmp;
    const float t = acc + y;
    cmp = (t - acc) - y;
    acc = t;
}

struct PlaneCoef {
    DF alpha, qx, qy;     // alpha, beta*sx, beta*sy
};
__device__ __forceinline__ PlaneCoef plane_coef(const PlaneBlock& pl, int p, int ha, int wa, int hb,
                                                int wb) {
    const double al = pl.alpha[p], be = pl.beta[p];
    const double sx = (double)wa / (double)wb, sy = (double)ha / (double)hb;
    return {df_split(al), df_split(be * sx), df_split(be * sy)};
}

// ------------------------------------------------------------ separable kernel
// CTA = (angular row br, block of PB planes).  Thread t owns column c = t % wa
// and rows rp + R*k (R = 512 / wa row phases).  Each slice (br, bc) is staged
// into shared memory with 4 zero columns on both sides: by one 2-D TMA copy of
// a (wa + 8) x ha box starting at column -4 (the columns outside the image come
// back as zeros, exactly the out-of-grid taps), or, for widths TMA cannot
// describe, by 4-byte cp.async copies of each thread's own pixels.  Every
// staged slice is interpolated along x for all PB planes; after the last bc the
// row's U images are interpolated along y and this angular row's contribution
// to each output pixel is written to partial[br][plane][pixel].  The reduce
// kernel adds the angular rows in a fixed order (compensated FP32).
//
// Variants: PB = 2 planes, <= 8 rows per thread, 2 CTAs per SM (small images);
// PB = 1 plane, <= 32 rows per thread, 1 CTA per SM (images up to ~128 x 128).
// kWA > 0 fixes the image width (and kHA the height) at compile time, so every
// row offset of the inner loop is an immediate.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int KR, int PB, int kWA, int kHA, bool kTma, int kStages, int kMinBlocks>
__global__ void __launch_bounds__(kThreads, kMinBlocks) refocus_sep_kernel(const __grid_constant__ CUtensorMap tm,
                                                                           const float* __restrict__ gamma,
                                                                           const RefocusGeom geo,
                                                                           const PlaneBlock pl,
                                                                           float* __restrict__ partial) {
    extern __shared__ __align__(128) float sm_raw[];
    const int ha = kWA ? kHA : geo.ha, wa = kWA ? kWA : geo.wa, hb = geo.hb, wb = geo.wb;
    const int WS = wa + kPadL + kPadR;                 // staged slice row stride (TMA box width)
    const int slice_f = (ha * WS + 31) & ~31;          // buffer stride: 128-byte multiples
    // 128-byte aligned start, computed on the shared-window offset so that the
    // pointers stay shared-space (the loads below compile to shared loads)
    float* const buf0 = sm_raw + (((128u - (static_cast<uint32_t>(__cvta_generic_to_shared(sm_raw)) & 127u)) & 127u) >> 2);
    float* const U = buf0 + kStages * slice_f;         // PB x (ha + 2) x wa, zero rows -1 and ha
    Tap* const xt = reinterpret_cast<Tap*>(U + PB * (ha + 2) * wa);   // [kStages][PB][wa]
    Tap* const yt = xt + kStages * PB * wa;                           // [PB][ha]
    __shared__ PlaneCoef coef[PB];                     // per-plane coefficients, computed once
    __shared__ __align__(8) uint64_t full[kStages];    // TMA completion of each slice buffer
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    const int R = kThreads / wa;
    const int c = tid % wa, rp = tid / wa;
    const bool active = rp < R;
    const int nk = active ? (ha - rp + R - 1) / R : 0;      // rows of this thread
    const int br = blockIdx.x;
    const int pbase = blockIdx.y * PB;                  // first plane of this CTA (in this launch)
    const int np = min(PB, geo.n_planes - pbase);
    const float cxa = 0.5f * (float)(wa - 1), cya = 0.5f * (float)(ha - 1);
    const float cxb = 0.5f * (float)(wb - 1), cyb = 0.5f * (float)(hb - 1);
    const int64_t Ma = (int64_t)ha * wa;
    const uint32_t slice_bytes = (uint32_t)(ha * WS * sizeof(float));

    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) mbar_init(&full[i], 1);
        abort_flag = 0;
        fence_barrier_init();
    }
    if (tid < np) coef[tid] = plane_coef(pl, pbase + tid, ha, wa, hb, wb);
    for (int i = tid; i < PB * wa; i += kThreads) {
        const int j = i / wa, x = i - j * wa;
        U[j * (ha + 2) * wa + x] = 0.0f;
        U[j * (ha + 2) * wa + (ha + 1) * wa + x] = 0.0f;
    }
    if constexpr (!kTma) {   // zero columns of every buffer row (cp.async writes the interior only)
        for (int i = tid; i < kStages * ha; i += kThreads) {
            float* row = buf0 + (i / ha) * slice_f + (i % ha) * WS;
#pragma unroll
            for (int q = 0; q < kPadL; ++q) row[q] = 0.0f;
#pragma unroll
            for (int q = 0; q < kPadR; ++q) row[kPadL + wa + q] = 0.0f;
        }
    }
    __syncthreads();   // barriers initialised, coef and pads visible
    auto issue = [&](int bc) {   // slice (br, bc) -> buffer bc % kStages
        const int sb = bc % kStages;
        if constexpr (kTma) {
            if (tid == 0) {
                mbar_arrive_expect_tx(&full[sb], slice_bytes);
                tma_load_2d(buf0 + sb * slice_f, &tm, &full[sb], -kPadL, (br * wb + bc) * ha);
            }
        } else {
            if (active) {
                const float* src = gamma + ((int64_t)br * wb + bc) * Ma + (int64_t)rp * wa + c;
                float* dst = buf0 + sb * slice_f + rp * WS + kPadL + c;
                for (int k = 0; k < nk; ++k) cp_async4(dst + k * R * WS, src + (int64_t)k * R * wa);
            }
            cp_async_commit();   // one group per slice, also when this thread copied nothing
        }
    };
    auto taps = [&](int bc) {    // x taps of slice bc for every plane
        const int sb = bc % kStages;
        for (int i = tid; i < np * wa; i += kThreads) {
            const int j = i / wa, x = i - j * wa;
            xt[(sb * PB + j) * wa + x] =
                axis_tap(coef[j].alpha, (float)x - cxa, coef[j].qx, (float)bc - cxb, cxa, wa, kPadL);
        }
    };
    // prologue: the first kStages - 1 slices in flight, their taps ready
    int last_issue[kStages];
#pragma unroll
    for (int i = 0; i < kStages; ++i) last_issue[i] = -1;
    for (int bc = 0; bc < kStages - 1; ++bc) {
        if (bc < wb) {
            issue(bc);
            last_issue[bc % kStages] = bc;
            taps(bc);
        } else if constexpr (!kTma) {
            cp_async_commit();   // keep one group per slot
        }
    }

    // U accumulates plainly (two fused multiply-adds per slice) over pairs of
    // slices (Ug); the pair sums are Kahan-added (Ua, Uc): error <= (4 + 2) 2^-24
    // of the summed magnitudes, to first order.
    float Ug[PB][KR], Ua[PB][KR], Uc[PB][KR];
#pragma unroll
    for (int j = 0; j < PB; ++j)
#pragma unroll
        for (int k = 0; k < KR; ++k) Ug[j][k] = Ua[j][k] = Uc[j][k] = 0.0f;

    for (int bc = 0; bc < wb; ++bc) {
        const int sb = bc % kStages;
        const uint32_t parity = (uint32_t)((bc / kStages) & 1);
        if constexpr (kTma) {
            // one thread waits for the copy; the others sleep in the barrier below
            if (tid == 0 && !mbar_wait_sleepy(&full[sb], parity, geo.status, geo.timeout_ns)) abort_flag = 1;
        } else {
            cp_async_wait<kStages - 2>();   // this thread's copies of slice bc have landed
        }
        __syncthreads();   // slice bc landed; every thread is done with slice bc - 1
        if (abort_flag) break;
        // refill the buffer slice bc - 1 used, and prepare its taps
        const int nxt = bc + kStages - 1;
        if (nxt < wb) {
            issue(nxt);
            last_issue[nxt % kStages] = nxt;
            taps(nxt);
        } else if constexpr (!kTma) {
            cp_async_commit();
        }
        if constexpr (kTma)
            mbar_wait_bounded(&full[sb], parity, &abort_flag, geo.status, geo.timeout_ns);   // completes at once
        if (active) {
            const float* S = buf0 + sb * slice_f + rp * WS;
            const int step = R * WS;
#pragma unroll
            for (int j = 0; j < PB; ++j) {
                if (j < np) {
                    const Tap tx = xt[(sb * PB + j) * wa + c];
                    const float* q = S + tx.off;
                    if constexpr (kWA > 0 && kHA % (kThreads / kWA) == 0) {
                        constexpr int kStep = (kThreads / kWA) * (kWA + kPadL + kPadR);
#pragma unroll
                        for (int k = 0; k < KR; ++k)
                            Ug[j][k] = __fmaf_rn(tx.w1, q[k * kStep + 1], __fmaf_rn(tx.w0, q[k * kStep], Ug[j][k]));
                    } else if (nk == KR) {
#pragma unroll
                        for (int k = 0; k < KR; ++k) {
                            Ug[j][k] = __fmaf_rn(tx.w1, q[1], __fmaf_rn(tx.w0, q[0], Ug[j][k]));
                            q += step;
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < KR; ++k) {
                            if (k < nk) Ug[j][k] = __fmaf_rn(tx.w1, q[1], __fmaf_rn(tx.w0, q[0], Ug[j][k]));
                            q += step;
                        }
                    }
                }
            }
        }
        if ((bc & 1) == 1 || bc == wb - 1) {   // uniform: every thread takes it together
#pragma unroll
            for (int j = 0; j < PB; ++j)
#pragma unroll
                for (int k = 0; k < KR; ++k) {
                    kahan_add(Ua[j][k], Uc[j][k], Ug[j][k]);
                    Ug[j][k] = 0.0f;
                }
        }
    }
    if constexpr (!kTma) cp_async_wait<0>();
    if (abort_flag) {
        // drain any copy still in flight before the CTA exits
        if (kTma && tid == 0)
            for (int i = 0; i < kStages; ++i)
                if (last_issue[i] >= 0)
                    mbar_wait_bounded(&full[i], (uint32_t)((last_issue[i] / kStages) & 1), nullptr,
                                      nullptr, geo.timeout_ns);
        return;
    }
    __syncthreads();   // all slices consumed before U is written

    // y-interpolation of this angular row
    if (active) {
#pragma unroll
        for (int j = 0; j < PB; ++j)
#pragma unroll
            for (int k = 0; k < KR; ++k) {
                const int y = rp + R * k;
                if (k < nk) U[(j * (ha + 2) + y + 1) * wa + c] = Ua[j][k] - Uc[j][k];
            }
    }
    for (int i = tid; i < np * ha; i += kThreads) {
        const int j = i / ha, y = i - j * ha;
        Tap t = axis_tap(coef[j].alpha, (float)y - cya, coef[j].qy, (float)br - cyb, cya, ha, 1);
        t.off = (j * (ha + 2) + t.off) * wa;
        yt[j * ha + y] = t;
    }
    __syncthreads();
    if (!active) return;
#pragma unroll
    for (int j = 0; j < PB; ++j) {
        if (j < np) {
            float* dst = partial + ((int64_t)br * geo.total_planes + geo.plane_offset + pbase + j) * Ma;
#pragma unroll
            for (int k = 0; k < KR; ++k) {
                const int r = rp + R * k;
                if (k < nk) {
                    const Tap ty = yt[j * ha + r];
                    const float v0 = U[ty.off + c], v1 = U[ty.off + wa + c];
                    dst[(int64_t)r * wa + c] = __fmaf_rn(ty.w1, v1, ty.w0 * v0);
                }
            }
        }
    }
}

// ------------------------------------------------------------ direct kernel
// Fallback for spatial images too large for the separable kernel's registers:
// CTA = (range of angular pixels, plane, band of output rows); each angular
// pixel's slice is staged with a zero border and its 4 taps read per output.
template <int KR>
__global__ void __launch_bounds__(kThreads) refocus_direct_kernel(const float* __restrict__ gamma,
                                                                  const RefocusGeom geo,
                                                                  const PlaneBlock pl,
                                                                  float* __restrict__ partial) {
    extern __shared__ __align__(16) float sm[];
    const int ha = geo.ha, wa = geo.wa, hb = geo.hb, wb = geo.wb;
    const int W2 = wa + 2;
    const int64_t Ma = (int64_t)ha * wa;
    float* slice = sm;                                                // (ha + 2) x (wa + 2)
    Tap* xt = reinterpret_cast<Tap*>(slice + (ha + 2) * W2);          // [wa]
    Tap* yt = xt + wa;                                                // [ha]
    const int tid = threadIdx.x;
    const int R = kThreads / wa;
    const int c = tid % wa, rp = tid / wa;
    const bool active = rp < R;
    const int row0 = blockIdx.z * (R * KR);
    const int p = blockIdx.y;
    const PlaneCoef pc = plane_coef(pl, p, ha, wa, hb, wb);
    const float cxa = 0.5f * (float)(wa - 1), cya = 0.5f * (float)(ha - 1);
    const float cxb = 0.5f * (float)(wb - 1), cyb = 0.5f * (float)(hb - 1);

    for (int i = tid; i < (ha + 2) * W2; i += kThreads) slice[i] = 0.0f;
    float acc[KR], cmp[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k) acc[k] = cmp[k] = 0.0f;
    const int nb = hb * wb;
    const int b_begin = blockIdx.x * geo.b_per_range;
    const int b_end = min(b_begin + geo.b_per_range, nb);
    const int rows_per_pass = kThreads / wa;
    for (int b = b_begin; b < b_end; ++b) {
        __syncthreads();
        const float* src = gamma + (int64_t)b * Ma;
        if (active)
            for (int r = rp; r < ha; r += rows_per_pass)
                slice[(r + 1) * W2 + c + 1] = __ldg(src + (int64_t)r * wa + c);
        const int br = b / wb, bc = b - br * wb;
        for (int j = tid; j < wa + ha; j += kThreads) {
            if (j < wa) {
                xt[j] = axis_tap(pc.alpha, (float)j - cxa, pc.qx, (float)bc - cxb, cxa, wa, 1);
            } else {
                Tap t = axis_tap(pc.alpha, (float)(j - wa) - cya, pc.qy, (float)br - cyb, cya, ha, 1);
                t.off *= W2;
                yt[j - wa] = t;
            }
        }
        __syncthreads();
        if (active) {
            const Tap tx = xt[c];
#pragma unroll
            for (int k = 0; k < KR; ++k) {
                const int r = row0 + rp + R * k;
                if (r < ha) {
                    const Tap ty = yt[r];
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
        for (int r = 0; r < n_ranges; ++r) kahan_add(acc, cmp, __ldg(partial + (int64_t)r * per_range + i));
        out[i] = acc - cmp;
    }
}

template <typename K>
cudaError_t set_smem_attr(K kernel, int slot) {
    static bool done[32][64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!done[slot][dev]) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e != cudaSuccess) return e;
        done[slot][dev] = true;
    }
    return cudaSuccess;
}

template <int KR, int PB, bool kTma, int kStages, int kMinBlocks, int kWA = 0, int kHA = 0>
cudaError_t launch_sep(const CUtensorMap* tm, const float* g, const RefocusGeom& geo, const PlaneBlock& pl,
                       float* partial, size_t smem, cudaStream_t st, int slot) {
    auto kern = refocus_sep_kernel<KR, PB, kWA, kHA, kTma, kStages, kMinBlocks>;
    cudaError_t e = set_smem_attr(kern, slot);
    if (e != cudaSuccess) return e;
    CUtensorMap dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    const int pblocks = (geo.n_planes + PB - 1) / PB;
    kern<<<dim3(geo.hb, pblocks), kThreads, smem, st>>>(tm ? *tm : dummy, g, geo, pl, partial);
    return cudaGetLastError();
}

template <int KR>
cudaError_t launch_direct(const float* g, const RefocusGeom& geo, const PlaneBlock& pl,
                          float* partial, int zchunks, size_t smem, cudaStream_t st, int slot) {
    cudaError_t e = set_smem_attr(refocus_direct_kernel<KR>, slot);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)geo.n_ranges, (unsigned)geo.n_planes, (unsigned)zchunks);
    refocus_direct_kernel<KR><<<grid, kThreads, smem, st>>>(g, geo, pl, partial);
    return cudaGetLastError();
}

int kr_for(int ha, int wa, int cap) {
    const int R = kThreads / wa;
    int kr = 1;
    while (kr < cap && R * kr < ha) kr *= 2;
    return kr;
}

}  // namespace

// Separable-kernel variant of an image shape.
struct SepVariant {
    bool ok;
    bool tma;       // TMA staging (width a multiple of 4, box sides <= 256)
    bool large;     // 1 plane per CTA, up to 32 rows per thread, 1 CTA per SM
    int kr;         // rows per thread (power of two)
    int stages;
};

static size_t sep_smem_for(int ha, int wa, int pb, int stages) {
    const size_t slice_f = ((size_t)ha * (wa + kPadL + kPadR) + 31) & ~(size_t)31;
    return 128 + sizeof(float) * (stages * slice_f + (size_t)pb * (ha + 2) * wa) +
           sizeof(Tap) * (stages * (size_t)pb * wa + (size_t)pb * ha);
}

static SepVariant sep_variant(int ha, int wa) {
    SepVariant v{false, false, false, 1, 3};
    if (wa > kThreads) return v;
    v.tma = (wa % 4 == 0) && (wa + kPadL + kPadR <= 256) && ha <= 256;
    const int R = kThreads / wa;
    const int rows = (ha + R - 1) / R;
    if (rows <= 8 && sep_smem_for(ha, wa, kSepPlanes, 3) <= 112 * 1024) {
        v.ok = true;
        v.kr = kr_for(ha, wa, 8);
        v.stages = 3;
        return v;
    }
    if (rows <= 32) {
        v.large = true;
        v.kr = rows <= 16 ? 16 : 32;
        v.stages = sep_smem_for(ha, wa, 1, 3) <= 220 * 1024 ? 3 : 2;
        v.ok = sep_smem_for(ha, wa, 1, v.stages) <= 220 * 1024;
    }
    return v;
}

bool refocus_separable(int ha, int wa) { return sep_variant(ha, wa).ok; }

size_t refocus_smem_bytes(int ha, int wa) {
    const SepVariant v = sep_variant(ha, wa);
    if (v.ok) return sep_smem_for(ha, wa, v.large ? 1 : kSepPlanes, v.stages);
    return sizeof(float) * (size_t)(ha + 2) * (wa + 2) + sizeof(Tap) * ((size_t)wa + ha);
}

bool refocus_uses_tma(int ha, int wa) {
    const SepVariant v = sep_variant(ha, wa);
    return v.ok && v.tma;
}

int refocus_ranges(int ha, int wa, int hb, int wb, int n_planes, int sm_count) {
    // separable kernel: one range per angular row; direct kernel: ranges of
    // angular pixels sized to fill the GPU
    if (refocus_separable(ha, wa)) return hb;
    const int units = hb * wb;
    int target = (4 * sm_count + n_planes - 1) / (n_planes > 0 ? n_planes : 1);
    if (target < 1) target = 1;
    if (target > units) target = units;
    const int per = (units + target - 1) / target;
    return (units + per - 1) / per;
}

int refocus_range_size(int ha, int wa, int hb, int wb, int n_ranges) {
    if (refocus_separable(ha, wa)) return 1;
    return (hb * wb + n_ranges - 1) / n_ranges;
}

cudaError_t launch_refocus(const float* gamma_f32, const CUtensorMap* tm, const RefocusGeom& geo,
                           const PlaneBlock& pl, float* partial, cudaStream_t st) {
    const size_t smem = refocus_smem_bytes(geo.ha, geo.wa);
    const SepVariant v = sep_variant(geo.ha, geo.wa);
    if (v.ok) {
        if (v.tma && tm == nullptr) return cudaErrorInvalidValue;
        const float* g = gamma_f32;
        if (!v.large) {
            if (v.tma) {
                // compile-time shapes of the common square detector sizes
                if (geo.wa == 64 && geo.ha == 64)
                    return launch_sep<8, 2, true, 3, 2, 64, 64>(tm, g, geo, pl, partial, smem, st, 10);
                if (geo.wa == 32 && geo.ha == 32)
                    return launch_sep<2, 2, true, 3, 2, 32, 32>(tm, g, geo, pl, partial, smem, st, 11);
                switch (v.kr) {
                    case 1: return launch_sep<1, 2, true, 3, 2>(tm, g, geo, pl, partial, smem, st, 0);
                    case 2: return launch_sep<2, 2, true, 3, 2>(tm, g, geo, pl, partial, smem, st, 1);
                    case 4: return launch_sep<4, 2, true, 3, 2>(tm, g, geo, pl, partial, smem, st, 2);
                    default: return launch_sep<8, 2, true, 3, 2>(tm, g, geo, pl, partial, smem, st, 3);
                }
            }
            switch (v.kr) {
                case 1: return launch_sep<1, 2, false, 3, 2>(nullptr, g, geo, pl, partial, smem, st, 4);
                case 2: return launch_sep<2, 2, false, 3, 2>(nullptr, g, geo, pl, partial, smem, st, 5);
                case 4: return launch_sep<4, 2, false, 3, 2>(nullptr, g, geo, pl, partial, smem, st, 6);
                default: return launch_sep<8, 2, false, 3, 2>(nullptr, g, geo, pl, partial, smem, st, 7);
            }
        }
        const CUtensorMap* t = v.tma ? tm : nullptr;
        if (v.stages == 3) {
            if (v.kr == 16)
                return v.tma ? launch_sep<16, 1, true, 3, 1>(t, g, geo, pl, partial, smem, st, 12)
                             : launch_sep<16, 1, false, 3, 1>(t, g, geo, pl, partial, smem, st, 13);
            return v.tma ? launch_sep<32, 1, true, 3, 1>(t, g, geo, pl, partial, smem, st, 14)
                         : launch_sep<32, 1, false, 3, 1>(t, g, geo, pl, partial, smem, st, 15);
        }
        if (v.kr == 16)
            return v.tma ? launch_sep<16, 1, true, 2, 1>(t, g, geo, pl, partial, smem, st, 16)
                         : launch_sep<16, 1, false, 2, 1>(t, g, geo, pl, partial, smem, st, 17);
        return v.tma ? launch_sep<32, 1, true, 2, 1>(t, g, geo, pl, partial, smem, st, 18)
                     : launch_sep<32, 1, false, 2, 1>(t, g, geo, pl, partial, smem, st, 19);
    }
    const int R = kThreads / geo.wa;
    const int kr = kr_for(geo.ha, geo.wa, 16);
    const int zchunks = (geo.ha + R * kr - 1) / (R * kr);
    switch (kr) {
        case 1: return launch_direct<1>(gamma_f32, geo, pl, partial, zchunks, smem, st, 5 + 20);
        case 2: return launch_direct<2>(gamma_f32, geo, pl, partial, zchunks, smem, st, 6 + 20);
        case 4: return launch_direct<4>(gamma_f32, geo, pl, partial, zchunks, smem, st, 7 + 20);
        case 8: return launch_direct<8>(gamma_f32, geo, pl, partial, zchunks, smem, st, 8 + 20);
        default: return launch_direct<16>(gamma_f32, geo, pl, partial, zchunks, smem, st, 9 + 20);
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
