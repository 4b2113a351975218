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
// sums are Kahan-compensated FP32; partial images of each range of angular rows
// are written in double and added in a fixed order by a second kernel, so the
// result is deterministic.
//
// Layout: Gamma arrives slice-major, float [Mb][Ma]; slice b is one contiguous
// spatial image, staged into shared memory with cp.async (double-buffered),
// with zero columns on both sides so that out-of-grid taps read 0.
//
// This file is compiled without FMA contraction: the double-float and Kahan
// steps depend on the written rounding order; the products use explicit fmaf.
#include "kernels.cuh"

namespace cpi {
namespace {

constexpr int kThreads = 512;
constexpr int kPadL = 4;      // zero columns left of the interior (keeps 16-byte alignment)
constexpr int kPadR = 4;

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

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

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
// CTA = (range of angular rows, plane).  Thread t owns column c = t % wa and rows
// rp + R*k (R = 512 / wa row phases), for both U and the output.
template <int KR>
__global__ void __launch_bounds__(kThreads, (KR >= 16 ? 1 : 2)) refocus_sep_kernel(const float* __restrict__ gamma,
                                                               const RefocusGeom geo,
                                                               const PlaneBlock pl,
                                                               double* __restrict__ partial) {
    extern __shared__ __align__(16) float sm[];
    const int ha = geo.ha, wa = geo.wa, hb = geo.hb, wb = geo.wb;
    const int WS = wa + kPadL + kPadR;                 // staged slice row stride
    const int slice_f = ha * WS;
    float* const buf0 = sm;                            // slice buffers: buf0 + (s & 1) * slice_f
    float* U = sm + 2 * slice_f;                       // (ha + 2) x wa, zero rows -1 and ha
    Tap* xt = reinterpret_cast<Tap*>(U + (ha + 2) * wa);   // [2][wa]
    Tap* yt = xt + 2 * wa;                             // [ha]

    const int tid = threadIdx.x;
    const int R = kThreads / wa;
    const int c = tid % wa, rp = tid / wa;
    const bool active = rp < R;
    const int p = blockIdx.y;
    const PlaneCoef pc = plane_coef(pl, p, ha, wa, hb, wb);
    const float cxa = 0.5f * (float)(wa - 1), cya = 0.5f * (float)(ha - 1);
    const float cxb = 0.5f * (float)(wb - 1), cyb = 0.5f * (float)(hb - 1);
    const int64_t Ma = (int64_t)ha * wa;
    const bool vec = (wa % 4) == 0 && (reinterpret_cast<uintptr_t>(gamma) % 16) == 0;

    // zero the pad columns of both slice buffers and the pad rows of U
    for (int i = tid; i < 2 * ha; i += kThreads) {
        float* row = buf0 + (i / ha) * slice_f + (i % ha) * WS;
#pragma unroll
        for (int q = 0; q < kPadL; ++q) row[q] = 0.0f;
#pragma unroll
        for (int q = 0; q < kPadR; ++q) row[kPadL + wa + q] = 0.0f;
    }
    for (int i = tid; i < wa; i += kThreads) {
        U[i] = 0.0f;
        U[(ha + 1) * wa + i] = 0.0f;
    }

    const int br0 = blockIdx.x * geo.b_per_range;            // b_per_range counts angular ROWS here
    const int br1 = min(br0 + geo.b_per_range, hb);
    const int n_slices = (br1 - br0) * wb;

    // stage slice s of this range into buffer s & 1, with its x taps
    auto stage = [&](int s) {
        const int br = br0 + s / wb, bc = s % wb;
        const float* src = gamma + ((int64_t)br * wb + bc) * Ma;
        float* dst = buf0 + (s & 1) * slice_f;
        if (vec) {
            const int per_row = wa / 4;
            for (int i = tid; i < ha * per_row; i += kThreads) {
                const int r = i / per_row, q = i - r * per_row;
                cp_async16(dst + r * WS + kPadL + 4 * q, src + (int64_t)r * wa + 4 * q);
            }
        } else {
            for (int i = tid; i < ha * wa; i += kThreads) {
                const int r = i / wa, q = i - r * wa;
                cp_async4(dst + r * WS + kPadL + q, src + (int64_t)r * wa + q);
            }
        }
        for (int j = tid; j < wa; j += kThreads)
            xt[(s & 1) * wa + j] = axis_tap(pc.alpha, (float)j - cxa, pc.qx, (float)bc - cxb, cxa, wa, kPadL);
    };

    // U accumulates plainly over groups of <= 4 slices (Ug), and the group sums
    // are Kahan-added (Ua, Uc): error <= (3 + 2) * 2^-24 of the summed magnitudes.
    float Ug[KR], Ua[KR], Uc[KR], Ra[KR], Rc[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k) Ug[k] = Ua[k] = Uc[k] = Ra[k] = Rc[k] = 0.0f;

    if (n_slices > 0) stage(0);
    cp_async_commit();
    for (int s = 0; s < n_slices; ++s) {
        if (s + 1 < n_slices) stage(s + 1);
        cp_async_commit();
        cp_async_wait_1();
        __syncthreads();   // slice s and its taps visible to all threads
        const int bc = s % wb;
        if (active) {
            const Tap tx = xt[(s & 1) * wa + c];
            const float* S = buf0 + (s & 1) * slice_f + tx.off;
            const bool group_end = (bc & 3) == 3 || bc == wb - 1;
#pragma unroll
            for (int k = 0; k < KR; ++k) {
                const int y = rp + R * k;
                if (y < ha) {
                    const float v0 = S[y * WS], v1 = S[y * WS + 1];
                    Ug[k] += __fmaf_rn(tx.w1, v1, tx.w0 * v0);
                }
                if (group_end) {
                    kahan_add(Ua[k], Uc[k], Ug[k]);
                    Ug[k] = 0.0f;
                }
            }
        }
        if (bc == wb - 1) {
            // angular row complete: y-interpolate U into the output
            const int br = br0 + s / wb;
            if (active) {
#pragma unroll
                for (int k = 0; k < KR; ++k) {
                    const int y = rp + R * k;
                    if (y < ha) U[(y + 1) * wa + c] = Ua[k] - Uc[k];
                    Ua[k] = Uc[k] = 0.0f;
                }
            }
            for (int j = tid; j < ha; j += kThreads) {
                Tap t = axis_tap(pc.alpha, (float)j - cya, pc.qy, (float)br - cyb, cya, ha, 1);
                t.off *= wa;
                yt[j] = t;
            }
            __syncthreads();
            if (active) {
#pragma unroll
                for (int k = 0; k < KR; ++k) {
                    const int r = rp + R * k;
                    if (r < ha) {
                        const Tap ty = yt[r];
                        const float v0 = U[ty.off + c], v1 = U[ty.off + wa + c];
                        kahan_add(Ra[k], Rc[k], __fmaf_rn(ty.w1, v1, ty.w0 * v0));
                    }
                }
            }
        }
        __syncthreads();   // buffer s & 1, U and yt free for reuse
    }
    cp_async_wait_0();
    if (!active) return;
    double* dst = partial + ((int64_t)blockIdx.x * geo.total_planes + geo.plane_offset + p) * Ma;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
        const int r = rp + R * k;
        if (r < ha) dst[(int64_t)r * wa + c] = (double)Ra[k] - (double)Rc[k];
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
                                                                  double* __restrict__ partial) {
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
    double* dst = partial + ((int64_t)blockIdx.x * geo.total_planes + geo.plane_offset + p) * Ma;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
        const int r = row0 + rp + R * k;
        if (r < ha) dst[(int64_t)r * wa + c] = (double)acc[k] - (double)cmp[k];
    }
}

__global__ void refocus_reduce_kernel(const double* __restrict__ partial, int n_ranges,
                                      int64_t per_range, float* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < per_range;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < n_ranges; ++r) s += partial[(int64_t)r * per_range + i];
        out[i] = (float)s;
    }
}

template <typename K>
cudaError_t set_smem_attr(K kernel, int slot) {
    static bool done[16][64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!done[slot][dev]) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        done[slot][dev] = true;
    }
    return cudaSuccess;
}

template <int KR>
cudaError_t launch_sep(const float* g, const RefocusGeom& geo, const PlaneBlock& pl, double* partial,
                       size_t smem, cudaStream_t st, int slot) {
    cudaError_t e = set_smem_attr(refocus_sep_kernel<KR>, slot);
    if (e != cudaSuccess) return e;
    refocus_sep_kernel<KR><<<dim3(geo.n_ranges, geo.n_planes), kThreads, smem, st>>>(g, geo, pl, partial);
    return cudaGetLastError();
}

template <int KR>
cudaError_t launch_direct(const float* g, const RefocusGeom& geo, const PlaneBlock& pl,
                          double* partial, int zchunks, size_t smem, cudaStream_t st, int slot) {
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

bool refocus_separable(int ha, int wa) {
    if (wa > kThreads) return false;
    const int R = kThreads / wa;
    if ((ha + R - 1) / R > 16) return false;
    return refocus_smem_bytes(ha, wa) <= 200 * 1024;
}

size_t refocus_smem_bytes(int ha, int wa) {
    const size_t sep = sizeof(float) * (2 * (size_t)ha * (wa + kPadL + kPadR) + (size_t)(ha + 2) * wa) +
                       sizeof(Tap) * (2 * (size_t)wa + (size_t)ha);
    const int R = wa <= kThreads ? kThreads / wa : 1;
    if (wa <= kThreads && (ha + R - 1) / R <= 16 && sep <= 200 * 1024) return sep;
    return sizeof(float) * (size_t)(ha + 2) * (wa + 2) + sizeof(Tap) * ((size_t)wa + ha);
}

int refocus_ranges(int ha, int wa, int hb, int wb, int n_planes, int sm_count) {
    // ranges of angular rows (separable kernel) or of angular pixels (direct kernel)
    const int units = refocus_separable(ha, wa) ? hb : hb * wb;
    int target = (4 * sm_count + n_planes - 1) / (n_planes > 0 ? n_planes : 1);
    if (target < 1) target = 1;
    if (target > units) target = units;
    const int per = (units + target - 1) / target;
    return (units + per - 1) / per;
}

int refocus_range_size(int ha, int wa, int hb, int wb, int n_ranges) {
    const int units = refocus_separable(ha, wa) ? hb : hb * wb;
    return (units + n_ranges - 1) / n_ranges;
}

cudaError_t launch_refocus(const float* gamma_f32, const RefocusGeom& geo, const PlaneBlock& pl,
                           double* partial, cudaStream_t st) {
    const size_t smem = refocus_smem_bytes(geo.ha, geo.wa);
    if (refocus_separable(geo.ha, geo.wa)) {
        switch (kr_for(geo.ha, geo.wa, 16)) {
            case 1: return launch_sep<1>(gamma_f32, geo, pl, partial, smem, st, 0);
            case 2: return launch_sep<2>(gamma_f32, geo, pl, partial, smem, st, 1);
            case 4: return launch_sep<4>(gamma_f32, geo, pl, partial, smem, st, 2);
            case 8: return launch_sep<8>(gamma_f32, geo, pl, partial, smem, st, 3);
            default: return launch_sep<16>(gamma_f32, geo, pl, partial, smem, st, 4);
        }
    }
    const int R = kThreads / geo.wa;
    const int kr = kr_for(geo.ha, geo.wa, 16);
    const int zchunks = (geo.ha + R * kr - 1) / (R * kr);
    switch (kr) {
        case 1: return launch_direct<1>(gamma_f32, geo, pl, partial, zchunks, smem, st, 5);
        case 2: return launch_direct<2>(gamma_f32, geo, pl, partial, zchunks, smem, st, 6);
        case 4: return launch_direct<4>(gamma_f32, geo, pl, partial, zchunks, smem, st, 7);
        case 8: return launch_direct<8>(gamma_f32, geo, pl, partial, zchunks, smem, st, 8);
        default: return launch_direct<16>(gamma_f32, geo, pl, partial, zchunks, smem, st, 9);
    }
}

cudaError_t launch_refocus_reduce(const double* partial, int n_ranges, int64_t per_range,
                                  float* out, cudaStream_t st) {
    int64_t blocks = (per_range + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    refocus_reduce_kernel<<<(unsigned)blocks, 256, 0, st>>>(partial, n_ranges, per_range, out);
    return cudaGetLastError();
}

}  // namespace cpi
