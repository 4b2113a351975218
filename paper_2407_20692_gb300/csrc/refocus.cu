// Step a5: refocusing (Section "CPI algorithm", item 2; Section 4.1, "Refocusing
// Optimization").  For plane (alpha, beta) and spatial output pixel x:
//     out(x) = sum over angular pixels b of  Gamma~_b(alpha * x + beta * rho_b~)
// where Gamma~_b is the bilinear interpolation of the spatial image Gamma[.][b]
// (zero outside the grid), x and rho_b are centred pixel coordinates and
// rho_b~ = rho_b * (wa/wb, ha/hb).
//
// Layout: Gamma comes slice-major, float [Mb][Ma], so each angular pixel's
// spatial image is one contiguous block.  CTA = (range of angular pixels, plane,
// band of output rows).  For every angular pixel of its range the CTA
//   1. stages the slice in shared memory inside a one-pixel zero border, so
//      out-of-grid taps read 0 without a branch;
//   2. computes, on the fly and in double precision, the tap offsets and weights
//      of its output columns (alpha*(c - cxa) + beta*sx*(bc - cxb) + cxa) and
//      rows: W_a + H_a coordinates per angular pixel instead of a table of
//      coordinates per plane (the paper's point in Section 4.1);
//   3. adds, for each output pixel it owns (registers), the 4-tap bilinear
//      sample with Kahan-compensated FP32 accumulation.
// The per-range partial images go to the workspace in double; a second kernel
// adds the ranges in a fixed order, so the result is deterministic.
// This file is compiled without FMA contraction, so the double-precision
// coordinates are evaluated exactly as written (same rounding as a plain C
// evaluation); the bilinear products use explicit fmaf.
#include "kernels.cuh"

namespace cpi {
namespace {

constexpr int kThreads = 512;

template <int kOpt>
__global__ void __launch_bounds__(kThreads) refocus_kernel(const float* __restrict__ gamma,
                                                           const RefocusGeom geo,
                                                           const PlaneBlock pl,
                                                           double* __restrict__ partial) {
    extern __shared__ float sm[];
    const int ha = geo.ha, wa = geo.wa, hb = geo.hb, wb = geo.wb;
    const int W2 = wa + 2;
    const int64_t Ma = (int64_t)ha * wa;
    float* slice = sm;                                     // (ha+2) x (wa+2)
    int* xoff = reinterpret_cast<int*>(slice + (ha + 2) * W2);
    float* xw0 = reinterpret_cast<float*>(xoff + wa);
    float* xw1 = xw0 + wa;
    int* yoff = reinterpret_cast<int*>(xw1 + wa);
    float* yw0 = reinterpret_cast<float*>(yoff + ha);
    float* yw1 = yw0 + ha;

    const int tid = threadIdx.x;
    const int R = kThreads / wa;                           // row phases per CTA
    const int c = tid % wa, rp = tid / wa;
    const bool active = rp < R;
    const int row0 = blockIdx.z * (R * kOpt);
    const int p = blockIdx.y;
    const double al = pl.alpha[p], be = pl.beta[p];
    const double cxa = (wa - 1) / 2.0, cya = (ha - 1) / 2.0;
    const double cxb = (wb - 1) / 2.0, cyb = (hb - 1) / 2.0;
    const double sx = (double)wa / (double)wb, sy = (double)ha / (double)hb;

    for (int i = tid; i < (ha + 2) * W2; i += kThreads) slice[i] = 0.0f;

    float acc[kOpt], cmp[kOpt];
#pragma unroll
    for (int k = 0; k < kOpt; ++k) acc[k] = cmp[k] = 0.0f;

    const int nb = hb * wb;
    const int b_begin = blockIdx.x * geo.b_per_range;
    const int b_end = min(b_begin + geo.b_per_range, nb);
    for (int b = b_begin; b < b_end; ++b) {
        __syncthreads();   // previous slice fully consumed (and border initialised)
        const float* src = gamma + (int64_t)b * Ma;
        for (int64_t i = tid; i < Ma; i += kThreads) {
            const int r = (int)(i / wa), cc = (int)(i - (int64_t)r * wa);
            slice[(r + 1) * W2 + cc + 1] = __ldg(src + i);
        }
        const int br = b / wb, bc = b - br * wb;
        for (int i = tid; i < wa + ha; i += kThreads) {
            const bool is_x = i < wa;
            const int j = is_x ? i : i - wa;
            const int n = is_x ? wa : ha;
            const double u = is_x ? al * (j - cxa) + be * sx * (bc - cxb) + cxa
                                  : al * (j - cya) + be * sy * (br - cyb) + cya;
            const double f0 = floor(u);
            int off = 0;
            float w0 = 0.0f, w1 = 0.0f;
            if (f0 >= -1.0 && f0 <= (double)(n - 1)) {   // at least one tap inside the grid
                const double f = u - f0;
                off = (int)f0 + 1;                        // +1: zero border
                w0 = (float)(1.0 - f);
                w1 = (float)f;
            }
            if (is_x) {
                xoff[j] = off;
                xw0[j] = w0;
                xw1[j] = w1;
            } else {
                yoff[j] = off * W2;
                yw0[j] = w0;
                yw1[j] = w1;
            }
        }
        __syncthreads();
        if (active) {
            const int xo = xoff[c];
            const float wx0 = xw0[c], wx1 = xw1[c];
#pragma unroll
            for (int k = 0; k < kOpt; ++k) {
                const int r = row0 + rp + R * k;
                if (r < ha) {
                    const int base = yoff[r] + xo;
                    const float wy0 = yw0[r], wy1 = yw1[r];
                    const float v00 = slice[base], v01 = slice[base + 1];
                    const float v10 = slice[base + W2], v11 = slice[base + W2 + 1];
                    const float top = __fmaf_rn(wx1, v01, wx0 * v00);
                    const float bot = __fmaf_rn(wx1, v11, wx0 * v10);
                    const float smp = __fmaf_rn(wy1, bot, wy0 * top);
                    // Kahan-compensated accumulation over angular pixels
                    const float y = smp - cmp[k];
                    const float t = acc[k] + y;
                    cmp[k] = (t - acc[k]) - y;
                    acc[k] = t;
                }
            }
        }
    }
    if (!active) return;
    double* dst = partial + ((int64_t)blockIdx.x * geo.total_planes + geo.plane_offset + p) * Ma;
#pragma unroll
    for (int k = 0; k < kOpt; ++k) {
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

template <int kOpt>
cudaError_t launch_opt(const float* g, const RefocusGeom& geo, const PlaneBlock& pl,
                       double* partial, int zchunks, size_t smem, cudaStream_t st) {
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        e = cudaFuncSetAttribute(refocus_kernel<kOpt>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    dim3 grid((unsigned)geo.n_ranges, (unsigned)geo.n_planes, (unsigned)zchunks);
    refocus_kernel<kOpt><<<grid, kThreads, smem, st>>>(g, geo, pl, partial);
    return cudaGetLastError();
}

}  // namespace

size_t refocus_smem_bytes(int ha, int wa) {
    return sizeof(float) * ((size_t)(ha + 2) * (wa + 2) + 3 * (size_t)wa + 3 * (size_t)ha);
}

int refocus_ranges(int hb, int wb, int n_planes, int sm_count) {
    const int nb = hb * wb;
    int target = (4 * sm_count + n_planes - 1) / (n_planes > 0 ? n_planes : 1);
    if (target < 1) target = 1;
    if (target > nb) target = nb;
    const int per = (nb + target - 1) / target;
    return (nb + per - 1) / per;
}

cudaError_t launch_refocus(const float* gamma_f32, const RefocusGeom& geo, const PlaneBlock& pl,
                           double* partial, cudaStream_t st) {
    const int R = kThreads / geo.wa;
    const size_t smem = refocus_smem_bytes(geo.ha, geo.wa);
    int opt = 1;
    while (opt < 32 && R * opt < geo.ha) opt *= 2;
    const int zchunks = (geo.ha + R * opt - 1) / (R * opt);
    switch (opt) {
        case 1: return launch_opt<1>(gamma_f32, geo, pl, partial, zchunks, smem, st);
        case 2: return launch_opt<2>(gamma_f32, geo, pl, partial, zchunks, smem, st);
        case 4: return launch_opt<4>(gamma_f32, geo, pl, partial, zchunks, smem, st);
        case 8: return launch_opt<8>(gamma_f32, geo, pl, partial, zchunks, smem, st);
        case 16: return launch_opt<16>(gamma_f32, geo, pl, partial, zchunks, smem, st);
        default: return launch_opt<32>(gamma_f32, geo, pl, partial, zchunks, smem, st);
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
