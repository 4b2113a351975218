// 4-D multilinear refocusing (Section 4.1: the prototype interpolates Gamma in
// all four coordinates, the interpolation points depending on the plane).
// Plane p has four coefficients (alpha, beta, gamma, delta).  For output pixel
// x (centred spatial coordinates) and angular pixel j (centred), Gamma is
// sampled at
//     u_a = alpha x + beta (j in spatial pixels)      (spatial point)
//     u_b = gamma (x in angular pixels) + delta j     (angular point)
// by multilinear interpolation over the 16 neighbouring grid points (taps
// outside either grid count as 0), and the samples are summed over j.
// gamma = 0, delta = 1 is the 2-D refocusing of refocus.cu.
//
// The sample point separates into a column part (x_c, j_c) -> (xa, xb) and a
// row part (x_r, j_r) -> (ya, yb).  Stage 1 contracts the columns: for every
// pair of rows (ya, yb), Gamma restricted to them is a W_b x W_a matrix
// G[xb][xa] (one 2-D box of Gamma's slice-major layout), and
//     C[p][ya][yb][x_c] = sum_{j_c} sum_{xa, xb taps} w w G[xb][xa],
// one CTA per (ya, yb) for every plane of the chunk, the box staged in shared
// memory with a 2-pixel zero border (or read from global memory when it does
// not fit), Kahan-compensated over j_c and stored as a float pair (sum and
// compensation).  Stage 2 contracts the rows (a 1/W_b share of the work) in
// double-float FP32 arithmetic, exact up to one final rounding:
//     out[p][x_r][x_c] = sum_{j_r} sum_{ya, yb taps} w w C[p][ya][yb][x_c].
// Coordinates are 32.32 fixed point, A(x) + B(j), each rounded once from FP64;
// fractions rounded to 24 bits (exact weights).
//
// This file is compiled without FMA contraction (Kahan steps).
#include "kernels.cuh"

namespace cpi {
namespace {

constexpr int kPad = 2;              // zero border of the staged box
constexpr int kR4Threads = 256;

__device__ __forceinline__ long long r4_fix(double v) { return __double2ll_rn(v * 4294967296.0); }

struct R4Frac {
    int i;
    float f;
};
__device__ __forceinline__ R4Frac r4_split(long long u) {
    const long long u24 = (u + 128) >> 8;
    return {(int)(u24 >> 24), (float)(int)(u24 & 0xFFFFFF) * 0x1p-24f};
}

__device__ __forceinline__ void r4_kahan(float& acc, float& cmp, float v) {
    const float y = v - cmp;
    const float t = acc + y;
    cmp = (t - acc) - y;
    acc = t;
}

// Per-plane coordinate tables (fixed point), chunk planes p0 .. p0 + np - 1:
//   x axis: TAx[p][c] = alpha (c - cxa) + cxa,        TBx[p][j] = beta sx (j - cxb)
//           TAbx[p][c] = gamma (c - cxa) / sx + cxb,  TBbx[p][j] = delta (j - cxb)
//   y axis: the same with rows (ha, hb, sy).
__global__ void r4_tables_kernel(const Plane4Block co, int np, int ha, int wa, int hb, int wb,
                                 long long* __restrict__ t, int64_t stride) {
    const int p = blockIdx.x;
    if (p >= np) return;
    const double al = co.c[p][0], be = co.c[p][1], ga = co.c[p][2], de = co.c[p][3];
    const double cxa = 0.5 * (wa - 1), cya = 0.5 * (ha - 1), cxb = 0.5 * (wb - 1), cyb = 0.5 * (hb - 1);
    const double sx = (double)wa / (double)wb, sy = (double)ha / (double)hb;
    long long* TAx = t + 0 * stride + (int64_t)p * wa;
    long long* TAbx = t + 1 * stride + (int64_t)p * wa;
    long long* TBx = t + 2 * stride + (int64_t)p * wb;
    long long* TBbx = t + 3 * stride + (int64_t)p * wb;
    long long* TAy = t + 4 * stride + (int64_t)p * ha;
    long long* TAby = t + 5 * stride + (int64_t)p * ha;
    long long* TBy = t + 6 * stride + (int64_t)p * hb;
    long long* TBby = t + 7 * stride + (int64_t)p * hb;
    for (int c = threadIdx.x; c < wa; c += blockDim.x) {
        TAx[c] = r4_fix(al * (c - cxa) + cxa);
        TAbx[c] = r4_fix(ga * (c - cxa) / sx + cxb);
    }
    for (int j = threadIdx.x; j < wb; j += blockDim.x) {
        TBx[j] = r4_fix(be * sx * (j - cxb));
        TBbx[j] = r4_fix(de * (j - cxb));
    }
    for (int r = threadIdx.x; r < ha; r += blockDim.x) {
        TAy[r] = r4_fix(al * (r - cya) + cya);
        TAby[r] = r4_fix(ga * (r - cya) / sy + cyb);
    }
    for (int j = threadIdx.x; j < hb; j += blockDim.x) {
        TBy[j] = r4_fix(be * sy * (j - cyb));
        TBby[j] = r4_fix(de * (j - cyb));
    }
}

// Stage 1: CTA (yb, ya0 .. ya0 + K - 1): the K boxes of those row pairs; every
// plane of the chunk, G planes at a time; thread w of a pass takes plane
// p0 + w / wa and column x_c = w % wa (so narrow images still give every thread
// work).  The taps of (plane, x_c, j_c) do not depend on the row pair, so each is
// formed once and applied to all K boxes.  sB holds the G planes' angular-column
// tables.
constexpr int kColThreads = 512;
template <bool kSmem, int K>
__global__ void __launch_bounds__(kColThreads) r4_cols_kernel(const float* __restrict__ g, int np, int G, int ha,
                                                              int wa, int hb, int wb, const long long* __restrict__ t,
                                                              int64_t stride, float* __restrict__ c_hi,
                                                              float* __restrict__ c_lo) {
    extern __shared__ __align__(16) float sm[];
    const int yb = blockIdx.x, ya0 = blockIdx.y * K;
    const int nb = min(K, ha - ya0);                       // boxes of this CTA
    const int64_t ma = (int64_t)ha * wa;
    const int WP = wa + 2 * kPad, HP = wb + 2 * kPad;     // padded box: HP rows (xb) x WP columns (xa)
    const int BS = HP * WP;
    long long* sB = reinterpret_cast<long long*>(sm);      // [G][2][wb]: TBx, TBbx of the pass's planes
    float* box = reinterpret_cast<float*>(sB + 2 * (size_t)G * wb);   // [K][HP][WP]
    if constexpr (kSmem) {
        for (int k = 0; k < nb; ++k)
            for (int i = threadIdx.x; i < BS; i += kColThreads) {
                const int r = i / WP, q = i - r * WP;
                const int xb = r - kPad, xa = q - kPad;
                box[k * BS + i] = (xb >= 0 && xb < wb && xa >= 0 && xa < wa)
                                      ? g[(int64_t)(yb * wb + xb) * ma + (int64_t)(ya0 + k) * wa + xa]
                                      : 0.0f;
            }
    }
    for (int p0 = 0; p0 < np; p0 += G) {
        const int gp = min(G, np - p0);
        __syncthreads();   // boxes ready / previous pass's tables consumed
        for (int i = threadIdx.x; i < gp * wb; i += kColThreads) {
            const int k = i / wb, j = i - k * wb;
            sB[(2 * k) * wb + j] = t[2 * stride + (int64_t)(p0 + k) * wb + j];
            sB[(2 * k + 1) * wb + j] = t[3 * stride + (int64_t)(p0 + k) * wb + j];
        }
        __syncthreads();
        for (int w = threadIdx.x; w < gp * wa; w += kColThreads) {
            const int kp = w / wa, xc = w - kp * wa, p = p0 + kp;
            const long long* B = sB + 2 * kp * wb;
            const long long ax = t[0 * stride + (int64_t)p * wa + xc];
            const long long abx = t[1 * stride + (int64_t)p * wa + xc];
            float acc[K], cmp[K];
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k] = cmp[k] = 0.0f;
            for (int jc = 0; jc < wb; ++jc) {
                const R4Frac fa = r4_split(ax + B[jc]);
                const R4Frac fb = r4_split(abx + B[wb + jc]);
                const float ga = 1.0f - fa.f, gb = 1.0f - fb.f;
                if constexpr (kSmem) {
                    const int xa = min(max(fa.i, -kPad), wa) + kPad;
                    const int xb = min(max(fb.i, -kPad), wb) + kPad;
                    const float* q0 = box + xb * WP + xa;
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        if (k < nb) {
                            const float* q = q0 + k * BS;
                            const float top = __fmaf_rn(fa.f, q[1], ga * q[0]);
                            const float bot = __fmaf_rn(fa.f, q[WP + 1], ga * q[WP]);
                            r4_kahan(acc[k], cmp[k], __fmaf_rn(fb.f, bot, gb * top));
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        if (k < nb) {
                            const float* gbase = g + ((int64_t)yb * wb) * ma + (int64_t)(ya0 + k) * wa;
                            float s[2][2];
#pragma unroll
                            for (int db = 0; db < 2; ++db)
#pragma unroll
                                for (int da = 0; da < 2; ++da) {
                                    const int xa = fa.i + da, xb = fb.i + db;
                                    s[db][da] = (xa >= 0 && xa < wa && xb >= 0 && xb < wb)
                                                    ? __ldg(gbase + (int64_t)xb * ma + xa)
                                                    : 0.0f;
                                }
                            const float top = __fmaf_rn(fa.f, s[0][1], ga * s[0][0]);
                            const float bot = __fmaf_rn(fa.f, s[1][1], ga * s[1][0]);
                            r4_kahan(acc[k], cmp[k], __fmaf_rn(fb.f, bot, gb * top));
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (k < nb) {
                    const int64_t o = (((int64_t)p * ha + ya0 + k) * hb + yb) * wa + xc;
                    c_hi[o] = acc[k];
                    c_lo[o] = -cmp[k];
                }
            }
        }
    }
}

// (sh, sl) += wa * wb * (ch + cl) with error-free FP32 transformations: the
// weight product and the leading product are split exactly with fused
// multiply-adds (TwoProduct), the leading term is added by TwoSum; the
// remaining second-order terms go to sl.  The sum is exact up to O(u^2) per
// term; one rounding (sh + sl) ends it.
__device__ __forceinline__ void r4_df_add(float& sh, float& sl, float wa, float wb, float ch, float cl) {
    const float pw = wa * wb;
    const float ew = __fmaf_rn(wa, wb, -pw);
    const float th = pw * ch;
    float te = __fmaf_rn(pw, ch, -th);
    te = __fmaf_rn(pw, cl, __fmaf_rn(ew, ch, te));
    const float s = sh + th;
    const float bb = s - sh;
    const float err = (sh - (s - bb)) + (th - bb);
    sl = sl + (err + te);
    sh = s;
}

// Stage 2: CTA (block of G output rows, plane); thread w takes row
// blockIdx.x * G + w / wa and column w % wa.  Double-float sums (r4_df_add).
__global__ void __launch_bounds__(kR4Threads) r4_rows_kernel(const float* __restrict__ c_hi,
                                                             const float* __restrict__ c_lo, int G, int ha, int wa,
                                                             int hb, const long long* __restrict__ t, int64_t stride,
                                                             float* __restrict__ out) {
    const int p = blockIdx.y;
    for (int w = threadIdx.x; w < G * wa; w += kR4Threads) {
        const int k = w / wa, xc = w - k * wa, xr = blockIdx.x * G + k;
        if (xr >= ha) continue;
        const long long ay = t[4 * stride + (int64_t)p * ha + xr];
        const long long aby = t[5 * stride + (int64_t)p * ha + xr];
        float sh = 0.0f, sl = 0.0f;
        for (int jr = 0; jr < hb; ++jr) {
            const R4Frac fa = r4_split(ay + t[6 * stride + (int64_t)p * hb + jr]);
            const R4Frac fb = r4_split(aby + t[7 * stride + (int64_t)p * hb + jr]);
#pragma unroll
            for (int db = 0; db < 2; ++db) {
                const int yb = fb.i + db;
                if (yb < 0 || yb >= hb) continue;
                const float wbw = db ? fb.f : 1.0f - fb.f;
#pragma unroll
                for (int da = 0; da < 2; ++da) {
                    const int ya = fa.i + da;
                    if (ya < 0 || ya >= ha) continue;
                    const float waw = da ? fa.f : 1.0f - fa.f;
                    const int64_t o = (((int64_t)p * ha + ya) * hb + yb) * wa + xc;
                    r4_df_add(sh, sl, waw, wbw, c_hi[o], c_lo[o]);
                }
            }
        }
        out[((int64_t)p * ha + xr) * wa + xc] = sh + sl;
    }
}

}  // namespace

Refocus4dLayout refocus4d_layout(int ha, int wa, int hb, int wb, int n_planes) {
    Refocus4dLayout L{};
    const int64_t per_plane = (int64_t)ha * hb * wa;          // C entries per plane
    int chunk = n_planes < kRefocus4dChunk ? n_planes : kRefocus4dChunk;
    while (chunk > 1 && (int64_t)chunk * per_plane * 8 > ((int64_t)4 << 30)) chunk /= 2;
    L.chunk = chunk;
    int m = ha;
    if (wa > m) m = wa;
    if (hb > m) m = hb;
    if (wb > m) m = wb;
    L.stride = (int64_t)chunk * m;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 255) / 256 * 256;
        return at;
    };
    L.tables = take(sizeof(long long) * 8 * (size_t)L.stride);
    L.c_hi = take(sizeof(float) * (size_t)(chunk * per_plane));
    L.c_lo = take(sizeof(float) * (size_t)(chunk * per_plane));
    L.bytes = o;
    return L;
}

namespace {
// planes per pass of the column stage
int r4_col_group(int wa, int wb, int np) {
    int G = wa < kColThreads ? kColThreads / wa : 1;
    if (G > np) G = np;
    while (G > 1 && (size_t)G * 2 * wb * sizeof(long long) > 16 * 1024) --G;
    return G < 1 ? 1 : G;
}
size_t r4_box_bytes(int wa, int wb) { return sizeof(float) * (size_t)(wb + 2 * kPad) * (wa + 2 * kPad); }
constexpr size_t kR4SmemCap = 200 * 1024;

template <bool kSmem, int K>
cudaError_t launch_cols(const float* g, int np, int G, int ha, int wa, int hb, int wb, const long long* t,
                        int64_t stride, float* c_hi, float* c_lo, size_t smem, cudaStream_t st) {
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        if ((e = cudaFuncSetAttribute(r4_cols_kernel<kSmem, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kR4SmemCap)) != cudaSuccess)
            return e;
        attr[dev] = true;
    }
    const dim3 grid((unsigned)hb, (unsigned)((ha + K - 1) / K));
    r4_cols_kernel<kSmem, K><<<grid, kColThreads, smem, st>>>(g, np, G, ha, wa, hb, wb, t, stride, c_hi, c_lo);
    return cudaGetLastError();
}
}  // namespace

bool refocus4d_box_fits(int wa, int wb) {
    return sizeof(long long) * 2 * (size_t)wb + r4_box_bytes(wa, wb) <= kR4SmemCap;
}

cudaError_t launch_refocus4d_chunk(const float* gamma_f32, int ha, int wa, int hb, int wb, const Plane4Block& coef,
                                   int np, uint8_t* ws, const Refocus4dLayout& L, float* out, cudaStream_t st) {
    long long* t = reinterpret_cast<long long*>(ws + L.tables);
    float* c_hi = reinterpret_cast<float*>(ws + L.c_hi);
    float* c_lo = reinterpret_cast<float*>(ws + L.c_lo);
    r4_tables_kernel<<<np, 128, 0, st>>>(coef, np, ha, wa, hb, wb, t, L.stride);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int G = r4_col_group(wa, wb, np);
    if (refocus4d_box_fits(wa, wb)) {
        const size_t box = r4_box_bytes(wa, wb);
        while (G > 1 && sizeof(long long) * 2 * (size_t)G * wb + box > kR4SmemCap) --G;
        const size_t tab = sizeof(long long) * 2 * (size_t)G * wb;
        // boxes per CTA: as many row pairs (4, 2, 1) as fit, while the grid
        // keeps at least ~4 CTAs per SM of a 152-SM GPU
        int K = 1;
        for (int k : {4, 2})
            if (tab + k * box <= kR4SmemCap && (int64_t)hb * ((ha + k - 1) / k) >= 4 * 152) {
                K = k;
                break;
            }
        const size_t smem = tab + K * box;
        if (K == 4) e = launch_cols<true, 4>(gamma_f32, np, G, ha, wa, hb, wb, t, L.stride, c_hi, c_lo, smem, st);
        else if (K == 2) e = launch_cols<true, 2>(gamma_f32, np, G, ha, wa, hb, wb, t, L.stride, c_hi, c_lo, smem, st);
        else e = launch_cols<true, 1>(gamma_f32, np, G, ha, wa, hb, wb, t, L.stride, c_hi, c_lo, smem, st);
    } else {
        e = launch_cols<false, 1>(gamma_f32, np, G, ha, wa, hb, wb, t, L.stride, c_hi, c_lo,
                                  sizeof(long long) * 2 * (size_t)G * wb, st);
    }
    if (e != cudaSuccess) return e;
    const int Gr = wa < kR4Threads ? kR4Threads / wa : 1;
    r4_rows_kernel<<<dim3((unsigned)((ha + Gr - 1) / Gr), (unsigned)np), kR4Threads, 0, st>>>(c_hi, c_lo, Gr, ha, wa,
                                                                                            hb, t, L.stride, out);
    return cudaGetLastError();
}

}  // namespace cpi
