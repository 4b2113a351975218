/*
 * Plain CPU oracle for correlation plenoptic imaging (CPI).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement
 * of what the GPU path computes.  It is used by the tests, by the smoke check and
 * by the benchmark's CPU-baseline leg, and by nothing else; the library never
 * links, loads or calls it.  It shares no code, header or table with the CUDA
 * path.
 *
 * What it computes:
 *   - pixel values of a frame region, read from the SwissSPAD2-style layout of
 *     the paper's Section 2 (A and B images side by side; 1 bit/pixel packed, or
 *     1 byte/pixel);
 *   - the correlation function of Eq. (1) (Section "CPI algorithm", item 1):
 *        Gamma[a][b] = (1/N) sum_i A_i[a] B_i[b] - (1/N sum_i A_i[a]) (1/N sum_i B_i[b]),
 *     written with exact integer sums S_ab, S_a, S_b and one rounding:
 *        Gamma = (double)(N*S_ab - S_a*S_b) / ((double)N * (double)N);
 *   - refocusing (Section "CPI algorithm", item 2; Section 4.1 "Refocusing
 *     Optimization"): for a plane (alpha, beta), the refocused image is the sum
 *     over every angular pixel rho_b of Gamma(., rho_b) sampled bilinearly at
 *     alpha*x + beta*rho_b~, evaluated directly in double precision.
 *
 * Readings of points the paper leaves open (each is listed in the design notes):
 *   - Gamma is stored row-major as [A pixel][B pixel], pixel index y*width + x;
 *   - bits are read least-significant-bit first unless bit_order == 1;
 *   - x, rho_b are centred pixel coordinates, rho_b~ = rho_b * (W_a/W_b, H_a/H_b);
 *     bilinear taps outside the spatial grid contribute 0; the output is the
 *     plain sum over rho_b.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no FMA contraction, so
 * x86-64 and aarch64 hosts give identical doubles).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    const uint8_t *data;       /* frame 0 */
    int32_t bits;              /* 1 or 8 */
    int32_t height, width;     /* region size */
    int32_t x0, y0;            /* region origin in the frame */
    int64_t row_stride;        /* pixels between consecutive frame rows */
    int64_t frame_stride_bytes;
    int32_t bit_order;         /* 0: LSB first, 1: MSB first */
} oracle_frames;

/* Pixel value of pixel p = y*width + x of frame i (Section 2 layout). */
static inline uint32_t oracle_pixel(const oracle_frames *d, int64_t i, int64_t p)
{
    int64_t y = p / d->width, x = p % d->width;
    int64_t e = (d->y0 + y) * d->row_stride + (d->x0 + x);
    const uint8_t *f = d->data + i * d->frame_stride_bytes;
    if (d->bits == 8) return f[e];
    uint32_t byte = f[e >> 3];
    int sh = (int)(e & 7);
    if (d->bit_order == 1) sh = 7 - sh;
    return (byte >> sh) & 1u;
}

/* out[p*n + i] = value of pixel p in frame i (pixel-major). */
int oracle_unpack(const oracle_frames *d, int64_t n, uint8_t *out)
{
    int64_t M = (int64_t)d->height * d->width;
    if (d->bits != 1 && d->bits != 8) return 1;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < M; ++p)
        for (int64_t i = 0; i < n; ++i) out[p * n + i] = (uint8_t)oracle_pixel(d, i, p);
    return 0;
}

/*
 * Eq. (1).  Rows [row_begin, row_end) of S_ab and Gamma (all rows when
 * row_end <= row_begin), S_a and S_b in full.  s_ab / gamma are indexed by the
 * full row number (a*Mb + b), so a caller sampling rows passes full-size arrays or
 * offsets them.  gamma may be NULL.  Returns 0, or 2 if N*S_ab could overflow int64.
 */
int oracle_correlate(const oracle_frames *A, const oracle_frames *B, int64_t n,
                     int64_t row_begin, int64_t row_end,
                     int64_t *s_ab, int64_t *s_a, int64_t *s_b, double *gamma)
{
    int64_t Ma = (int64_t)A->height * A->width, Mb = (int64_t)B->height * B->width;
    if (n <= 0 || Ma <= 0 || Mb <= 0) return 1;
    if (row_end <= row_begin) { row_begin = 0; row_end = Ma; }
    double vmax_a = A->bits == 1 ? 1.0 : 255.0, vmax_b = B->bits == 1 ? 1.0 : 255.0;
    /* |N*S_ab| <= N^2 * maxA * maxB must stay below 2^63 */
    if ((double)n * (double)n * vmax_a * vmax_b >= 9.2e18) return 2;

    uint8_t *ua = (uint8_t *)malloc((size_t)Ma * (size_t)n);
    uint8_t *ub = (uint8_t *)malloc((size_t)Mb * (size_t)n);
    if (!ua || !ub) { free(ua); free(ub); return 3; }
    oracle_unpack(A, n, ua);
    oracle_unpack(B, n, ub);

    /* marginal sums of Eq. (1): S_a = sum_i A_i, S_b = sum_i B_i */
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < Ma; ++a) {
        int64_t s = 0;
        for (int64_t i = 0; i < n; ++i) s += ua[a * n + i];
        s_a[a] = s;
    }
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < Mb; ++b) {
        int64_t s = 0;
        for (int64_t i = 0; i < n; ++i) s += ub[b * n + i];
        s_b[b] = s;
    }
    /* raw moment S_ab = sum_i A_i[a] * B_i[b], then the mean subtraction */
    const double nd = (double)n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t a = row_begin; a < row_end; ++a) {
        const uint8_t *pa = ua + a * n;
        for (int64_t b = 0; b < Mb; ++b) {
            const uint8_t *pb = ub + b * n;
            int64_t s = 0;
            for (int64_t i = 0; i < n; ++i) s += (int64_t)((uint32_t)pa[i] * (uint32_t)pb[i]);
            s_ab[a * Mb + b] = s;
            if (gamma) {
                int64_t num = n * s - s_a[a] * s_b[b];
                gamma[a * Mb + b] = (double)num / (nd * nd);
            }
        }
    }
    free(ua);
    free(ub);
    return 0;
}

/*
 * Refocusing, evaluated directly in double precision.
 *   gamma  : [Ma][Mb] row-major, Ma = ha*wa spatial pixels, Mb = hb*wb angular pixels
 *   planes : alpha[p], beta[p]
 *   out    : [n_planes][ha][wa]
 * For output pixel (r, c) of plane p:
 *   u_x = alpha*(c - cxa) + beta*sx*(bc - cxb) + cxa,  u_y likewise with rows,
 *   cxa = (wa-1)/2, cxb = (wb-1)/2, sx = wa/wb (and cya, cyb, sy for rows);
 *   out = sum over (br, bc) of the bilinear interpolation of Gamma[., (br, bc)]
 *         at (u_y, u_x), taps outside the ha x wa grid counting as 0.
 */
int oracle_refocus(const double *gamma, int32_t ha, int32_t wa, int32_t hb, int32_t wb,
                   const double *alpha, const double *beta, int32_t n_planes, double *out)
{
    if (ha <= 0 || wa <= 0 || hb <= 0 || wb <= 0 || n_planes < 0) return 1;
    const int64_t Mb = (int64_t)hb * wb;
    const double cxa = (wa - 1) / 2.0, cya = (ha - 1) / 2.0;
    const double cxb = (wb - 1) / 2.0, cyb = (hb - 1) / 2.0;
    const double sx = (double)wa / (double)wb, sy = (double)ha / (double)hb;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int32_t p = 0; p < n_planes; ++p) {
        for (int32_t r = 0; r < ha; ++r) {
            const double al = alpha[p], be = beta[p];
            for (int32_t c = 0; c < wa; ++c) {
                double acc = 0.0;
                for (int32_t br = 0; br < hb; ++br) {
                    double uy = al * (r - cya) + be * sy * (br - cyb) + cya;
                    double fy0 = floor(uy);
                    double fy = uy - fy0;
                    int64_t y0 = (int64_t)fy0;
                    for (int32_t bc = 0; bc < wb; ++bc) {
                        double ux = al * (c - cxa) + be * sx * (bc - cxb) + cxa;
                        double fx0 = floor(ux);
                        double fx = ux - fx0;
                        int64_t x0 = (int64_t)fx0;
                        int64_t b = (int64_t)br * wb + bc;
                        for (int dy = 0; dy <= 1; ++dy) {
                            int64_t yy = y0 + dy;
                            if (yy < 0 || yy >= ha) continue;
                            double wy = dy ? fy : 1.0 - fy;
                            for (int dx = 0; dx <= 1; ++dx) {
                                int64_t xx = x0 + dx;
                                if (xx < 0 || xx >= wa) continue;
                                double wx = dx ? fx : 1.0 - fx;
                                acc += wy * wx * gamma[(yy * wa + xx) * Mb + b];
                            }
                        }
                    }
                }
                out[((int64_t)p * ha + r) * wa + c] = acc;
            }
        }
    }
    return 0;
}

/*
 * 4-D multilinear refocusing (Section 4.1: the prototype interpolates Gamma in
 * all four coordinates, the points depending on the plane).  Reading: plane p
 * has four coefficients (alpha, beta, gamma, delta); for output pixel x
 * (centred spatial coordinates) and angular pixel j (centred), Gamma is sampled
 * at the spatial point  u_a = alpha*x + beta*(j scaled to spatial pixels)  and
 * the angular point     u_b = gamma*(x scaled to angular pixels) + delta*j,
 * by multilinear interpolation over the 2 x 2 x 2 x 2 neighbouring grid points
 * (taps outside either grid count as 0), and the samples are summed over j.
 * gamma = 0, delta = 1 is the refocusing of oracle_refocus.
 *   planes : alpha[p], beta[p], gam[p], delta[p]
 */
int oracle_refocus4d(const double *g, int32_t ha, int32_t wa, int32_t hb, int32_t wb,
                     const double *alpha, const double *beta, const double *gam, const double *delta,
                     int32_t n_planes, double *out)
{
    if (ha <= 0 || wa <= 0 || hb <= 0 || wb <= 0 || n_planes < 0) return 1;
    const int64_t Mb = (int64_t)hb * wb;
    const double cxa = (wa - 1) / 2.0, cya = (ha - 1) / 2.0;
    const double cxb = (wb - 1) / 2.0, cyb = (hb - 1) / 2.0;
    const double sx = (double)wa / (double)wb, sy = (double)ha / (double)hb;   /* angular -> spatial */
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int32_t p = 0; p < n_planes; ++p) {
        for (int32_t r = 0; r < ha; ++r) {
            const double al = alpha[p], be = beta[p], ga = gam[p], de = delta[p];
            for (int32_t c = 0; c < wa; ++c) {
                double acc = 0.0;
                for (int32_t jr = 0; jr < hb; ++jr) {
                    const double uay = al * (r - cya) + be * sy * (jr - cyb) + cya;
                    const double uby = ga * (r - cya) / sy + de * (jr - cyb) + cyb;
                    const double fay0 = floor(uay), fby0 = floor(uby);
                    const double fay = uay - fay0, fby = uby - fby0;
                    for (int32_t jc = 0; jc < wb; ++jc) {
                        const double uax = al * (c - cxa) + be * sx * (jc - cxb) + cxa;
                        const double ubx = ga * (c - cxa) / sx + de * (jc - cxb) + cxb;
                        const double fax0 = floor(uax), fbx0 = floor(ubx);
                        const double fax = uax - fax0, fbx = ubx - fbx0;
                        for (int t = 0; t < 16; ++t) {
                            const int dya = t & 1, dxa = (t >> 1) & 1, dyb = (t >> 2) & 1, dxb = (t >> 3) & 1;
                            const int64_t ya = (int64_t)fay0 + dya, xa = (int64_t)fax0 + dxa;
                            const int64_t yb = (int64_t)fby0 + dyb, xb = (int64_t)fbx0 + dxb;
                            if (ya < 0 || ya >= ha || xa < 0 || xa >= wa) continue;
                            if (yb < 0 || yb >= hb || xb < 0 || xb >= wb) continue;
                            const double w = (dya ? fay : 1.0 - fay) * (dxa ? fax : 1.0 - fax) *
                                             (dyb ? fby : 1.0 - fby) * (dxb ? fbx : 1.0 - fbx);
                            acc += w * g[(ya * wa + xa) * Mb + yb * wb + xb];
                        }
                    }
                }
                out[((int64_t)p * ha + r) * wa + c] = acc;
            }
        }
    }
    return 0;
}

/* Number of threads an OpenMP parallel region of this library uses. */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
