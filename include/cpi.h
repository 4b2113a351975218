/*
 * cpi.h -- C ABI of the GB300 (sm_103a) correlation plenoptic imaging library.
 *
 * The library computes the two steps of the CPI processing chain described in
 * "GPU-based data processing for speeding-up correlation plenoptic imaging"
 * (arXiv 2407.20692):
 *   1. the correlation function Gamma of Eq. (1) (Section "CPI algorithm",
 *      item 1) between the frames of a spatial detector A and an angular
 *      detector B, and
 *   2. refocusing of Gamma into a stack of planes (Section "CPI algorithm",
 *      item 2; Section 4.1, "Refocusing Optimization").
 *
 * Conventions for every entry point:
 *   - Every buffer pointer is DEVICE memory owned by the caller, unless marked
 *     "host".  The library never allocates device memory; scratch space is a
 *     caller-provided workspace whose size is given by the *_workspace_size
 *     queries.  The library keeps no pointer after a call returns.
 *   - Work is enqueued asynchronously on `stream` (NULL = legacy default stream).
 *     Argument errors are detected on the host and returned before anything is
 *     launched.  A launch failure returns CPI_ERR_CUDA.
 *   - Errors found by a kernel while it runs (a pipeline wait that exceeded its
 *     time limit) are recorded in a per-device status word and returned by
 *     cpi_device_status(); kernels never trap.
 *   - Gamma and the raw sums use the index map row = A pixel, column = B pixel,
 *     pixel index = y * width + x inside each image's region of interest.
 *   - Not thread-safe for concurrent calls that share a workspace.
 */
#ifndef CPI_H
#define CPI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define CPI_API __attribute__((visibility("default")))
#else
#define CPI_API
#endif

struct CUstream_st;
typedef struct CUstream_st *cpi_stream; /* a cudaStream_t */

typedef enum cpi_status {
    CPI_OK = 0,
    CPI_ERR_INVALID_ARG = 1, /* a NULL/misaligned pointer, a bad size or descriptor */
    CPI_ERR_OVERFLOW = 2,    /* N^2 * max(A) * max(B) >= 2^63: int64 exactness not guaranteed */
    CPI_ERR_WORKSPACE = 3,   /* workspace NULL or smaller than the size query */
    CPI_ERR_UNSUPPORTED = 4, /* a valid request this build does not implement */
    CPI_ERR_CUDA = 5,        /* a CUDA runtime call or kernel launch failed */
    CPI_ERR_TIMEOUT = 6      /* a device-side wait ran out of its time limit */
} cpi_status;

/*
 * Frames of one detector image (Section 2 of the paper: each SwissSPAD2 frame is
 * a 256 x 512 image holding A on the left and B on the right, 1 bit per pixel).
 * Pixel (y, x) of the region, frame i, is element
 *     e = (y0 + y) * row_stride + (x0 + x)
 * of frame i, which starts at byte i * frame_stride_bytes of `data`:
 *   bits == 8: byte e;   bits == 1: bit (e % 8) of byte e / 8, counted from the
 *   least significant bit (bit_order 0) or the most significant (bit_order 1).
 * A and B may point into the same frame buffer with different regions.
 */
typedef struct cpi_frames {
    const void *data;           /* device pointer to frame 0; caller-owned */
    int32_t bits;               /* 1 (bit-packed binary frames) or 8 (uint8 counts) */
    int32_t height, width;      /* region size in pixels, each >= 1 */
    int32_t x0, y0;             /* region origin inside the frame, >= 0 */
    int64_t row_stride;         /* elements (pixels) between frame rows, >= x0 + width */
    int64_t frame_stride_bytes; /* bytes between consecutive frames, > 0 */
    int32_t bit_order;          /* 0 = LSB first, 1 = MSB first (bits == 1 only) */
} cpi_frames;

/* One refocusing plane: sample point alpha * x + beta * rho_b~ (see cpi_refocus). */
typedef struct cpi_plane {
    double alpha, beta;
} cpi_plane;

/* Human-readable name of a status code (static string). */
CPI_API const char *cpi_status_string(cpi_status s);

/* ABI version of this header: 1. */
CPI_API int32_t cpi_abi_version(void);

/* --------------------------------------------------------------------------
 * Correlation function, Eq. (1):
 *   Gamma[a][b] = (1/N) sum_i A_i[a] B_i[b] - (1/N sum_i A_i[a]) (1/N sum_i B_i[b])
 * computed as exact integer sums
 *   S_ab[a][b] = sum_i A_i[a] B_i[b],  S_a[a] = sum_i A_i[a],  S_b[b] = sum_i B_i[b]
 * and one correctly rounded double division of the exact int64 numerator:
 *   Gamma = (double)(N * S_ab - S_a * S_b) / ((double)N * (double)N).
 * The integer products run on the tensor cores with exact FP32 partial sums
 * (every partial sum is an integer below 2^24) folded into int32/int64, so S_ab,
 * S_a, S_b are bit-exact and Gamma is bit-identical to the exact-numerator
 * formula.  (Section "CPI algorithm"; Section 4.1, "Cross-correlation
 * Optimization": the binary frames stay bit-packed in memory and are unpacked
 * inside the correlation path.)
 *
 * Shapes: M_a = a->height * a->width, M_b = b->height * b->width.
 *   s_ab  : int64 [M_a][M_b] row-major; may be NULL (not written) when gamma or
 *           gamma_f32 is given, except for accumulating calls
 *   s_a   : int64 [M_a],  s_b : int64 [M_b]; may be NULL (then kept in the
 *           workspace), except for accumulating calls
 *   gamma : double [M_a][M_b] row-major, or NULL to skip
 *   gamma_f32 : float [M_b][M_a] ("slice-major": one M_a image per angular
 *           pixel, the input layout of cpi_refocus), or NULL to skip
 * Requirements: 1 <= n_frames; N^2 * max(A) * max(B) < 2^63 (else
 * CPI_ERR_OVERFLOW); M_a, M_b <= 2^24; output pointers 16-byte aligned.
 * -------------------------------------------------------------------------- */

/* Workspace bytes cpi_correlate / cpi_correlate_accumulate / cpi_correlate_stage
 * need for these descriptors and n_frames (0 on invalid arguments). */
CPI_API size_t cpi_correlate_workspace_size(const cpi_frames *a, const cpi_frames *b, int64_t n_frames);

/* Whole Eq. (1): overwrites s_ab, s_a, s_b, and gamma / gamma_f32 when non-NULL. */
CPI_API cpi_status cpi_correlate(const cpi_frames *a, const cpi_frames *b, int64_t n_frames,
                         int64_t *s_ab, int64_t *s_a, int64_t *s_b, double *gamma,
                         float *gamma_f32, void *workspace, size_t workspace_bytes,
                         cpi_stream stream);

/* Streaming form (the paper processes the acquisition in blocks of files):
 * ADDS this block's sums into s_ab, s_a, s_b (all three required).  Call
 * cpi_correlate_finalize with the total frame count once every block has been
 * added.  The running sums are the complete state of a correlation, so saving
 * them checkpoints it. */
CPI_API cpi_status cpi_correlate_accumulate(const cpi_frames *a, const cpi_frames *b, int64_t n_frames,
                                    int64_t *s_ab, int64_t *s_a, int64_t *s_b, void *workspace,
                                    size_t workspace_bytes, cpi_stream stream);

/* Gamma from accumulated sums: n_total frames in all (1 <= n_total < 2^31,
 * else CPI_ERR_OVERFLOW); m_a x m_b entries; any int64 sums.  The numerator
 * n_total * s_ab - s_a * s_b is formed exactly in 128 bits (sums added over many
 * blocks can make the products leave int64 although each block passed the
 * per-call check), rounded once to double and divided by RN(n_total^2):
 * bit-identical to the exact-numerator formula whenever the numerator fits
 * int64.  gamma and/or gamma_f32 (layouts as above) may be NULL, not both. */
CPI_API cpi_status cpi_correlate_finalize(const int64_t *s_ab, const int64_t *s_a, const int64_t *s_b,
                                  int64_t m_a, int64_t m_b, int64_t n_total, double *gamma,
                                  float *gamma_f32, cpi_stream stream);

/* The three steps of cpi_correlate as separate calls, for timing and for
 * overlapping them with other work.  Call them in order with identical
 * arguments and the same workspace:
 *   CPI_STAGE_INGEST : frames -> tensor-core operands (in the workspace) and the
 *                      marginal sums s_a, s_b (Eq. (1) second term);
 *   CPI_STAGE_MOMENTS: the raw-moment contraction sum_i A_i[a] B_i[b] into exact
 *                      int32 partial sums per frame chunk (in the workspace);
 *   CPI_STAGE_FOLD   : partial sums -> s_ab (int64), then gamma / gamma_f32 if
 *                      non-NULL (with N = n_frames).
 * accumulate != 0 adds into s_ab, s_a, s_b instead of overwriting them; such a
 * call writes no Gamma (gamma and gamma_f32 must be NULL, else
 * CPI_ERR_INVALID_ARG): use cpi_correlate_finalize with the total frame count. */
enum { CPI_STAGE_INGEST = 1, CPI_STAGE_MOMENTS = 2, CPI_STAGE_FOLD = 3 };
CPI_API cpi_status cpi_correlate_stage(int32_t stage, const cpi_frames *a, const cpi_frames *b,
                               int64_t n_frames, int32_t accumulate, int64_t *s_ab, int64_t *s_a,
                               int64_t *s_b, double *gamma, float *gamma_f32, void *workspace,
                               size_t workspace_bytes, cpi_stream stream);

/* --------------------------------------------------------------------------
 * Streamed acquisitions: Eq. (1) fed block by block from HOST memory while the
 * frames are being acquired (the paper processes an acquisition in blocks of
 * files, Section 4.1; a SPAD camera delivers ~10^5 binary frames per second,
 * Section 1).  The acquisition keeps two staging buffers in the caller's
 * workspace: the copy of one block to the GPU runs on the acquisition's own
 * copy stream while the previous block is accumulated (as
 * cpi_correlate_accumulate) on the caller's stream.  The running sums s_ab,
 * s_a, s_b and the frame count are the whole state of the correlation:
 * cpi_acq_sync makes them consistent (a checkpoint), and cpi_acq_begin with
 * frames_done > 0 resumes from saved sums.  Between checkpoints s_ab may lag
 * the pushed frames: for binary frames the sums of full blocks stay in the
 * workspace until the next cpi_acq_sync, cpi_acq_finalize, cpi_acq_end or a
 * block of fewer frames.
 *
 * Layout: a and b describe the two regions inside ONE frame buffer (their
 * `data` is ignored; both must have the same frame_stride_bytes); a host block
 * holds n consecutive frames of frame_stride_bytes each (e.g. the paper's .bin
 * files: 512 frames of 256 x 512 bits, A left, B right).
 *
 * cpi_acq_workspace_size : DEVICE workspace bytes for blocks of up to
 *        block_frames frames (0 on invalid layouts).
 * cpi_acq_begin : creates the handle (host memory; one CUDA stream and four
 *        events).  s_ab [M_a][M_b], s_a [M_a], s_b [M_b]: DEVICE int64,
 *        caller-owned; zeroed on `stream` when frames_done == 0, else they must
 *        hold the sums of the first frames_done frames.  `stream` is where the
 *        accumulation and cpi_acq_finalize run.  Make calls on the device that
 *        was current at cpi_acq_begin.
 * cpi_acq_push : enqueues one block of 1 <= n_frames <= block_frames frames
 *        from host memory (pinned memory lets the copy overlap).  Returns once
 *        the copy of the PREVIOUS block has completed: the caller may overwrite
 *        a host block as soon as the following cpi_acq_push (or cpi_acq_sync /
 *        cpi_acq_end) has returned.  CPI_ERR_OVERFLOW once the total would
 *        reach 2^31 frames.
 * cpi_acq_frames : frames pushed so far (including frames_done), -1 on NULL.
 * cpi_acq_finalize : enqueues Gamma of every frame pushed so far (as
 *        cpi_correlate_finalize) on `stream`; the acquisition continues.
 * cpi_acq_sync : waits for every copy and accumulation enqueued so far.
 * cpi_acq_end : cpi_acq_sync, then releases the handle.
 * -------------------------------------------------------------------------- */
typedef struct cpi_acq cpi_acq;
CPI_API size_t cpi_acq_workspace_size(const cpi_frames *a, const cpi_frames *b, int64_t block_frames);
CPI_API cpi_status cpi_acq_begin(cpi_acq **out, const cpi_frames *a, const cpi_frames *b, int64_t block_frames,
                                 int64_t *s_ab, int64_t *s_a, int64_t *s_b, int64_t frames_done, void *workspace,
                                 size_t workspace_bytes, cpi_stream stream);
CPI_API cpi_status cpi_acq_push(cpi_acq *acq, const void *host_frames, int64_t n_frames);
CPI_API int64_t cpi_acq_frames(const cpi_acq *acq);
CPI_API cpi_status cpi_acq_finalize(cpi_acq *acq, double *gamma, float *gamma_f32);
CPI_API cpi_status cpi_acq_sync(cpi_acq *acq);
CPI_API cpi_status cpi_acq_end(cpi_acq *acq);

/* --------------------------------------------------------------------------
 * Refocusing (Section "CPI algorithm", item 2; Section 4.1, "Refocusing
 * Optimization": interpolation coordinates are computed on the fly inside the
 * refocusing kernel).  The paper gives no formula; this library implements the
 * per-plane shift-and-sum of Gamma over the angular pixels with bilinear
 * interpolation in the spatial coordinate:
 *   x  = (c - (wa-1)/2, r - (ha-1)/2)             centred spatial pixel (r, c)
 *   rb = ((bc - (wb-1)/2) * wa/wb, (br - (hb-1)/2) * ha/hb)   scaled angular pixel
 *   out[p][r][c] = sum over (br, bc) of  Gamma~(alpha_p * x + beta_p * rb ; (br, bc))
 * where Gamma~(u; b) interpolates the spatial image Gamma[.][b] bilinearly at
 * the centred point u, taps outside the ha x wa grid counting as 0.
 * (alpha, beta) = (1, 0) is the plane the spatial detector is focused on.
 *
 *   gamma_f32 : float [hb*wb][ha*wa], slice-major (cpi_correlate's gamma_f32)
 *   planes    : HOST array of n_planes (alpha, beta), |alpha|, |beta| <= 1e6
 *               (else CPI_ERR_INVALID_ARG)
 *   out       : float [n_planes][ha][wa]
 * Sums use compensated FP32 accumulation; coordinates are computed on the fly
 * in 32.32 fixed point from FP64 products, and each interpolation fraction is
 * rounded to 24 bits (the two weights are exact and sum to 1).  Requires
 * ha, wa, hb, wb >= 1, wa <= 512, hb <= 12800, hb*wb*ha < 2^31 - 1024,
 * gamma_f32 16-byte aligned; Gamma values must be finite (a non-finite value
 * may reach outputs through zero-weight taps).  Any image height: the spatial
 * image is processed in bands of rows.
 * -------------------------------------------------------------------------- */
CPI_API size_t cpi_refocus_workspace_size(int32_t ha, int32_t wa, int32_t hb, int32_t wb,
                                  int32_t n_planes);

CPI_API cpi_status cpi_refocus(const float *gamma_f32, int32_t ha, int32_t wa, int32_t hb, int32_t wb,
                       const cpi_plane *planes, int32_t n_planes, float *out, void *workspace,
                       size_t workspace_bytes, cpi_stream stream);

/* --------------------------------------------------------------------------
 * 4-D multilinear refocusing (Section 4.1: the prototype interpolates Gamma in
 * all four coordinates, the interpolation points depending on the refocusing
 * plane).  Plane p has four coefficients; with x and rb as in cpi_refocus and
 * the angular pixel j (centred), Gamma is sampled at
 *   spatial point  u_a = alpha_p * x + beta_p * rb
 *   angular point  u_b = gamma_p * (x scaled to angular pixels: x * wb/wa, hb/ha) + delta_p * j
 * by multilinear interpolation over the 16 neighbouring grid points (taps
 * outside either grid count as 0), and the samples are summed over j:
 *   out[p][r][c] = sum over j of Gamma~(u_a, u_b).
 * gamma = 0, delta = 1 is cpi_refocus.  Error: at most ~1e-6 of
 * max|Gamma| times the total in-grid interpolation weight of the output
 * (compensated FP32 sums over the angular columns; over the rows, FP32
 * double-float sums rounded once).
 *
 *   gamma_f32 : float [hb*wb][ha*wa], slice-major (as cpi_refocus)
 *   planes    : HOST array of n_planes cpi_plane4, |coefficients| <= 1e6
 *   out       : float [n_planes][ha][wa]
 *   workspace : DEVICE, 256-byte aligned, cpi_refocus4d_workspace_size bytes
 *               (planes are processed in chunks of up to 64)
 * Requires ha, wa, hb, wb >= 1 and ha * wa, hb * wb <= 2^24.
 * -------------------------------------------------------------------------- */
typedef struct {
    double alpha, beta, gamma, delta;
} cpi_plane4;
CPI_API size_t cpi_refocus4d_workspace_size(int32_t ha, int32_t wa, int32_t hb, int32_t wb, int32_t n_planes);
CPI_API cpi_status cpi_refocus4d(const float *gamma_f32, int32_t ha, int32_t wa, int32_t hb, int32_t wb,
                                 const cpi_plane4 *planes, int32_t n_planes, float *out, void *workspace,
                                 size_t workspace_bytes, cpi_stream stream);

/* --------------------------------------------------------------------------
 * Batches of independent acquisitions of uneven sizes (many correlations and
 * their refocusings in one call).  The paper processes one acquisition at a
 * time; a batch runs every item's Eq. (1) and refocusing as above, but the
 * raw-moment units of all items of one operand kind share persistent grouped
 * tensor-core launches (up to 64 problems each, larger units first), and the
 * whole sequence can be replayed as one CUDA graph.
 *
 * Per item: a, b, n_frames and the outputs exactly as for cpi_correlate (s_ab,
 * s_a, s_b required; gamma optional; gamma_f32 optional unless refocusing);
 * n_planes > 0 also refocuses gamma_f32 into refocus_out [n_planes][ha][wa]
 * with the HOST array planes (as cpi_refocus).  Items must not share outputs.
 *
 * flags: CPI_BATCH_GRAPH captures the launches into a CUDA graph on first use
 *   and replays it on later calls whose items (shapes, pointers, planes),
 *   workspace and settings are the same (a small per-device cache; the CUDA
 *   driver may reserve memory for each instantiated graph).
 *   CPI_BATCH_TUNE chooses, on first use of a batch shape, the decomposition
 *   of the grouped raw-moment launches by timing all six candidates on the
 *   batch's operands: the frame-chunk split (1, 2 or 4 times the minimum)
 *   times the output tile width (128 x 256 or 128 x 128); this first call
 *   synchronises the stream.  Without it: split 1 and 128 x 256 tiles, or
 *   128 x 128 tiles with CPI_BATCH_N128.  When the environment variable
 *   CPI_TUNE_CACHE names a file, tuned decompositions are read from it and
 *   appended to it (one text line per batch shape and GPU model), so a later
 *   process skips the timing.
 * -------------------------------------------------------------------------- */
typedef struct cpi_batch_item {
    cpi_frames a, b;
    int64_t n_frames;
    int64_t *s_ab, *s_a, *s_b;  /* device, as cpi_correlate */
    double *gamma;              /* device, [Ma][Mb], or NULL */
    float *gamma_f32;           /* device, [Mb][Ma] slice-major; required when n_planes > 0 */
    const cpi_plane *planes;    /* HOST, n_planes entries */
    int32_t n_planes;           /* 0: no refocusing */
    float *refocus_out;         /* device, [n_planes][ha][wa] */
} cpi_batch_item;

enum { CPI_BATCH_GRAPH = 1, CPI_BATCH_TUNE = 2, CPI_BATCH_N128 = 4 };

/* Workspace bytes of a batch (0 on invalid items). */
CPI_API size_t cpi_batch_workspace_size(const cpi_batch_item *items, int32_t n_items);

CPI_API cpi_status cpi_batch_correlate(const cpi_batch_item *items, int32_t n_items, void *workspace,
                                       size_t workspace_bytes, int32_t flags, cpi_stream stream);

/* --------------------------------------------------------------------------
 * Correlation without a caller workspace.
 *
 * For callers that cannot allocate device memory: a real-time acquisition loop
 * for which cudaMalloc's implicit device synchronisation and unbounded latency
 * are not acceptable, or a host application or plugin whose own allocator owns
 * all device memory and forbids allocations by libraries.  Same inputs, outputs
 * and results as cpi_correlate; the scratch is instead a fixed array of
 * CPI_NOALLOC_SCRATCH_BYTES that the library keeps in the device memory of every
 * GPU that loads it, until the process exits.  The call allocates nothing and
 * calls no allocating routine.
 *   - Problems whose workspace (cpi_correlate_workspace_size) exceeds
 *     CPI_NOALLOC_SCRATCH_BYTES are refused with CPI_ERR_WORKSPACE.
 *   - The first call on a device looks up the array's device address (set-up,
 *     once per device, with that device current); make that first call before
 *     any stream capture.
 *   - All calls on a device share the one array and leave their data in it:
 *     calls that may overlap on the GPU (different streams, or the same stream
 *     from several host threads without ordering) race on it; serialise them.
 *     Nothing in the array needs to start at zero: each call writes every
 *     scratch byte before reading it.
 * -------------------------------------------------------------------------- */
#define CPI_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
CPI_API cpi_status cpi_correlate_noalloc(const cpi_frames *a, const cpi_frames *b, int64_t n_frames,
                                         int64_t *s_ab, int64_t *s_a, int64_t *s_b, double *gamma,
                                         float *gamma_f32, cpi_stream stream);

/* --------------------------------------------------------------------------
 * Learned denoiser of Gamma.  The paper has no counterpart: this is the
 * project's "learned denoiser" row, a small convolutional network that maps
 * Gamma of Eq. (1) measured from few frames to Gamma of many frames, trained on
 * pairs the method generates; the plain Gamma stays the fallback and the
 * reference its error is measured against.
 *
 * Network, per angular slice b = (br, bc) of Gamma (float [hb*wb][ha*wa],
 * slice-major: cpi_correlate's gamma_f32):
 *   x  = 9 channels, the slices of the 3 x 3 angular neighbourhood
 *        (br + dy, bc + dx), channel 3 (dy + 1) + (dx + 1), zero outside the
 *        angular grid; the whole Gamma scaled by s = 1 / rms(gamma_in);
 *   a1 = relu(conv(x; 9 -> 32)), a2 = relu(conv(a1; 32 -> 32)),
 *   a3 = relu(conv(a2; 32 -> 32)), y = x[4] + conv(a3; 32 -> 1)
 *   (3 x 3 kernels, zero padding 1, with biases); gamma_out = y / s.
 * x, a1..a3 and the weights in use are rounded to bfloat16; sums are float32.
 *
 * model: DEVICE float [CPI_DENOISER_PARAMS], float32 master weights, per layer
 *   l = 0..3 the weights W_l [Cout][Cin][3][3] then the biases b_l [Cout].
 * workspace: DEVICE, 256-byte aligned, cpi_denoise_workspace_size bytes
 *   (training != 0 for cpi_denoise_grad; about 3.2 GB for 64x64 vs 32x32).
 * Requires ha, wa, hb, wb >= 1 and hb * wb <= 65535; errors are reported before
 * any launch.
 *
 * cpi_denoise      : gamma_out = denoised gamma_in (same layout).
 * cpi_denoise_grad : training loss L = mean over all outputs of
 *                    (y - s * gamma_target)^2 into *loss (DEVICE float) and
 *                    dL/d(model) into grad (DEVICE float [CPI_DENOISER_PARAMS]).
 * cpi_denoise_adam : one Adam step (beta1 0.9, beta2 0.999, eps 1e-8,
 *                    bias-corrected; step counts from 1) of model with moment
 *                    buffers m, v (DEVICE float [CPI_DENOISER_PARAMS], zero
 *                    before the first step).
 * -------------------------------------------------------------------------- */
#define CPI_DENOISER_PARAMS 21409
CPI_API size_t cpi_denoise_workspace_size(int32_t ha, int32_t wa, int32_t hb, int32_t wb, int32_t training);
CPI_API cpi_status cpi_denoise(const float *model, const float *gamma_in, float *gamma_out, int32_t ha,
                               int32_t wa, int32_t hb, int32_t wb, void *workspace, size_t workspace_bytes,
                               cpi_stream stream);
CPI_API cpi_status cpi_denoise_grad(const float *model, const float *gamma_in, const float *gamma_target,
                                    int32_t ha, int32_t wa, int32_t hb, int32_t wb, float *grad, float *loss,
                                    void *workspace, size_t workspace_bytes, cpi_stream stream);
CPI_API cpi_status cpi_denoise_adam(float *model, float *m, float *v, const float *grad, int64_t step,
                                    float lr, cpi_stream stream);

/* --------------------------------------------------------------------------
 * Device status.  Kernels record failures (a wait on a pipeline barrier that
 * exceeded the time limit; the kernel then drains its own copies, frees its
 * tensor memory and returns) in a status word of the current device.
 * cpi_device_status synchronizes `stream`, reads the word and clears it when
 * clear != 0.  Returns CPI_OK, CPI_ERR_TIMEOUT or CPI_ERR_CUDA.
 * -------------------------------------------------------------------------- */
CPI_API cpi_status cpi_device_status(cpi_stream stream, int32_t clear);

/* Time limit of every device-side wait, in nanoseconds (default 2e9). */
CPI_API void cpi_set_wait_timeout_ns(int64_t ns);

/* Self-test of the failure path: launches one CTA that waits on a barrier
 * nothing arrives on, with limit timeout_ns.  The wait gives up, the kernel
 * records CPI_ERR_TIMEOUT in the status word and returns; the context stays
 * usable.  Returns the launch status. */
CPI_API cpi_status cpi_selftest_wait_timeout(int64_t timeout_ns, cpi_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* CPI_H */
