// C ABI of the library (include/cpi.h): argument validation, the execution plan
// of the correlation (operand format, tiles, frame chunks, workspace layout),
// TMA descriptors, launches and the per-device status word.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "../../include/cpi.h"
#include "kernels.cuh"

namespace cpi {

// Status word of each device that loads the library (kernels atomically OR
// error bits into it).  A file-scope __device__ variable: no allocation.
__device__ unsigned int g_device_status;

// Built-in scratch of cpi_correlate_noalloc: CPI_NOALLOC_SCRATCH_BYTES of device
// memory that every GPU loading the library holds until the process exits.
// Host code must not pass its name to a kernel (on the host it is only a
// stand-in); the device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[CPI_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
constexpr int64_t kMaxPixels = (int64_t)1 << 24;
// Exactness bound of one partial slot: the products are non-negative, so a
// chunk's sums stay below 65536 x 255 x 255 < 2^32 and are exact in uint32 (and
// every binary sum is an FP32 integer below 2^24).
constexpr int kChunkFrames = 65536;
unsigned long long g_timeout_ns = 2000000000ull;

struct DeviceInfo {
    bool ready = false;
    int sm_count = 0;
    unsigned int* status = nullptr;       // device address of g_device_status
};
DeviceInfo g_dev[kMaxDevices];
std::mutex g_dev_mu;

cudaError_t device_info(DeviceInfo** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DeviceInfo& d = g_dev[dev];
    if (!d.ready) {
        e = cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_device_status);
        if (e != cudaSuccess) return e;
        d.status = static_cast<unsigned int*>(p);
        d.ready = true;
    }
    *out = &d;
    return cudaSuccess;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 2-D K-major operand [rows][kstride_bytes], 128B swizzle.  BF16: tile box = 64
// elements (128 bytes) x box_rows.  Binary (E2M1 packed two per byte): box =
// 128 elements (64 bytes in HBM) x box_rows, each 8-byte group of 16 elements
// landing in 16 bytes of shared memory (128 bytes per box row, the layout the
// tensor cores read 4-bit operands in).
bool make_operand_map(CUtensorMap* m, void* base, bool bf16, int64_t rows, int64_t kstride_bytes,
                      int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)(bf16 ? kstride_bytes / 2 : kstride_bytes * 2), (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kstride_bytes};
    cuuint32_t box[2] = {(cuuint32_t)(bf16 ? 64 : 128), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_16U4_ALIGN16B, 2,
                     base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

static bool make_bf16_map_swz(CUtensorMap* m, const void* base, int rank, const uint64_t* dims,
                              const uint64_t* strides, const uint32_t* box, CUtensorMapSwizzle swz) {
    EncodeTiledFn enc = encode_fn();
    if (!enc || rank < 3 || rank > 4) return false;
    cuuint64_t d[4], st[3];
    cuuint32_t bx[4], es[4] = {1, 1, 1, 1};
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        bx[i] = box[i];
    }
    for (int i = 0; i < rank - 1; ++i) st[i] = strides[i];
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base), d, st, bx,
                           es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool make_bf16_map_sw128(CUtensorMap* m, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                         const uint32_t* box) {
    return make_bf16_map_swz(m, base, rank, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B);
}

bool make_bf16_map_sw64(CUtensorMap* m, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                        const uint32_t* box) {
    EncodeTiledFn enc = encode_fn();
    if (!enc || rank < 3 || rank > 4) return false;
    cuuint64_t d[4], st[3];
    cuuint32_t bx[4], es[4] = {1, 1, 1, 1};
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        bx[i] = box[i];
    }
    for (int i = 0; i < rank - 1; ++i) st[i] = strides[i];
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base), d, st, bx,
                           es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool make_f32_map(CUtensorMap* m, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                  const uint32_t* box) {
    EncodeTiledFn enc = encode_fn();
    if (!enc || rank < 1 || rank > 3) return false;
    cuuint64_t d[3], st[2];
    cuuint32_t bx[3], es[3] = {1, 1, 1};
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        bx[i] = box[i];
    }
    for (int i = 0; i < rank - 1; ++i) st[i] = strides[i];
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void*>(base), d, st, bx,
                           es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

namespace {

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

cpi_status check_frames(const cpi_frames* f) {
    if (!f || !f->data) return CPI_ERR_INVALID_ARG;
    if (f->bits != 1 && f->bits != 8) return CPI_ERR_INVALID_ARG;
    if (f->height < 1 || f->width < 1 || f->x0 < 0 || f->y0 < 0) return CPI_ERR_INVALID_ARG;
    if (f->bit_order != 0 && f->bit_order != 1) return CPI_ERR_INVALID_ARG;
    if (f->bits == 8 && f->bit_order != 0) return CPI_ERR_INVALID_ARG;
    if (f->row_stride < (int64_t)f->x0 + f->width || f->frame_stride_bytes <= 0)
        return CPI_ERR_INVALID_ARG;
    if ((int64_t)f->height * f->width > kMaxPixels) return CPI_ERR_INVALID_ARG;
    // the region must lie inside one frame
    const int64_t last = ((int64_t)f->y0 + f->height - 1) * f->row_stride + f->x0 + f->width - 1;
    const int64_t last_byte = f->bits == 8 ? last : last / 8;
    if (last_byte >= f->frame_stride_bytes) return CPI_ERR_INVALID_ARG;
    return CPI_OK;
}

FramesDev to_dev(const cpi_frames* f) {
    FramesDev d;
    d.data = static_cast<const uint8_t*>(f->data);
    d.bits = f->bits;
    d.height = f->height;
    d.width = f->width;
    d.x0 = f->x0;
    d.y0 = f->y0;
    d.row_stride = f->row_stride;
    d.frame_stride = f->frame_stride_bytes;
    d.bit_order = f->bit_order;
    return d;
}

// Execution plan of one correlation.
struct CorrPlan {
    bool bf16;                 // BF16 operands (any 8-bit input) or FP8 (both binary)
    int64_t Ma, Mb, n;
    int64_t kstride_bytes;     // operand row length in bytes (frames padded to the ingest tile;
                               // 2 bytes per frame BF16, half a byte E2M1)
    int k_blocks, kb_per_chunk, n_chunks;
    int block_n, tiles_m, tiles_n, n_units;
    size_t off_a, off_b, off_part, off_vmax, off_sa, off_sb, ws_bytes;   // off_sa/off_sb: S_a, S_b when the caller passes none
};

// split == 0: single correlation (more frame chunks when the tiles alone cannot
// fill the GPU); split >= 1: member of a batch, split x the minimum chunk count.
// block_n: output tile width (256; batches may choose 128).
cpi_status make_plan(const cpi_frames* a, const cpi_frames* b, int64_t n, int sm_count,
                     CorrPlan* pl, int split = 0, int block_n = 256) {
    cpi_status s = check_frames(a);
    if (s != CPI_OK) return s;
    s = check_frames(b);
    if (s != CPI_OK) return s;
    if (n < 1 || n > ((int64_t)1 << 31) - 1) return CPI_ERR_INVALID_ARG;
    const double va = a->bits == 1 ? 1.0 : 255.0, vb = b->bits == 1 ? 1.0 : 255.0;
    if ((double)n * (double)n * va * vb >= 9.2e18) return CPI_ERR_OVERFLOW;
    CorrPlan p{};
    p.bf16 = !(a->bits == 1 && b->bits == 1);
    p.Ma = (int64_t)a->height * a->width;
    p.Mb = (int64_t)b->height * b->width;
    p.n = n;
    const int fpc = ingest_frames_per_cta(p.bf16);
    const int64_t kpad = (int64_t)round_up((size_t)n, (size_t)fpc);
    p.kstride_bytes = p.bf16 ? kpad * 2 : kpad / 2;   // BF16, or E2M1 two frames per byte
    if (block_n != 128 && block_n != 256) return CPI_ERR_INVALID_ARG;
    const MomentsShape sh = moments_shape(p.bf16, block_n);
    p.k_blocks = (int)(kpad / sh.k_per_block);
    p.block_n = sh.block_n;
    p.tiles_m = (int)((p.Ma + 127) / 128);
    p.tiles_n = (int)((p.Mb + p.block_n - 1) / p.block_n);
    const int max_kb_chunk = kChunkFrames / sh.k_per_block;
    const int64_t tiles = (int64_t)p.tiles_m * p.tiles_n;
    int n_chunks = (p.k_blocks + max_kb_chunk - 1) / max_kb_chunk;
    if (split >= 1) {
        const int max_by_len = p.k_blocks / 8 > 0 ? p.k_blocks / 8 : 1;
        n_chunks = n_chunks * split < max_by_len ? n_chunks * split : (max_by_len > n_chunks ? max_by_len : n_chunks);
    } else if (tiles < sm_count) {
        // small outputs: split the frames further so every SM gets work, but keep
        // each chunk at least 8 K blocks long
        int want = (int)(sm_count / tiles);
        int max_by_len = p.k_blocks / 8;
        if (max_by_len < 1) max_by_len = 1;
        if (want > max_by_len) want = max_by_len;
        if (want > n_chunks) n_chunks = want;
    }
    p.kb_per_chunk = (p.k_blocks + n_chunks - 1) / n_chunks;
    if (p.kb_per_chunk > max_kb_chunk) p.kb_per_chunk = max_kb_chunk;
    p.n_chunks = (p.k_blocks + p.kb_per_chunk - 1) / p.kb_per_chunk;
    const int64_t units = tiles * p.n_chunks;
    if (units > 0x7fffffff) return CPI_ERR_UNSUPPORTED;
    p.n_units = (int)units;
    p.off_a = 0;
    p.off_b = round_up(p.off_a + (size_t)p.Ma * (size_t)p.kstride_bytes, 1024);
    p.off_part = round_up(p.off_b + (size_t)p.Mb * (size_t)p.kstride_bytes, 1024);
    p.off_vmax = round_up(p.off_part + (size_t)p.n_chunks * (size_t)p.Ma * (size_t)p.Mb * 4, 256);
    p.off_sa = round_up(p.off_vmax + 2 * sizeof(uint32_t), 256);
    p.off_sb = round_up(p.off_sa + (size_t)p.Ma * 8, 256);
    p.ws_bytes = round_up(p.off_sb + (size_t)p.Mb * 8, 1024);
    *pl = p;
    return CPI_OK;
}

cpi_status cuda_status(cudaError_t e) { return e == cudaSuccess ? CPI_OK : CPI_ERR_CUDA; }


// vmax: the ingest's value maxima (BF16 path), which set the exact FP32
// segment length on the device.
void fill_problem(const CorrPlan& pl, int32_t* part, int unit_begin, MomentsProblem* P, const uint32_t* vmax) {
    P->partial = part;
    P->M = (int32_t)pl.Ma;
    P->N = (int32_t)pl.Mb;
    P->k_blocks = pl.k_blocks;
    P->kb_per_chunk = pl.kb_per_chunk;
    P->n_chunks = pl.n_chunks;
    P->tiles_m = pl.tiles_m;
    P->tiles_n = pl.tiles_n;
    P->unit_begin = unit_begin;
    P->vmax = pl.bf16 ? vmax : nullptr;
    P->add_partial = 0;
}

cpi_status run_stage(int stage, const CorrPlan& pl, const cpi_frames* a, const cpi_frames* b,
                     int accumulate, int64_t* s_ab, int64_t* s_a, int64_t* s_b, double* gamma,
                     float* gamma_f32, void* ws, DeviceInfo* dev, cudaStream_t st, int add_partial = 0) {
    uint8_t* w = static_cast<uint8_t*>(ws);
    uint8_t* op_a = w + pl.off_a;
    uint8_t* op_b = w + pl.off_b;
    int32_t* part = reinterpret_cast<int32_t*>(w + pl.off_part);
    uint32_t* vmax = reinterpret_cast<uint32_t*>(w + pl.off_vmax);
    if (s_a == nullptr) s_a = reinterpret_cast<int64_t*>(w + pl.off_sa);
    if (s_b == nullptr) s_b = reinterpret_cast<int64_t*>(w + pl.off_sb);
    if (stage == CPI_STAGE_INGEST) {
        if (!accumulate) {
            cudaError_t e = cudaMemsetAsync(s_a, 0, (size_t)pl.Ma * 8, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(s_b, 0, (size_t)pl.Mb * 8, st);
            if (e != cudaSuccess) return CPI_ERR_CUDA;
        }
        if (pl.bf16 && cudaMemsetAsync(vmax, 0, 2 * sizeof(uint32_t), st) != cudaSuccess) return CPI_ERR_CUDA;
        return cuda_status(launch_ingest(pl.bf16, to_dev(a), to_dev(b), pl.n, pl.kstride_bytes,
                                         op_a, op_b, s_a, s_b, pl.bf16 ? vmax : nullptr, st));
    }
    if (stage == CPI_STAGE_MOMENTS) {
        CUtensorMap tm_a, tm_b;
        if (!make_operand_map(&tm_a, op_a, pl.bf16, pl.Ma, pl.kstride_bytes, 128) ||
            !make_operand_map(&tm_b, op_b, pl.bf16, pl.Mb, pl.kstride_bytes, pl.block_n))
            return CPI_ERR_CUDA;
        MomentsLaunch<1> L;
        std::memset(&L, 0, sizeof(L));
        L.map_a[0] = tm_a;
        L.map_b[0] = tm_b;
        fill_problem(pl, part, 0, &L.prob[0], vmax);
        L.prob[0].add_partial = add_partial;
        L.n_problems = 1;
        L.n_units = pl.n_units;
        L.status = dev->status;
        L.timeout_ns = g_timeout_ns;
        return cuda_status(launch_moments(pl.bf16, pl.block_n, L, dev->sm_count, st));
    }
    if (stage == CPI_STAGE_FOLD) {
        return cuda_status(launch_fold(part, pl.n_chunks, pl.Ma, pl.Mb, s_ab, accumulate, s_ab != nullptr ? 1 : 0,
                                       s_a, s_b, pl.n, gamma, gamma_f32, st));
    }
    return CPI_ERR_INVALID_ARG;
}

cpi_status correlate_common(const int32_t* stages, int n_stages, const cpi_frames* a,
                            const cpi_frames* b, int64_t n_frames, int accumulate, int64_t* s_ab,
                            int64_t* s_a, int64_t* s_b, double* gamma, float* gamma_f32, void* ws,
                            size_t ws_bytes, cpi_stream stream, int add_partial = 0) {
    DeviceInfo* dev = nullptr;
    if (device_info(&dev) != cudaSuccess) return CPI_ERR_CUDA;
    CorrPlan pl;
    cpi_status s = make_plan(a, b, n_frames, dev->sm_count, &pl);
    if (s != CPI_OK) return s;
    // accumulating calls need the caller's sums; otherwise S_a, S_b may live in
    // the workspace and S_ab may be skipped when a Gamma output is asked for
    if (accumulate && (!s_ab || !s_a || !s_b)) return CPI_ERR_INVALID_ARG;
    // an accumulating call has no total frame count: Gamma comes from
    // cpi_correlate_finalize once every block has been added
    if (accumulate && (gamma || gamma_f32)) return CPI_ERR_INVALID_ARG;
    if (!s_ab && !gamma && !gamma_f32) return CPI_ERR_INVALID_ARG;
    if ((s_ab && !aligned(s_ab, 16)) || (s_a && !aligned(s_a, 16)) || (s_b && !aligned(s_b, 16)))
        return CPI_ERR_INVALID_ARG;
    if ((gamma && !aligned(gamma, 16)) || (gamma_f32 && !aligned(gamma_f32, 16)))
        return CPI_ERR_INVALID_ARG;
    if (!ws || ws_bytes < pl.ws_bytes || !aligned(ws, 256)) return CPI_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (int i = 0; i < n_stages; ++i) {
        s = run_stage(stages[i], pl, a, b, accumulate, s_ab, s_a, s_b, gamma, gamma_f32, ws, dev,
                      st, add_partial);
        if (s != CPI_OK) return s;
    }
    return CPI_OK;
}

size_t refocus_ws_size(int32_t ha, int32_t wa, int32_t hb, int32_t wb, int32_t n_planes) {
    if (ha < 1 || wa < 1 || hb < 1 || wb < 1 || n_planes < 1) return 0;
    return refocus_ws_bytes(ha, wa, hb, wb, n_planes);
}

cpi_status run_refocus(const float* gamma_f32, int32_t ha, int32_t wa, int32_t hb, int32_t wb,
                       const cpi_plane* planes, int32_t n_planes, float* out, void* workspace,
                       size_t workspace_bytes, cudaStream_t st) {
    if (!gamma_f32 || !planes || !out || n_planes < 1) return CPI_ERR_INVALID_ARG;
    if (ha < 1 || wa < 1 || hb < 1 || wb < 1 || wa > 512) return CPI_ERR_INVALID_ARG;
    if ((int64_t)hb * wb > kMaxPixels) return CPI_ERR_INVALID_ARG;
    if (!refocus_supported(ha, wa, hb, wb)) return CPI_ERR_UNSUPPORTED;
    if (!aligned(gamma_f32, 16) || !aligned(out, 4)) return CPI_ERR_INVALID_ARG;
    std::vector<double> alpha(n_planes), beta(n_planes);
    for (int i = 0; i < n_planes; ++i) {
        if (!(std::fabs(planes[i].alpha) <= kRefocusMaxCoef) || !(std::fabs(planes[i].beta) <= kRefocusMaxCoef))
            return CPI_ERR_INVALID_ARG;
        alpha[i] = planes[i].alpha;
        beta[i] = planes[i].beta;
    }
    DeviceInfo* dev = nullptr;
    if (device_info(&dev) != cudaSuccess) return CPI_ERR_CUDA;
    const size_t need = refocus_ws_size(ha, wa, hb, wb, n_planes);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256)) return CPI_ERR_WORKSPACE;
    return cuda_status(refocus_run(gamma_f32, ha, wa, hb, wb, alpha.data(), beta.data(), n_planes, out, workspace,
                                   dev->sm_count, dev->status, g_timeout_ns, st));
}


// ------------------------------------------------------------------ batches
// A batch of independent correlations (and refocusings): every item gets its
// own region of the workspace; the items' ingest, fold and refocus kernels are
// launched per item on forked streams, and the raw-moment units of all items of
// one operand kind run in persistent grouped launches of up to kMaxGroup
// problems, larger units first.  The whole sequence can be captured once into a
// CUDA graph and replayed.
struct BatchItemPlan {
    CorrPlan pl;
    size_t ws_off = 0, rws_off = 0, rws_bytes = 0;
};
struct BatchPlan {
    std::vector<BatchItemPlan> it;
    int block_n = 256;          // output tile width of every grouped launch
    size_t ws_bytes = 0;
};

// Decompositions the batch tuner times: frame-chunk split x output tile width.
struct BatchShape {
    int split, block_n;
};
constexpr BatchShape kBatchCandidates[6] = {{1, 256}, {2, 256}, {4, 256}, {1, 128}, {2, 128}, {4, 128}};

cpi_status check_batch_item(const cpi_batch_item& b) {
    if (!b.s_ab || !b.s_a || !b.s_b || !aligned(b.s_ab, 16) || !aligned(b.s_a, 16) || !aligned(b.s_b, 16))
        return CPI_ERR_INVALID_ARG;
    if ((b.gamma && !aligned(b.gamma, 16)) || (b.gamma_f32 && !aligned(b.gamma_f32, 16)))
        return CPI_ERR_INVALID_ARG;
    if (b.n_planes < 0) return CPI_ERR_INVALID_ARG;
    if (b.n_planes > 0) {
        if (!b.planes || !b.refocus_out || !b.gamma_f32) return CPI_ERR_INVALID_ARG;
        if (b.a.width > 512) return CPI_ERR_INVALID_ARG;
        if (!refocus_supported(b.a.height, b.a.width, b.b.height, b.b.width)) return CPI_ERR_UNSUPPORTED;
        for (int i = 0; i < b.n_planes; ++i)
            if (!(std::fabs(b.planes[i].alpha) <= kRefocusMaxCoef) || !(std::fabs(b.planes[i].beta) <= kRefocusMaxCoef))
                return CPI_ERR_INVALID_ARG;
    }
    return CPI_OK;
}

cpi_status make_batch_plan(const cpi_batch_item* items, int n, int sm, BatchShape shape, BatchPlan* bp) {
    if (!items || n < 1) return CPI_ERR_INVALID_ARG;
    bp->it.assign(n, BatchItemPlan{});
    bp->block_n = shape.block_n;
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        const cpi_batch_item& b = items[i];
        cpi_status s = check_batch_item(b);
        if (s != CPI_OK) return s;
        BatchItemPlan& ip = bp->it[i];
        s = make_plan(&b.a, &b.b, b.n_frames, sm, &ip.pl, shape.split, shape.block_n);
        if (s != CPI_OK) return s;
        ip.ws_off = off;
        off = round_up(off + ip.pl.ws_bytes, 1024);
        if (b.n_planes > 0) {
            ip.rws_bytes = refocus_ws_size(b.a.height, b.a.width, b.b.height, b.b.width, b.n_planes);
            ip.rws_off = off;
            off = round_up(off + ip.rws_bytes, 1024);
        }
    }
    bp->ws_bytes = off;
    return CPI_OK;
}

// Grouped raw-moment launches of the batch: one operand kind at a time, items
// ordered by decreasing units (K blocks per unit, then unit count).
cpi_status launch_batch_moments(const cpi_batch_item* items, const BatchPlan& bp, uint8_t* ws,
                                DeviceInfo* dev, cudaStream_t st) {
    std::unique_ptr<MomentsLaunch<kMaxGroup>> L(new MomentsLaunch<kMaxGroup>);
    for (int kind = 0; kind < 2; ++kind) {
        const bool bf16 = kind == 1;
        std::vector<int> idx;
        for (int i = 0; i < (int)bp.it.size(); ++i)
            if (bp.it[i].pl.bf16 == bf16) idx.push_back(i);
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
            const CorrPlan &p = bp.it[x].pl, &q = bp.it[y].pl;
            if (p.kb_per_chunk != q.kb_per_chunk) return p.kb_per_chunk > q.kb_per_chunk;
            return p.n_units > q.n_units;
        });
        for (size_t g0 = 0; g0 < idx.size(); g0 += kMaxGroup) {
            std::memset(L.get(), 0, sizeof(*L));
            int64_t units = 0;
            int np = 0;
            for (size_t g = g0; g < idx.size() && g < g0 + kMaxGroup; ++g, ++np) {
                const BatchItemPlan& ip = bp.it[idx[g]];
                uint8_t* w = ws + ip.ws_off;
                if (!make_operand_map(&L->map_a[np], w + ip.pl.off_a, ip.pl.bf16, ip.pl.Ma,
                                      ip.pl.kstride_bytes, 128) ||
                    !make_operand_map(&L->map_b[np], w + ip.pl.off_b, ip.pl.bf16, ip.pl.Mb,
                                      ip.pl.kstride_bytes, ip.pl.block_n))
                    return CPI_ERR_CUDA;
                fill_problem(ip.pl, reinterpret_cast<int32_t*>(w + ip.pl.off_part), (int)units, &L->prob[np],
                             reinterpret_cast<const uint32_t*>(w + ip.pl.off_vmax));
                units += ip.pl.n_units;
                if (units > 0x7fffffff) return CPI_ERR_UNSUPPORTED;
            }
            L->n_problems = np;
            L->n_units = (int)units;
            L->status = dev->status;
            L->timeout_ns = g_timeout_ns;
            if (launch_moments_group(bf16, bp.block_n, *L, dev->sm_count, st) != cudaSuccess) return CPI_ERR_CUDA;
        }
    }
    (void)items;
    return CPI_OK;
}

// Independent per-item work of a batch is spread over kForks side streams
// (parallel branches when captured into a graph), longest first, each item to
// the branch with the least work so far, so that small launches overlap and one
// item's tail overlaps the others' work.  Every branch joins the caller's stream
// before the call returns.
constexpr int kForks = 4;
struct ForkStreams {
    std::mutex mu;
    bool ready[kMaxDevices] = {};
    cudaStream_t side[kMaxDevices][kForks] = {};
    cudaEvent_t fork[kMaxDevices] = {};
    cudaEvent_t join[kMaxDevices][kForks] = {};
};
ForkStreams g_forks;

template <class Cost, class One>
cpi_status run_forked(std::vector<int> idx, Cost cost, One one, cudaStream_t st) {
    if (idx.size() < 2) return idx.empty() ? CPI_OK : one(idx[0], st);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CPI_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_forks.mu);
    if (!g_forks.ready[dev]) {
        if (cudaEventCreateWithFlags(&g_forks.fork[dev], cudaEventDisableTiming) != cudaSuccess) return CPI_ERR_CUDA;
        for (int k = 0; k < kForks; ++k)
            if (cudaStreamCreateWithFlags(&g_forks.side[dev][k], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&g_forks.join[dev][k], cudaEventDisableTiming) != cudaSuccess)
                return CPI_ERR_CUDA;
        g_forks.ready[dev] = true;
    }
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return cost(x) > cost(y); });
    if (cudaEventRecord(g_forks.fork[dev], st) != cudaSuccess) return CPI_ERR_CUDA;
    for (int k = 0; k < kForks; ++k)
        if (cudaStreamWaitEvent(g_forks.side[dev][k], g_forks.fork[dev], 0) != cudaSuccess) return CPI_ERR_CUDA;
    double load[kForks] = {};
    cpi_status result = CPI_OK;
    for (int i : idx) {
        int k = 0;
        for (int q = 1; q < kForks; ++q)
            if (load[q] < load[k]) k = q;
        load[k] += cost(i);
        result = one(i, g_forks.side[dev][k]);
        if (result != CPI_OK) break;
    }
    // join every branch, also after an error (a capture must not end with a branch open)
    for (int k = 0; k < kForks; ++k)
        if (cudaEventRecord(g_forks.join[dev][k], g_forks.side[dev][k]) != cudaSuccess ||
            cudaStreamWaitEvent(st, g_forks.join[dev][k], 0) != cudaSuccess)
            result = CPI_ERR_CUDA;
    return result;
}

cpi_status run_batch(const cpi_batch_item* items, const BatchPlan& bp, uint8_t* ws, DeviceInfo* dev,
                     cudaStream_t st) {
    const int n = (int)bp.it.size();
    std::vector<int> all(n);
    for (int i = 0; i < n; ++i) all[i] = i;
    // ingest of every item (forked), the grouped raw-moment launches, then per
    // item its fold and refocusing (forked)
    cpi_status s = run_forked(
        all, [&](int i) { return (double)(bp.it[i].pl.Ma + bp.it[i].pl.Mb) * (double)bp.it[i].pl.n; },
        [&](int i, cudaStream_t cs) {
            const cpi_batch_item& b = items[i];
            return run_stage(CPI_STAGE_INGEST, bp.it[i].pl, &b.a, &b.b, 0, b.s_ab, b.s_a, b.s_b, b.gamma,
                             b.gamma_f32, ws + bp.it[i].ws_off, dev, cs);
        },
        st);
    if (s != CPI_OK) return s;
    s = launch_batch_moments(items, bp, ws, dev, st);
    if (s != CPI_OK) return s;
    return run_forked(
        all,
        [&](int i) {
            const cpi_batch_item& b = items[i];
            return (double)bp.it[i].pl.Ma * (double)bp.it[i].pl.Mb * (6.0 + (double)b.n_planes);
        },
        [&](int i, cudaStream_t cs) {
            const cpi_batch_item& b = items[i];
            cpi_status r = run_stage(CPI_STAGE_FOLD, bp.it[i].pl, &b.a, &b.b, 0, b.s_ab, b.s_a, b.s_b, b.gamma,
                                     b.gamma_f32, ws + bp.it[i].ws_off, dev, cs);
            if (r != CPI_OK || b.n_planes == 0) return r;
            return run_refocus(b.gamma_f32, b.a.height, b.a.width, b.b.height, b.b.width, b.planes, b.n_planes,
                               b.refocus_out, ws + bp.it[i].rws_off, bp.it[i].rws_bytes, cs);
        },
        st);
}

uint64_t fnv(uint64_t h, const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

// Shape of a batch (what the tuned decomposition depends on).
uint64_t batch_shape_key(const cpi_batch_item* items, int n, int dev) {
    uint64_t h = fnv(1469598103934665603ull, &n, sizeof(n));
    h = fnv(h, &dev, sizeof(dev));
    for (int i = 0; i < n; ++i) {
        const cpi_batch_item& b = items[i];
        const int64_t f[] = {b.a.bits, b.a.height, b.a.width, b.b.bits, b.b.height, b.b.width, b.n_frames,
                             b.n_planes};
        h = fnv(h, f, sizeof(f));
    }
    return h;
}

// Everything a captured graph bakes in: shapes, pointers, plane coefficients,
// workspace and the chosen decomposition.
uint64_t batch_graph_key(const cpi_batch_item* items, int n, const void* ws, BatchShape shape, int dev) {
    uint64_t h = fnv(1469598103934665603ull, &n, sizeof(n));
    h = fnv(h, &ws, sizeof(ws));
    h = fnv(h, &shape.split, sizeof(shape.split));
    h = fnv(h, &shape.block_n, sizeof(shape.block_n));
    h = fnv(h, &dev, sizeof(dev));
    h = fnv(h, &g_timeout_ns, sizeof(g_timeout_ns));
    for (int i = 0; i < n; ++i) {
        h = fnv(h, &items[i], sizeof(cpi_batch_item));
        if (items[i].n_planes > 0) h = fnv(h, items[i].planes, sizeof(cpi_plane) * items[i].n_planes);
    }
    return h;
}

struct BatchCache {
    std::mutex mu;
    std::unordered_map<uint64_t, BatchShape> tuned;       // shape key -> tuned decomposition
    std::vector<std::pair<uint64_t, cudaGraphExec_t>> graphs[kMaxDevices];
    cudaStream_t capture_stream[kMaxDevices] = {};
};
BatchCache g_batch;
constexpr size_t kMaxGraphs = 16;

// Persistent tuner cache: when the environment variable CPI_TUNE_CACHE names a
// file, tuned decompositions are looked up there and appended to it, one line
// per (batch shape, GPU model): "<key in hex> <split> <tile width>".  The key
// hashes the items' shapes with the GPU's name, SM count and compute
// capability, so a cache file can be shared by processes and boxes.
uint64_t tune_file_key(const cpi_batch_item* items, int n, int dev) {
    uint64_t h = batch_shape_key(items, n, 0);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
        h = fnv(h, prop.name, strnlen(prop.name, sizeof(prop.name)));
        h = fnv(h, &prop.multiProcessorCount, sizeof(prop.multiProcessorCount));
        h = fnv(h, &prop.major, sizeof(prop.major));
        h = fnv(h, &prop.minor, sizeof(prop.minor));
    }
    return h;
}

bool tune_file_lookup(uint64_t key, BatchShape* out) {
    const char* path = std::getenv("CPI_TUNE_CACHE");
    if (!path || !*path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    unsigned long long k = 0;
    int split = 0, bn = 0;
    bool found = false;
    while (std::fscanf(f, "%llx %d %d", &k, &split, &bn) == 3) {
        if (k == key) {
            for (const BatchShape& c : kBatchCandidates)
                if (c.split == split && c.block_n == bn) {
                    *out = c;
                    found = true;
                }
        }
    }
    std::fclose(f);
    return found;
}

void tune_file_store(uint64_t key, BatchShape s) {
    const char* path = std::getenv("CPI_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%016llx %d %d\n", (unsigned long long)key, s.split, s.block_n);
    std::fclose(f);
}

// Decomposition of the grouped raw-moment launches (frame-chunk split x output
// tile width), tuned on first use of a batch shape by timing every candidate on
// the batch's own operands (or read from the CPI_TUNE_CACHE file).
cpi_status tuned_shape(const cpi_batch_item* items, int n, uint8_t* ws, DeviceInfo* dev, int dev_id,
                       cudaStream_t st, BatchShape* shape_out) {
    const uint64_t key = batch_shape_key(items, n, dev_id);
    {
        std::lock_guard<std::mutex> lk(g_batch.mu);
        auto it = g_batch.tuned.find(key);
        if (it != g_batch.tuned.end()) {
            *shape_out = it->second;
            return CPI_OK;
        }
        BatchShape cached;
        if (tune_file_lookup(tune_file_key(items, n, dev_id), &cached)) {
            g_batch.tuned[key] = cached;
            *shape_out = cached;
            return CPI_OK;
        }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return CPI_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return CPI_ERR_CUDA;
    }
    float best = 1e30f;
    BatchShape best_shape = kBatchCandidates[0];
    cpi_status s = CPI_OK;
    for (int c = 0; c < 6 && s == CPI_OK; ++c) {
        BatchPlan bp;
        s = make_batch_plan(items, n, dev->sm_count, kBatchCandidates[c], &bp);
        if (s != CPI_OK) break;
        // real operands and value maxima in this candidate's layout, so that the
        // timed launches run the GEMM variant the batch will run
        for (int i = 0; i < n && s == CPI_OK; ++i)
            s = run_stage(CPI_STAGE_INGEST, bp.it[i].pl, &items[i].a, &items[i].b, 0, items[i].s_ab,
                          items[i].s_a, items[i].s_b, items[i].gamma, items[i].gamma_f32,
                          ws + bp.it[i].ws_off, dev, st);
        if (s != CPI_OK) break;
        s = launch_batch_moments(items, bp, ws, dev, st);                 // warm-up
        if (s != CPI_OK) break;
        if (cudaEventRecord(e0, st) != cudaSuccess) { s = CPI_ERR_CUDA; break; }
        for (int r = 0; r < 2 && s == CPI_OK; ++r) s = launch_batch_moments(items, bp, ws, dev, st);
        if (s != CPI_OK) break;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            s = CPI_ERR_CUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_shape = kBatchCandidates[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != CPI_OK) return s;
    std::lock_guard<std::mutex> lk(g_batch.mu);
    g_batch.tuned[key] = best_shape;
    tune_file_store(tune_file_key(items, n, dev_id), best_shape);
    *shape_out = best_shape;
    return CPI_OK;
}

// ------------------------------------------------------------------ streamed acquisitions
// A correlation fed block by block from host memory while it is acquired (the
// paper processes its acquisitions in blocks of files; a SPAD camera delivers
// ~10^5 frames per second).  Two staging buffers in the caller's workspace: the
// copy of block k runs on the acquisition's own copy stream while block k - 1 is
// accumulated on the caller's stream; the running sums are the whole state.
struct Acquisition {
    int dev = 0;
    cpi_frames a{}, b{};              // layout of the two regions inside one frame
    int64_t block_frames = 0, frame_bytes = 0;
    int64_t *s_ab = nullptr, *s_a = nullptr, *s_b = nullptr;
    uint8_t* staging[2] = {nullptr, nullptr};
    uint8_t* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t compute = nullptr;   // the caller's stream
    cudaStream_t copy = nullptr;      // created by cpi_acq_begin
    cudaEvent_t arrived[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
    bool copied_once[2] = {false, false};
    int next = 0;
    int64_t n_done = 0;
    // Binary frames: full blocks add their raw moments into the workspace's
    // uint32 partial slots (every entry counts at most the 2^31 frames of an
    // acquisition) and the fold into the int64 S_ab waits for a checkpoint
    // (sync, finalize, end) or a block of another size.
    bool defer = false;
    int64_t deferred = 0;             // full blocks whose moments are still in the partial slots
    size_t off_part = 0;              // partial slots of a full block's workspace layout
    int n_chunks = 0;
};

// Fold the deferred partial sums into S_ab on the compute stream.
cpi_status acq_flush(Acquisition* q) {
    if (q->deferred == 0) return CPI_OK;
    const int64_t ma = (int64_t)q->a.height * q->a.width, mb = (int64_t)q->b.height * q->b.width;
    const int32_t* part = reinterpret_cast<const int32_t*>(q->ws + q->off_part);
    const cudaError_t e = launch_fold(part, q->n_chunks, ma, mb, q->s_ab, 1, 1, q->s_a, q->s_b, q->n_done, nullptr,
                                      nullptr, q->compute, 0);
    if (e != cudaSuccess) return CPI_ERR_CUDA;
    q->deferred = 0;
    return CPI_OK;
}

size_t acq_staging_bytes(const cpi_frames* a, int64_t block_frames) {
    return round_up((size_t)block_frames * (size_t)a->frame_stride_bytes, 256);
}

cpi_status acq_check_layout(const cpi_frames* a, const cpi_frames* b, int64_t block_frames) {
    if (!a || !b || block_frames < 1) return CPI_ERR_INVALID_ARG;
    if (a->frame_stride_bytes != b->frame_stride_bytes) return CPI_ERR_INVALID_ARG;
    // validate with a placeholder data pointer (the regions' data come from the staging buffers)
    cpi_frames ta = *a, tb = *b;
    ta.data = tb.data = reinterpret_cast<const void*>(uintptr_t(256));
    if (check_frames(&ta) != CPI_OK || check_frames(&tb) != CPI_OK) return CPI_ERR_INVALID_ARG;
    return CPI_OK;
}

}  // namespace
}  // namespace cpi

using namespace cpi;

extern "C" {

const char* cpi_status_string(cpi_status s) {
    switch (s) {
        case CPI_OK: return "CPI_OK";
        case CPI_ERR_INVALID_ARG: return "CPI_ERR_INVALID_ARG";
        case CPI_ERR_OVERFLOW: return "CPI_ERR_OVERFLOW";
        case CPI_ERR_WORKSPACE: return "CPI_ERR_WORKSPACE";
        case CPI_ERR_UNSUPPORTED: return "CPI_ERR_UNSUPPORTED";
        case CPI_ERR_CUDA: return "CPI_ERR_CUDA";
        case CPI_ERR_TIMEOUT: return "CPI_ERR_TIMEOUT";
    }
    return "CPI_ERR_UNKNOWN";
}

int32_t cpi_abi_version(void) { return 1; }

size_t cpi_correlate_workspace_size(const cpi_frames* a, const cpi_frames* b, int64_t n_frames) {
    DeviceInfo* dev = nullptr;
    int sm = 152;
    if (device_info(&dev) == cudaSuccess) sm = dev->sm_count;
    CorrPlan pl;
    if (make_plan(a, b, n_frames, sm, &pl) != CPI_OK) return 0;
    return pl.ws_bytes;
}

cpi_status cpi_correlate(const cpi_frames* a, const cpi_frames* b, int64_t n_frames,
                         int64_t* s_ab, int64_t* s_a, int64_t* s_b, double* gamma,
                         float* gamma_f32, void* workspace, size_t workspace_bytes,
                         cpi_stream stream) {
    static const int32_t stages[3] = {CPI_STAGE_INGEST, CPI_STAGE_MOMENTS, CPI_STAGE_FOLD};
    return correlate_common(stages, 3, a, b, n_frames, 0, s_ab, s_a, s_b, gamma, gamma_f32,
                            workspace, workspace_bytes, stream);
}

cpi_status cpi_correlate_accumulate(const cpi_frames* a, const cpi_frames* b, int64_t n_frames,
                                    int64_t* s_ab, int64_t* s_a, int64_t* s_b, void* workspace,
                                    size_t workspace_bytes, cpi_stream stream) {
    static const int32_t stages[3] = {CPI_STAGE_INGEST, CPI_STAGE_MOMENTS, CPI_STAGE_FOLD};
    return correlate_common(stages, 3, a, b, n_frames, 1, s_ab, s_a, s_b, nullptr, nullptr,
                            workspace, workspace_bytes, stream);
}

cpi_status cpi_correlate_stage(int32_t stage, const cpi_frames* a, const cpi_frames* b,
                               int64_t n_frames, int32_t accumulate, int64_t* s_ab, int64_t* s_a,
                               int64_t* s_b, double* gamma, float* gamma_f32, void* workspace,
                               size_t workspace_bytes, cpi_stream stream) {
    if (stage < CPI_STAGE_INGEST || stage > CPI_STAGE_FOLD) return CPI_ERR_INVALID_ARG;
    return correlate_common(&stage, 1, a, b, n_frames, accumulate ? 1 : 0, s_ab, s_a, s_b, gamma,
                            gamma_f32, workspace, workspace_bytes, stream);
}

cpi_status cpi_correlate_finalize(const int64_t* s_ab, const int64_t* s_a, const int64_t* s_b,
                                  int64_t m_a, int64_t m_b, int64_t n_total, double* gamma,
                                  float* gamma_f32, cpi_stream stream) {
    if (!s_ab || !s_a || !s_b || (!gamma && !gamma_f32)) return CPI_ERR_INVALID_ARG;
    if (m_a < 1 || m_b < 1 || m_a > kMaxPixels || m_b > kMaxPixels || n_total < 1)
        return CPI_ERR_INVALID_ARG;
    if (!aligned(s_ab, 8) || !aligned(s_a, 8) || !aligned(s_b, 8)) return CPI_ERR_INVALID_ARG;
    if ((gamma && !aligned(gamma, 8)) || (gamma_f32 && !aligned(gamma_f32, 4)))
        return CPI_ERR_INVALID_ARG;
    if (n_total > ((int64_t)1 << 31) - 1) return CPI_ERR_OVERFLOW;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    return cuda_status(launch_fold(nullptr, 0, m_a, m_b, const_cast<int64_t*>(s_ab), 1, 0, s_a, s_b,
                                   n_total, gamma, gamma_f32, st, 1));
}

size_t cpi_refocus_workspace_size(int32_t ha, int32_t wa, int32_t hb, int32_t wb,
                                  int32_t n_planes) {
    return refocus_ws_size(ha, wa, hb, wb, n_planes);
}

cpi_status cpi_refocus(const float* gamma_f32, int32_t ha, int32_t wa, int32_t hb, int32_t wb,
                       const cpi_plane* planes, int32_t n_planes, float* out, void* workspace,
                       size_t workspace_bytes, cpi_stream stream) {
    return run_refocus(gamma_f32, ha, wa, hb, wb, planes, n_planes, out, workspace, workspace_bytes,
                       reinterpret_cast<cudaStream_t>(stream));
}

size_t cpi_batch_workspace_size(const cpi_batch_item* items, int32_t n_items) {
    DeviceInfo* dev = nullptr;
    int sm = 152;
    if (device_info(&dev) == cudaSuccess) sm = dev->sm_count;
    size_t most = 0;
    for (int c = 0; c < 6; ++c) {
        BatchPlan bp;
        if (make_batch_plan(items, n_items, sm, kBatchCandidates[c], &bp) != CPI_OK) return 0;
        most = bp.ws_bytes > most ? bp.ws_bytes : most;
    }
    return most;
}

cpi_status cpi_batch_correlate(const cpi_batch_item* items, int32_t n_items, void* workspace,
                               size_t workspace_bytes, int32_t flags, cpi_stream stream) {
    DeviceInfo* dev = nullptr;
    if (device_info(&dev) != cudaSuccess) return CPI_ERR_CUDA;
    int dev_id = 0;
    if (cudaGetDevice(&dev_id) != cudaSuccess) return CPI_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    BatchPlan probe;
    cpi_status s = make_batch_plan(items, n_items, dev->sm_count, kBatchCandidates[0], &probe);   // validates the items
    if (s != CPI_OK) return s;
    if (!workspace || !aligned(workspace, 256) || workspace_bytes < cpi_batch_workspace_size(items, n_items))
        return CPI_ERR_WORKSPACE;
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    BatchShape shape = (flags & CPI_BATCH_N128) ? BatchShape{1, 128} : kBatchCandidates[0];
    if (flags & CPI_BATCH_TUNE) {
        s = tuned_shape(items, n_items, ws, dev, dev_id, st, &shape);
        if (s != CPI_OK) return s;
    }
    BatchPlan bp;
    s = make_batch_plan(items, n_items, dev->sm_count, shape, &bp);
    if (s != CPI_OK) return s;
    if (!(flags & CPI_BATCH_GRAPH)) return run_batch(items, bp, ws, dev, st);

    const uint64_t key = batch_graph_key(items, n_items, workspace, shape, dev_id);
    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_batch.mu);
        for (auto& g : g_batch.graphs[dev_id])
            if (g.first == key) exec = g.second;
        if (exec == nullptr && g_batch.capture_stream[dev_id] == nullptr &&
            cudaStreamCreateWithFlags(&g_batch.capture_stream[dev_id], cudaStreamNonBlocking) != cudaSuccess)
            return CPI_ERR_CUDA;
    }
    if (exec == nullptr) {
        cudaStream_t cap = g_batch.capture_stream[dev_id];
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CPI_ERR_CUDA;
        s = run_batch(items, bp, ws, dev, cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(cap, &graph);
        if (s != CPI_OK || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return s != CPI_OK ? s : CPI_ERR_CUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return CPI_ERR_CUDA;
        std::lock_guard<std::mutex> lk(g_batch.mu);
        auto& v = g_batch.graphs[dev_id];
        if (v.size() >= kMaxGraphs) {
            cudaGraphExecDestroy(v.front().second);
            v.erase(v.begin());
        }
        v.emplace_back(key, exec);
    }
    return cudaGraphLaunch(exec, st) == cudaSuccess ? CPI_OK : CPI_ERR_CUDA;
}

size_t cpi_refocus4d_workspace_size(int32_t ha, int32_t wa, int32_t hb, int32_t wb, int32_t n_planes) {
    if (ha < 1 || wa < 1 || hb < 1 || wb < 1 || n_planes < 1) return 0;
    if ((int64_t)ha * wa > kMaxPixels || (int64_t)hb * wb > kMaxPixels) return 0;
    return refocus4d_layout(ha, wa, hb, wb, n_planes).bytes;
}

cpi_status cpi_refocus4d(const float* gamma_f32, int32_t ha, int32_t wa, int32_t hb, int32_t wb,
                         const cpi_plane4* planes, int32_t n_planes, float* out, void* workspace,
                         size_t workspace_bytes, cpi_stream stream) {
    if (!gamma_f32 || !planes || !out || n_planes < 1) return CPI_ERR_INVALID_ARG;
    if (ha < 1 || wa < 1 || hb < 1 || wb < 1) return CPI_ERR_INVALID_ARG;
    if ((int64_t)ha * wa > kMaxPixels || (int64_t)hb * wb > kMaxPixels) return CPI_ERR_INVALID_ARG;
    if (!aligned(gamma_f32, 4) || !aligned(out, 4)) return CPI_ERR_INVALID_ARG;
    for (int i = 0; i < n_planes; ++i) {
        const double c[4] = {planes[i].alpha, planes[i].beta, planes[i].gamma, planes[i].delta};
        for (double v : c)
            if (!(std::fabs(v) <= kRefocusMaxCoef)) return CPI_ERR_INVALID_ARG;
    }
    const Refocus4dLayout L = refocus4d_layout(ha, wa, hb, wb, n_planes);
    if (!workspace || workspace_bytes < L.bytes || !aligned(workspace, 256)) return CPI_ERR_WORKSPACE;
    DeviceInfo* dev = nullptr;
    if (device_info(&dev) != cudaSuccess) return CPI_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Plane4Block pb;
    for (int p0 = 0; p0 < n_planes; p0 += L.chunk) {
        const int np = n_planes - p0 < L.chunk ? n_planes - p0 : L.chunk;
        std::memset(&pb, 0, sizeof(pb));
        for (int i = 0; i < np; ++i) {
            pb.c[i][0] = planes[p0 + i].alpha;
            pb.c[i][1] = planes[p0 + i].beta;
            pb.c[i][2] = planes[p0 + i].gamma;
            pb.c[i][3] = planes[p0 + i].delta;
        }
        const cudaError_t e = launch_refocus4d_chunk(gamma_f32, ha, wa, hb, wb, pb, np, static_cast<uint8_t*>(workspace),
                                                     L, out + (int64_t)p0 * ha * wa, st);
        if (e != cudaSuccess) return CPI_ERR_CUDA;
    }
    return CPI_OK;
}

static bool denoise_shape_ok(int32_t ha, int32_t wa, int32_t hb, int32_t wb) {
    return ha >= 1 && wa >= 1 && hb >= 1 && wb >= 1 && (int64_t)hb * wb <= 65535 &&
           (int64_t)ha * wa <= ((int64_t)1 << 24);
}

size_t cpi_denoise_workspace_size(int32_t ha, int32_t wa, int32_t hb, int32_t wb, int32_t training) {
    if (!denoise_shape_ok(ha, wa, hb, wb)) return 0;
    return denoise_layout(ha, wa, hb, wb, training != 0).bytes;
}

cpi_status cpi_denoise(const float* model, const float* gamma_in, float* gamma_out, int32_t ha, int32_t wa,
                       int32_t hb, int32_t wb, void* workspace, size_t workspace_bytes, cpi_stream stream) {
    if (!model || !gamma_in || !gamma_out || !denoise_shape_ok(ha, wa, hb, wb)) return CPI_ERR_INVALID_ARG;
    const DenoiseLayout L = denoise_layout(ha, wa, hb, wb, false);
    if (!workspace || workspace_bytes < L.bytes || !aligned(workspace, 256)) return CPI_ERR_WORKSPACE;
    DeviceInfo* dev = nullptr;
    if (device_info(&dev) != cudaSuccess) return CPI_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    cudaError_t e = denoise_forward(model, gamma_in, ha, wa, hb, wb, ws, L, false, dev->status, g_timeout_ns, st);
    if (e == cudaSuccess) e = denoise_output(ws, L, (int64_t)hb * wb * ha * wa, gamma_out, st);
    return cuda_status(e);
}

cpi_status cpi_denoise_grad(const float* model, const float* gamma_in, const float* gamma_target, int32_t ha,
                            int32_t wa, int32_t hb, int32_t wb, float* grad, float* loss, void* workspace,
                            size_t workspace_bytes, cpi_stream stream) {
    if (!model || !gamma_in || !gamma_target || !grad || !loss || !denoise_shape_ok(ha, wa, hb, wb))
        return CPI_ERR_INVALID_ARG;
    const DenoiseLayout L = denoise_layout(ha, wa, hb, wb, true);
    if (!workspace || workspace_bytes < L.bytes || !aligned(workspace, 256)) return CPI_ERR_WORKSPACE;
    DeviceInfo* dev = nullptr;
    if (device_info(&dev) != cudaSuccess) return CPI_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    cudaError_t e = denoise_forward(model, gamma_in, ha, wa, hb, wb, ws, L, true, dev->status, g_timeout_ns, st);
    if (e == cudaSuccess)
        e = denoise_backward(model, gamma_target, ha, wa, hb, wb, ws, L, grad, loss, dev->sm_count, dev->status,
                             g_timeout_ns, st);
    return cuda_status(e);
}

cpi_status cpi_denoise_adam(float* model, float* m, float* v, const float* grad, int64_t step, float lr,
                            cpi_stream stream) {
    if (!model || !m || !v || !grad || step < 1 || !(lr > 0.0f) || !std::isfinite(lr)) return CPI_ERR_INVALID_ARG;
    DeviceInfo* dev = nullptr;
    if (device_info(&dev) != cudaSuccess) return CPI_ERR_CUDA;
    return cuda_status(denoise_adam(model, m, v, grad, step, lr, reinterpret_cast<cudaStream_t>(stream)));
}

cpi_status cpi_device_status(cpi_stream stream, int32_t clear) {
    DeviceInfo* dev = nullptr;
    if (device_info(&dev) != cudaSuccess) return CPI_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return CPI_ERR_CUDA;
    unsigned int word = 0;
    if (cudaMemcpyFromSymbol(&word, g_device_status, sizeof(word)) != cudaSuccess)
        return CPI_ERR_CUDA;
    if (clear && word) {
        const unsigned int zero = 0;
        if (cudaMemcpyToSymbol(g_device_status, &zero, sizeof(zero)) != cudaSuccess)
            return CPI_ERR_CUDA;
    }
    return (word & kStatusTimeoutBit) ? CPI_ERR_TIMEOUT : CPI_OK;
}

void cpi_set_wait_timeout_ns(int64_t ns) {
    g_timeout_ns = ns > 0 ? (unsigned long long)ns : 2000000000ull;
}

cpi_status cpi_correlate_noalloc(const cpi_frames* a, const cpi_frames* b, int64_t n_frames,
                                 int64_t* s_ab, int64_t* s_a, int64_t* s_b, double* gamma,
                                 float* gamma_f32, cpi_stream stream) {
    // Set-up, once per device with that device current: the device address of
    // the built-in scratch array.
    static void* scratch[kMaxDevices] = {};
    static std::mutex scratch_mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CPI_ERR_CUDA;
    void* ws = nullptr;
    {
        std::lock_guard<std::mutex> lk(scratch_mu);
        if (scratch[dev] == nullptr) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
                return CPI_ERR_CUDA;
            scratch[dev] = p;
        }
        ws = scratch[dev];
    }
    // The problem must fit the built-in scratch; nothing is allocated otherwise.
    DeviceInfo* info = nullptr;
    if (device_info(&info) != cudaSuccess) return CPI_ERR_CUDA;
    CorrPlan pl;
    const cpi_status s = make_plan(a, b, n_frames, info->sm_count, &pl);
    if (s != CPI_OK) return s;
    if (pl.ws_bytes > (size_t)CPI_NOALLOC_SCRATCH_BYTES) return CPI_ERR_WORKSPACE;
    // Every scratch byte a call reads is written earlier in the same call
    // (operand rows including their zero padding, then one partial slot per
    // unit), so nothing left by a previous call needs clearing.
    static const int32_t stages[3] = {CPI_STAGE_INGEST, CPI_STAGE_MOMENTS, CPI_STAGE_FOLD};
    return correlate_common(stages, 3, a, b, n_frames, 0, s_ab, s_a, s_b, gamma, gamma_f32, ws,
                            (size_t)CPI_NOALLOC_SCRATCH_BYTES, stream);
}

cpi_status cpi_selftest_wait_timeout(int64_t timeout_ns, cpi_stream stream) {
    if (timeout_ns <= 0 || timeout_ns > 10000000000ll) return CPI_ERR_INVALID_ARG;
    DeviceInfo* dev = nullptr;
    if (device_info(&dev) != cudaSuccess) return CPI_ERR_CUDA;
    return cuda_status(launch_wait_selftest(dev->status, (unsigned long long)timeout_ns,
                                            reinterpret_cast<cudaStream_t>(stream)));
}


size_t cpi_acq_workspace_size(const cpi_frames* a, const cpi_frames* b, int64_t block_frames) {
    if (acq_check_layout(a, b, block_frames) != CPI_OK) return 0;
    cpi_frames ta = *a, tb = *b;
    ta.data = tb.data = reinterpret_cast<const void*>(uintptr_t(256));
    const size_t ws = cpi_correlate_workspace_size(&ta, &tb, block_frames);
    if (ws == 0) return 0;
    return 2 * acq_staging_bytes(a, block_frames) + ws;
}

cpi_status cpi_acq_begin(cpi_acq** out, const cpi_frames* a, const cpi_frames* b, int64_t block_frames,
                         int64_t* s_ab, int64_t* s_a, int64_t* s_b, int64_t frames_done, void* workspace,
                         size_t workspace_bytes, cpi_stream stream) {
    if (!out) return CPI_ERR_INVALID_ARG;
    *out = nullptr;
    cpi_status st = acq_check_layout(a, b, block_frames);
    if (st != CPI_OK) return st;
    if (!s_ab || !s_a || !s_b || !aligned(s_ab, 16) || !aligned(s_a, 16) || !aligned(s_b, 16))
        return CPI_ERR_INVALID_ARG;
    if (frames_done < 0 || frames_done > ((int64_t)1 << 31) - 1) return CPI_ERR_INVALID_ARG;
    const size_t need = cpi_acq_workspace_size(a, b, block_frames);
    if (need == 0) return CPI_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256)) return CPI_ERR_WORKSPACE;
    std::unique_ptr<Acquisition> q(new Acquisition);
    if (cudaGetDevice(&q->dev) != cudaSuccess) return CPI_ERR_CUDA;
    q->a = *a;
    q->b = *b;
    q->block_frames = block_frames;
    q->frame_bytes = a->frame_stride_bytes;
    q->s_ab = s_ab;
    q->s_a = s_a;
    q->s_b = s_b;
    uint8_t* w = static_cast<uint8_t*>(workspace);
    const size_t sb = acq_staging_bytes(a, block_frames);
    q->staging[0] = w;
    q->staging[1] = w + sb;
    q->ws = w + 2 * sb;
    q->ws_bytes = workspace_bytes - 2 * sb;
    q->compute = reinterpret_cast<cudaStream_t>(stream);
    q->n_done = frames_done;
    if (a->bits == 1 && b->bits == 1) {
        DeviceInfo* dev = nullptr;
        if (device_info(&dev) != cudaSuccess) return CPI_ERR_CUDA;
        cpi_frames ta = *a, tb = *b;
        ta.data = tb.data = w;
        CorrPlan pl;
        if (make_plan(&ta, &tb, block_frames, dev->sm_count, &pl) == CPI_OK) {
            q->defer = true;
            q->off_part = pl.off_part;
            q->n_chunks = pl.n_chunks;
        }
    }
    if (cudaStreamCreateWithFlags(&q->copy, cudaStreamNonBlocking) != cudaSuccess) return CPI_ERR_CUDA;
    for (int k = 0; k < 2; ++k)
        if (cudaEventCreateWithFlags(&q->arrived[k], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&q->consumed[k], cudaEventDisableTiming) != cudaSuccess) {
            cpi_acq_end(reinterpret_cast<cpi_acq*>(q.release()));
            return CPI_ERR_CUDA;
        }
    if (frames_done == 0) {       // a new acquisition: the running sums start at zero
        cudaStream_t cs = q->compute;
        const int64_t ma = (int64_t)a->height * a->width, mb = (int64_t)b->height * b->width;
        if (cudaMemsetAsync(s_ab, 0, (size_t)ma * mb * 8, cs) != cudaSuccess ||
            cudaMemsetAsync(s_a, 0, (size_t)ma * 8, cs) != cudaSuccess ||
            cudaMemsetAsync(s_b, 0, (size_t)mb * 8, cs) != cudaSuccess) {
            cpi_acq_end(reinterpret_cast<cpi_acq*>(q.release()));
            return CPI_ERR_CUDA;
        }
    }
    *out = reinterpret_cast<cpi_acq*>(q.release());
    return CPI_OK;
}

cpi_status cpi_acq_push(cpi_acq* handle, const void* host_frames, int64_t n_frames) {
    Acquisition* q = reinterpret_cast<Acquisition*>(handle);
    if (!q || !host_frames || n_frames < 1 || n_frames > q->block_frames) return CPI_ERR_INVALID_ARG;
    if (q->n_done + n_frames > ((int64_t)1 << 31) - 1) return CPI_ERR_OVERFLOW;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != q->dev) return CPI_ERR_INVALID_ARG;
    const int k = q->next;
    uint8_t* dst = q->staging[k];
    // staging k is free once the block it held two pushes ago has been accumulated
    if (q->copied_once[k] && cudaStreamWaitEvent(q->copy, q->consumed[k], 0) != cudaSuccess) return CPI_ERR_CUDA;
    if (cudaMemcpyAsync(dst, host_frames, (size_t)n_frames * (size_t)q->frame_bytes, cudaMemcpyHostToDevice,
                        q->copy) != cudaSuccess ||
        cudaEventRecord(q->arrived[k], q->copy) != cudaSuccess ||
        cudaStreamWaitEvent(q->compute, q->arrived[k], 0) != cudaSuccess)
        return CPI_ERR_CUDA;
    cpi_frames a = q->a, b = q->b;
    a.data = dst;
    b.data = dst;
    static const int32_t stages[3] = {CPI_STAGE_INGEST, CPI_STAGE_MOMENTS, CPI_STAGE_FOLD};
    const bool defer = q->defer && n_frames == q->block_frames;
    if (!defer) {
        const cpi_status f = acq_flush(q);   // a block of another size uses another layout
        if (f != CPI_OK) return f;
    }
    const cpi_status st = correlate_common(stages, defer ? 2 : 3, &a, &b, n_frames, 1, q->s_ab, q->s_a, q->s_b,
                                           nullptr, nullptr, q->ws, q->ws_bytes,
                                           reinterpret_cast<cpi_stream>(q->compute), defer && q->deferred > 0 ? 1 : 0);
    if (st != CPI_OK) return st;
    if (defer) ++q->deferred;
    if (cudaEventRecord(q->consumed[k], q->compute) != cudaSuccess) return CPI_ERR_CUDA;
    q->copied_once[k] = true;
    // the previous block's host buffer is free once its copy has arrived
    const int prev = k ^ 1;
    if (q->copied_once[prev] && cudaEventSynchronize(q->arrived[prev]) != cudaSuccess) return CPI_ERR_CUDA;
    q->n_done += n_frames;
    q->next = prev;
    return CPI_OK;
}

int64_t cpi_acq_frames(const cpi_acq* handle) {
    const Acquisition* q = reinterpret_cast<const Acquisition*>(handle);
    return q ? q->n_done : -1;
}

cpi_status cpi_acq_finalize(cpi_acq* handle, double* gamma, float* gamma_f32) {
    Acquisition* q = reinterpret_cast<Acquisition*>(handle);
    if (!q || q->n_done < 1) return CPI_ERR_INVALID_ARG;
    const int64_t ma = (int64_t)q->a.height * q->a.width, mb = (int64_t)q->b.height * q->b.width;
    const cpi_status f = acq_flush(q);
    if (f != CPI_OK) return f;
    return cpi_correlate_finalize(q->s_ab, q->s_a, q->s_b, ma, mb, q->n_done, gamma, gamma_f32,
                                  reinterpret_cast<cpi_stream>(q->compute));
}

cpi_status cpi_acq_sync(cpi_acq* handle) {
    Acquisition* q = reinterpret_cast<Acquisition*>(handle);
    if (!q) return CPI_ERR_INVALID_ARG;
    const cpi_status f = acq_flush(q);
    if (f != CPI_OK) return f;
    if (cudaStreamSynchronize(q->copy) != cudaSuccess || cudaStreamSynchronize(q->compute) != cudaSuccess)
        return CPI_ERR_CUDA;
    return CPI_OK;
}

cpi_status cpi_acq_end(cpi_acq* handle) {
    Acquisition* q = reinterpret_cast<Acquisition*>(handle);
    if (!q) return CPI_ERR_INVALID_ARG;
    cpi_status st = acq_flush(q);
    if (q->copy && cudaStreamSynchronize(q->copy) != cudaSuccess) st = CPI_ERR_CUDA;
    if (q->compute && cudaStreamSynchronize(q->compute) != cudaSuccess) st = CPI_ERR_CUDA;
    for (int k = 0; k < 2; ++k) {
        if (q->arrived[k]) cudaEventDestroy(q->arrived[k]);
        if (q->consumed[k]) cudaEventDestroy(q->consumed[k]);
    }
    if (q->copy) cudaStreamDestroy(q->copy);
    delete q;
    return st;
}

}  // extern "C"

