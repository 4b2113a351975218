// Step a2: the raw-moment contraction S_ab[a][b] = sum_i A_i[a] B_i[b] (the
// first term of Eq. (1)) on the 5th-generation tensor cores.
//
// Operands are the K-major rows written by the ingest step (one row per pixel,
// K = frames): E2M1 0/1 values for binary frames (tcgen05 kind::f8f6f4, packed
// two per byte in HBM and spread to 16-byte groups in shared memory by TMA), or
// BF16 integers 0..255 (kind::f16).  Products are small integers, accumulated
// in FP32 in tensor memory; a sum of integers stays exact while it is below
// 2^24, and the schedule guarantees that:
//   - binary frames: a frame chunk has at most 65536 frames, so every sum is
//     <= 65536;
//   - 8-bit values: the FP32 accumulator is folded into exact uint32 running
//     sums (in the epilogue threads' registers) every S frames, S the largest
//     multiple of 64 with S x max A x max B < 2^24 (at least 256 frames, since
//     256 x 255^2 < 2^24).  The maxima are the ones the ingest records for the
//     call's frames, read on the device, so photon counts far below 255 fold
//     rarely or never.  Each segment sum, an integer below 2^24, converts
//     exactly (cvt.rni.u32.f32).  (Bounding the segments by 2^23 instead, where
//     f + 2^23 gives the integer in its bit pattern without a conversion,
//     halves S; measured slower, 3.95 -> 4.23 ms on 128x128 vs 64x64 with
//     N = 50000.)  A chunk of <= 65536 frames keeps each total below
//     65536 x 255^2 < 2^32 (the running sums are uint32: every product is
//     non-negative).
// Each (frame chunk, 128 x 256 output tile) of a problem is one work unit; its
// exact partial sum goes to its own slot of the workspace, and the fold step
// adds the slots into int64.  (Finishing Eq. (1) in this epilogue was measured
// slower on GB300: the correctly rounded quotients keep the epilogue warps from
// draining the next tile's segments, and the MMAs wait; the fold kernel spreads
// that work over every SM instead.)  Integer addition is associative, so the
// split over chunks, segments and CTAs never changes the result.  One launch
// serves one problem (a correlation) or up to kMaxGroup problems of uneven
// shapes (a batch): the persistent CTAs walk one list of units, each unit naming
// its problem by a binary search over the problems' first units.
//
// Persistent, warp-specialised CTA (one per SM, 320 threads):
//   warp 0   : TMA producer (128-byte swizzled tiles, 4-deep ring)
//   warp 1   : tensor-memory allocator and single-thread MMA issuer
//   warps 2-9: epilogue, tensor memory -> registers -> global (TMEM lanes 32*(w%4)..)
// Two TMEM accumulators let the epilogue of one unit (binary frames) or one
// exact FP32 segment (8-bit frames) overlap the MMAs of the next; the 8-bit
// int32 running sums of a unit stay in the epilogue threads' registers.  Every barrier wait is bounded; on a
// time-out the CTA records the error, drains its own copies and MMAs, frees its
// tensor memory and returns.
#include "kernels.cuh"
#include "ptx.cuh"

namespace cpi {
namespace {

constexpr int kBlockM = 128;
constexpr int kRowBytes = 128;                 // K-block: one 128-byte swizzle row
constexpr int kThreads = 320;                  // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int kEpiThreads = 256;

template <bool kBf16, int kBN>
struct MomentsCfg {
    static constexpr int kBlockN = kBN;                         // 256 or 128 (batches tune it)
    static constexpr int kStages = kBN == 256 ? 4 : 6;
    static constexpr int kElem = kBf16 ? 2 : 1;
    static constexpr int kKPerBlock = kRowBytes / kElem;     // 64 / 128 elements
    static constexpr int kABytes = kBlockM * kRowBytes;       // 16 KiB
    static constexpr int kBBytes = kBlockN * kRowBytes;       // 32 KiB
    // bytes a stage's copies deliver: E2M1 rows are 64 bytes in HBM, spread over
    // the 128-byte shared-memory row (8 bytes of values per 16-byte group)
    static constexpr uint32_t kTxBytes = kBf16 ? kABytes + kBBytes : (kABytes + kBBytes) / 2;
    // tensor memory (2 x kBN columns): two FP32 accumulators, so the epilogue of
    // one unit (FP8) or segment (BF16) overlaps the MMAs of the next; the BF16
    // int32 running sums live in the epilogue threads' registers
    static constexpr int kAcc = 2;
    static constexpr uint32_t kTmemCols = 2 * kBN;
    static constexpr size_t kSmem = 1024 + (size_t)kStages * (kABytes + kBBytes) + 256;
};

// Write (with add_partial: add) 32 exact sums of output row m, columns
// nb .. nb+31 (those < N), to the chunk's partial slot (uint32 bit patterns).
__device__ __forceinline__ void store_row_chunk(const MomentsProblem& P, int chunk, int m, int nb,
                                                const int32_t (&v)[32]) {
    if (m >= P.M) return;
    int32_t* out = P.partial + ((size_t)chunk * P.M + (size_t)m) * P.N;
    const bool add = P.add_partial != 0;
    if ((P.N & 3) == 0 && nb + 32 <= P.N) {
        int4* o4 = reinterpret_cast<int4*>(out + nb);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int4 w = make_int4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            if (add) {
                const int4 o = o4[j];
                w = make_int4((int)((uint32_t)w.x + (uint32_t)o.x), (int)((uint32_t)w.y + (uint32_t)o.y),
                              (int)((uint32_t)w.z + (uint32_t)o.z), (int)((uint32_t)w.w + (uint32_t)o.w));
            }
            o4[j] = w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (nb + j < P.N) out[nb + j] = add ? (int32_t)((uint32_t)out[nb + j] + (uint32_t)v[j]) : v[j];
    }
}

struct Unit {
    int prob, chunk, tm, tn, kb0, kb1;
};

// Unit u of the launch: its problem (binary search over first units), frame
// chunk, output tile and K-block range.  Within a chunk the tiles run in groups
// of kGroupM tile rows, column by column (row fastest), so the persistent CTAs
// working at one time cover a block of about kGroupM rows x (CTAs / kGroupM)
// columns of tiles: the A and B rows they stream stay within L2 (a row-by-row
// order has every CTA of a wave read its own B rows, which for wide problems
// do not fit and come from DRAM once per tile row).
constexpr int kGroupM = 16;
template <int K>
__device__ __forceinline__ Unit decode_unit(const MomentsLaunch<K>& L, int u) {
    int lo = 0;
    if constexpr (K > 1) {
        int hi = L.n_problems - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (L.prob[mid].unit_begin <= u) lo = mid;
            else hi = mid - 1;
        }
    }
    const MomentsProblem& P = L.prob[lo];
    const int local = u - P.unit_begin;
    const int per_chunk = P.tiles_m * P.tiles_n;
    Unit w;
    w.prob = lo;
    w.chunk = local / per_chunk;
    const int t = local - w.chunk * per_chunk;
    const int g = t / (kGroupM * P.tiles_n);                       // group of tile rows
    const int m0 = g * kGroupM;
    const int gm = min(kGroupM, P.tiles_m - m0);                   // rows in this group
    const int r = t - g * kGroupM * P.tiles_n;
    w.tn = r / gm;
    w.tm = m0 + (r - w.tn * gm);
    w.kb0 = w.chunk * P.kb_per_chunk;
    w.kb1 = min(w.kb0 + P.kb_per_chunk, P.k_blocks);
    return w;
}

// K blocks (64 frames) per exact FP32 segment of a BF16 problem: the largest S
// with S x 64 x max A x max B < 2^24, from the ingest's maxima (worst case
// 255 x 255 when they are missing).
__device__ __forceinline__ int segment_kblocks(const MomentsProblem& P) {
    uint64_t prod = 255u * 255u;
    if (P.vmax != nullptr) prod = (uint64_t)__ldcg(P.vmax) * (uint64_t)__ldcg(P.vmax + 1);
    if (prod < 1) prod = 1;
    const uint64_t frames = ((1ull << 24) - 1) / prod;
    const uint64_t kb = frames / 64;
    return kb < 1 ? 1 : (kb > 0x40000000ull ? 0x40000000 : (int)kb);
}

template <bool kBf16, int kBN, int K>
__global__ void __launch_bounds__(kThreads, 1)
    moments_kernel(const __grid_constant__ MomentsLaunch<K> L) {
    using C = MomentsCfg<kBf16, kBN>;
    __shared__ int seg_kb[K];   // BF16: K blocks per exact FP32 segment, per problem
    if constexpr (kBf16)
        for (int p = threadIdx.x; p < L.n_problems; p += blockDim.x) seg_kb[p] = segment_kblocks(L.prob[p]);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    uint8_t* sA = smem;
    uint8_t* sB = sA + C::kStages * C::kABytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + C::kStages * C::kBBytes);
    uint64_t* empty = full + C::kStages;
    uint64_t* tfull = empty + C::kStages;      // [kAcc] accumulator ready for the epilogue
    uint64_t* tempty = tfull + C::kAcc;        // [kAcc] accumulator drained by the epilogue
    uint64_t* drain = tempty + C::kAcc;        // MMA drain on abort
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t tmo = L.timeout_ns;
    unsigned int* const status = L.status;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < C::kAcc; ++s) {
            mbar_init(&tfull[s], 1);
            mbar_init(&tempty[s], kEpiThreads);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_barrier_init();
        fence_proxy_async_smem();
        if constexpr (K == 1) {
            tma_prefetch_desc(&L.map_a[0]);
            tma_prefetch_desc(&L.map_b[0]);
        }
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, C::kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------------- producer
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued_mask = 0, issued_phase = 0;   // per stage: loaded at least once / parity
            bool ok = true;
            for (int u = blockIdx.x; ok && u < L.n_units; u += gridDim.x) {
                const Unit w = decode_unit<K>(L, u);
                const CUtensorMap* ma = &L.map_a[w.prob];
                const CUtensorMap* mb = &L.map_b[w.prob];
                for (int kb = w.kb0; kb < w.kb1; ++kb) {
                    if (!mbar_wait_bounded(&empty[stage], phase ^ 1, abort_flag, status, tmo)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[stage], C::kTxBytes);
                    tma_load_2d(sA + stage * C::kABytes, ma, &full[stage], kb * C::kKPerBlock,
                                w.tm * kBlockM);
                    tma_load_2d(sB + stage * C::kBBytes, mb, &full[stage], kb * C::kKPerBlock,
                                w.tn * C::kBlockN);
                    issued_mask |= 1u << stage;
                    issued_phase = (issued_phase & ~(1u << stage)) | (phase << stage);
                    if (++stage == C::kStages) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
            }
            if (!ok) {
                // Wait (bounded, regardless of the abort flag) for the copies this
                // thread issued, so no TMA write lands after the CTA exits.
                for (int s = 0; s < C::kStages; ++s)
                    if (issued_mask & (1u << s))
                        mbar_wait_bounded(&full[s], (issued_phase >> s) & 1u, nullptr, nullptr, tmo);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------------- MMA issuer
            // The tensor pipe takes one 128 x 256 x 16 (BF16) or x 32 (E2M1) MMA
            // per 128 cycles only while this thread issues the next one within
            // that time, so the loop keeps its per-K-block work to a few adds:
            // segment bounds are counted down (no division), descriptors step
            // by the stage size.
            constexpr uint32_t idesc = idesc_f32acc<kBf16>(kBlockM, C::kBlockN);
            const uint64_t da0 = sdesc_kmajor_sw128(smem_u32(sA));
            const uint64_t db0 = sdesc_kmajor_sw128(smem_u32(sB));
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true, issued_any = false;
            for (int u = blockIdx.x; ok && u < L.n_units; u += gridDim.x) {
                const Unit w = decode_unit<K>(L, u);
                const int nkb = w.kb1 - w.kb0;
                const int kb_per_seg = kBf16 ? seg_kb[w.prob] : nkb;
                int seg_left = 0;   // K blocks left in the current segment
                for (int i = 0; i < nkb; ++i) {
                    const bool seg_start = seg_left == 0;
                    if (seg_start) {
                        seg_left = min(kb_per_seg, nkb - i);
                        if (!mbar_wait_bounded(&tempty[acc], acc_phase ^ 1, abort_flag, status, tmo)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                    }
                    --seg_left;
                    if (!mbar_wait_bounded(&full[stage], phase, abort_flag, status, tmo)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem_base + (uint32_t)(acc * C::kBlockN);
                    const uint64_t da = da0 + (uint64_t)(stage * (C::kABytes >> 4));
                    const uint64_t db = db0 + (uint64_t)(stage * (C::kBBytes >> 4));
#pragma unroll
                    for (int k = 0; k < kRowBytes / 32; ++k) {
                        // advance the start address by 32 bytes (2 x 16-byte units) per MMA
                        umma_f32<kBf16>(d, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc,
                                        (seg_start && k == 0) ? 0u : 1u);
                    }
                    issued_any = true;
                    umma_commit(&empty[stage]);
                    if (++stage == C::kStages) {
                        stage = 0;
                        phase ^= 1;
                    }
                    if (seg_left == 0) {   // segment (BF16) or unit (E2M1) done: hand the accumulator over
                        umma_commit(&tfull[acc]);
                        if (++acc == C::kAcc) {
                            acc = 0;
                            acc_phase ^= 1;
                        }
                    }
                }
            }
            if (!ok && issued_any) {
                umma_commit(drain);
                mbar_wait_bounded(drain, 0, nullptr, nullptr, tmo);
            }
        }
    } else {
        // -------------------------------------------------------------- epilogue
        // Warps 2..9: warp w reads TMEM lanes 32*(w%4).. (its rows) and one half
        // of the tile's columns.
        const int q = warp & 3;                       // TMEM lane quarter of this warp
        const int half = (warp - 2) >> 2;             // column half
        constexpr int kHalf = C::kBlockN / 2;
        const int row = q * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        int acc = 0;
        uint32_t acc_phase = 0;
        bool ok = true;
        for (int u = blockIdx.x; ok && u < L.n_units; u += gridDim.x) {
            const Unit w = decode_unit<K>(L, u);
            const MomentsProblem& P = L.prob[w.prob];
            const int chunk = w.chunk;
            const int kb0 = w.kb0, kb1 = w.kb1;
            const int m = w.tm * kBlockM + row;
            const int n0 = w.tn * C::kBlockN + half * kHalf;
            const uint32_t col0 = (uint32_t)(half * kHalf);
            if constexpr (!kBf16) {
                if (!mbar_wait_bounded(&tfull[acc], acc_phase, abort_flag, status, tmo)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll 1
                for (int c = 0; c < kHalf / 32; ++c) {
                    uint32_t r[32];
                    tmem_ld_32x32b_x32(tmem_base + lane_addr + (uint32_t)(acc * C::kBlockN) + col0 + c * 32, r);
                    tmem_ld_wait();
                    int32_t v[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = __float2int_rn(__uint_as_float(r[j]));
                    store_row_chunk(P, chunk, m, n0 + c * 32, v);
                }
                tc_fence_before();
                mbar_arrive(&tempty[acc]);
                if (++acc == C::kAcc) {
                    acc = 0;
                    acc_phase ^= 1;
                }
            } else {
                // Every segment: running sums (registers, uint32) += the FP32
                // segment sums (integers < 2^24, converted exactly); after the
                // last segment they go to the partial slot.
                const int seg = seg_kb[w.prob];
                const int nseg = (kb1 - kb0 + seg - 1) / seg;
                uint32_t run[kHalf / 16][16];
#pragma unroll
                for (int c = 0; c < kHalf / 16; ++c)
#pragma unroll
                    for (int j = 0; j < 16; ++j) run[c][j] = 0u;
                for (int sgm = 0; sgm < nseg; ++sgm) {
                    if (!mbar_wait_bounded(&tfull[acc], acc_phase, abort_flag, status, tmo)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int c = 0; c < kHalf / 16; ++c) {
                        uint32_t r[16];
                        tmem_ld_32x32b_x16(tmem_base + lane_addr + (uint32_t)(acc * C::kBlockN) + col0 + c * 16, r);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            run[c][j] += __float2uint_rn(__uint_as_float(r[j]));
                    }
                    tc_fence_before();
                    mbar_arrive(&tempty[acc]);
                    if (++acc == C::kAcc) {
                        acc = 0;
                        acc_phase ^= 1;
                    }
                }
                if (!ok) break;
#pragma unroll
                for (int c = 0; c < kHalf / 32; ++c) {
                    int32_t v[32];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        v[j] = (int32_t)run[2 * c][j];
                        v[16 + j] = (int32_t)run[2 * c + 1][j];
                    }
                    store_row_chunk(P, chunk, m, n0 + c * 32, v);
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, C::kTmemCols);
    }
}

}  // namespace

MomentsShape moments_shape(bool bf16, int block_n) {
    if (block_n == 128) {
        if (bf16)
            return {128, MomentsCfg<true, 128>::kKPerBlock, MomentsCfg<true, 128>::kStages, MomentsCfg<true, 128>::kSmem};
        return {128, MomentsCfg<false, 128>::kKPerBlock, MomentsCfg<false, 128>::kStages, MomentsCfg<false, 128>::kSmem};
    }
    if (bf16)
        return {256, MomentsCfg<true, 256>::kKPerBlock, MomentsCfg<true, 256>::kStages, MomentsCfg<true, 256>::kSmem};
    return {256, MomentsCfg<false, 256>::kKPerBlock, MomentsCfg<false, 256>::kStages, MomentsCfg<false, 256>::kSmem};
}

template <bool kBf16, int kBN, int K>
static cudaError_t launch_impl(const MomentsLaunch<K>& L, int sm_count, cudaStream_t st) {
    // The shared-memory opt-in is a per-device function attribute: set it once per device.
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    using C = MomentsCfg<kBf16, kBN>;
    if (!attr_set[dev]) {
        e = cudaFuncSetAttribute(moments_kernel<kBf16, kBN, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)C::kSmem);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    const int grid = L.n_units < sm_count ? L.n_units : sm_count;
    moments_kernel<kBf16, kBN, K><<<grid, kThreads, C::kSmem, st>>>(L);
    return cudaGetLastError();
}

template <int K>
static cudaError_t launch_any(bool bf16, int block_n, const MomentsLaunch<K>& L, int sm_count, cudaStream_t st) {
    if (block_n == 128)
        return bf16 ? launch_impl<true, 128, K>(L, sm_count, st) : launch_impl<false, 128, K>(L, sm_count, st);
    if (block_n == 256)
        return bf16 ? launch_impl<true, 256, K>(L, sm_count, st) : launch_impl<false, 256, K>(L, sm_count, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_moments(bool bf16, int block_n, const MomentsLaunch<1>& L, int sm_count, cudaStream_t st) {
    return launch_any<1>(bf16, block_n, L, sm_count, st);
}

cudaError_t launch_moments_group(bool bf16, int block_n, const MomentsLaunch<kMaxGroup>& L, int sm_count,
                                 cudaStream_t st) {
    return launch_any<kMaxGroup>(bf16, block_n, L, sm_count, st);
}

}  // namespace cpi
