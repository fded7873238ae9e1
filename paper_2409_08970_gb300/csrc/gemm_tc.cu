// Split-TF32 tensor-core GEMM  Y[M x N] = A[M x K] * B[N x K]^T  (FP32 in/out).
//
// Used for the dense Cauchy product of Theorem 3.1 at large n (A = the DCT
// coefficients s of a batch, B = W = X^T U from the plan, y = W s per signal)
// and for the dense-GFT comparison (A = x, B = X^T).
//
// Each FP32 operand is hi + lo with hi, lo TF32: A_hi is A itself (the MMA
// reads it truncated to TF32) and A_lo = rn_tf32(A - trunc_tf32(A)), either
// formed on chip from the landed A slice by converter warps (a source without
// an A_lo array) or loaded (a source whose A is itself a rounded hi / lo pair);
// B_hi, B_lo are both rounded (plan tables). A product takes A_hi B_lo +
// A_lo B_hi (issued first) + A_hi B_hi.
//
// Accumulation: the MMA accumulates in FP32 rounding toward zero, which over
// K = n (up to 4096) would bias results by many ulps. Each K chunk of 32 is
// therefore accumulated in a fresh TMEM buffer (4 large-sum roundings) and the
// epilogue warps add the chunk into FP32 registers with round-to-nearest.
//
// K segments: an output column tile may contract several K ranges, each from
// its own (A, B) source pair: a segment is nch chunks of 32 with A columns
// a_col + 32 c of source src and B columns b_col + 32 c. The band product of
// the hierarchical mode is one segment (a window of s against a slab of W),
// plus a second one that adds the far field (the leaf-local coefficients
// against the L2P weights); the multilevel far field has one segment per
// tree level. Without a segment table every tile has one segment of source 0,
// A columns from kbeg[tile], B columns from 0, K / 32 chunks.
// Optional second output: the TF32 remainder of Y (for a Y that feeds another
// split-TF32 product).
//
// Tiles 128 x BN (BN = 128, or 64 for products with few tiles), persistent CTAs
// (one per SM), 448 threads:
//   warp 0      TMA producer: A_hi, (A_lo,) B_hi, B_lo K-slices of 32 (3 stages)
//   warp 1      TMEM owner (2 BN columns: two chunk buffers), MMA issuer
//   warps 2..9  chunk promotion into registers, final store; two warps per
//               TMEM lane quarter, BN / 2 columns each. A warp writes its
//               32 x BN / 2 block as 32 x 32 boxes staged in its own 4 KB of
//               shared memory and stored by TMA (rows past M are clipped):
//               stores of rows straight from registers would put 32
//               partial-sector L2 writes per instruction into the load/store
//               unit.
//   warps 10..13 A_lo of each landed stage whose source has no A_lo array,
//               written next to A_hi in the same swizzled layout (the
//               remainder is elementwise, so the byte offsets are A_hi's).
//               (Measured: this costs the MMA some shared-memory bandwidth,
//               about 15 % at K = 4096, against loading a stored remainder;
//               keeping A_lo in tensor memory for the MMA was slower still.)
// Bounded waits as in the small-n kernel.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace dctplus {

namespace gemm {

constexpr int kBM = 128, kBK = 32;
constexpr int kStages = 3;
constexpr int kThreads = 448;
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr uint32_t kSlice = kBM * kBK * 4;  // 16 KB: one 128 x 32 FP32 A slice

// Shared-memory layout and TMEM use of a tile 128 x BN (BN = 128 or 64): per stage
// A_hi, A_lo (16 KB each), B_hi, B_lo (BN x 32 FP32 each), then the output staging
// (8 warps x 4 KB) and the barriers; two BN-column TMEM chunk buffers; each of the 8
// epilogue warps owns BN / 2 columns of its lane quarter.
template <int BN>
struct Tile {
    static_assert(BN == 64 || BN == 128, "tile width");
    static constexpr uint32_t kSliceB = BN * kBK * 4;
    static constexpr uint32_t kOffAlo = kSlice, kOffBhi = 2 * kSlice, kOffBlo = 2 * kSlice + kSliceB;
    static constexpr uint32_t kStageBytes = 2 * kSlice + 2 * kSliceB;
    static constexpr uint32_t kOffY = kStages * kStageBytes;
    static constexpr uint32_t kOffBar = kOffY + 8 * 4096;
    static constexpr uint32_t kSmemBytes = kOffBar + 256 + 1024;
    static constexpr int kTmemCols = 2 * BN;
    static constexpr int kWarpCols = BN / 2;
};

constexpr int kMaxTilesN = 256;
constexpr int kMaxSrc = 2;
constexpr int kMaxSeg = 8;
constexpr int kTabStride = 2 + 4 * kMaxSeg;  // per column tile: nseg, nk, {src, a_col, b_col, nch} x kMaxSeg
static_assert(kTabStride == kGemmTabStride && kMaxSeg == kGemmMaxSeg, "table layout");

struct Src {
    CUtensorMap a_hi, a_lo, b_hi, b_lo;  // A: [M x Ka] box 32 x 128, B: [N x Kb] box 32 x BN, FP32
};

struct Params {
    Src src[kMaxSrc];
    CUtensorMap y_map;    // y [M x N], box 32 x 32, 128-byte swizzle
    CUtensorMap ylo_map;  // TF32 remainder of y (when has_lo)
    int has_lo;
    int lo_chip[kMaxSrc]; // 1: form the source's A_lo on chip (no A_lo array)
    int M, N, K;
    int tiles_m, tiles_n;
    unsigned* err;
    const int* tab;       // segment table (device, kTabStride ints per column tile) or null
    int kbeg[kMaxTilesN];
};

// chunks of column tile tn
__device__ __forceinline__ int tile_chunks(const Params& P, int tn) {
    return P.tab ? __ldg(P.tab + tn * kTabStride + 1) : P.K / kBK;
}

// TF32 remainder of v for an operand whose hi part is v itself (the MMA reads v
// truncated to TF32)
__device__ __forceinline__ float tf32_rem(float v) {
    return __uint_as_float(ptx::cvt_rna_tf32(v - __uint_as_float(__float_as_uint(v) & ~0x1FFFu)));
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(const __grid_constant__ Params P) {
    using T = Tile<BN>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + T::kOffBar);
    uint64_t* full = bars + 0;        // [kStages]
    uint64_t* empty = bars + 4;       // [kStages]
    uint64_t* acc_full = bars + 8;    // [2]
    uint64_t* acc_empty = bars + 10;  // [2]
    uint64_t* drain = bars + 12;
    uint64_t* lo_full = bars + 13;    // [kStages] A_lo of the stage written (or loaded)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 16);
    static_assert(13 + kStages <= 16, "barrier block");

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = P.tiles_m * P.tiles_n;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            ptx::mbar_init(&full[i], 1);
            ptx::mbar_init(&empty[i], 1);
            ptx::mbar_init(&lo_full[i], 4);
        }
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&acc_full[i], 1);
            ptx::mbar_init(&acc_empty[i], 8);
        }
        ptx::mbar_init(drain, 1);
        ptx::fence_mbar_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc(tmem_slot, T::kTmemCols);
        ptx::tmem_relinquish();
        ptx::tc_fence_before();
    }
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0, issued = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int m0 = (t / P.tiles_n) * kBM, tn = t % P.tiles_n, n0 = tn * BN;
                const int* tab = P.tab ? P.tab + tn * kTabStride : nullptr;
                const int nseg = tab ? __ldg(tab) : 1;
                for (int sg = 0; sg < nseg && ok; ++sg) {
                    int src = 0, acol = P.kbeg[tn], bcol = 0, nch = P.K / kBK;
                    if (tab) {
                        src = __ldg(tab + 2 + 4 * sg);
                        acol = __ldg(tab + 3 + 4 * sg);
                        bcol = __ldg(tab + 4 + 4 * sg);
                        nch = __ldg(tab + 5 + 4 * sg);
                    }
                    const Src& S = P.src[src];
                    const bool chip = P.lo_chip[src] != 0;
                    for (int kc = 0; kc < nch; ++kc, ++it) {
                        const int s = it % kStages;
                        if (!ptx::mbar_wait(&empty[s], ((it / kStages) & 1) ^ 1, kWaitLimit)) { ok = false; break; }
                        unsigned char* st = sm + s * T::kStageBytes;
                        ptx::mbar_expect_tx(&full[s], chip ? T::kStageBytes - kSlice : T::kStageBytes);
                        ptx::tma_load_2d(st, &S.a_hi, acol + kc * kBK, m0, &full[s]);
                        if (!chip) ptx::tma_load_2d(st + T::kOffAlo, &S.a_lo, acol + kc * kBK, m0, &full[s]);
                        ptx::tma_load_2d(st + T::kOffBhi, &S.b_hi, bcol + kc * kBK, n0, &full[s]);
                        ptx::tma_load_2d(st + T::kOffBlo, &S.b_lo, bcol + kc * kBK, n0, &full[s]);
                        issued = it + 1;
                    }
                }
            }
            if (!ok) {
                atomicOr(P.err, kErrTimeout);
                for (int i = max(0, issued - kStages); i < issued; ++i)
                    ptx::mbar_wait(&full[i % kStages], (i / kStages) & 1, kWaitLimit);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = ptx::idesc_tf32(kBM, BN);
            const uint64_t d0 = ptx::desc_sw128(ptx::smem_u32(sm));
            int it = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int nk = tile_chunks(P, t % P.tiles_n);
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % kStages, b = it & 1;
                    if (!ptx::mbar_wait(&acc_empty[b], ((it >> 1) & 1) ^ 1, kWaitLimit)) { ok = false; break; }
                    if (!ptx::mbar_wait(&full[s], (it / kStages) & 1, kWaitLimit)) { ok = false; break; }
                    if (!ptx::mbar_wait(&lo_full[s], (it / kStages) & 1, kWaitLimit)) { ok = false; break; }
                    ptx::tc_fence_after();
                    const uint32_t d = tmem + b * BN;
                    const uint64_t ds = d0 + (uint64_t)(s * (T::kStageBytes >> 4));
                    const uint64_t ahi = ds, alo = ds + (T::kOffAlo >> 4), bhi = ds + (T::kOffBhi >> 4),
                                   blo = ds + (T::kOffBlo >> 4);
#pragma unroll
                    for (int k = 0; k < 4; ++k) ptx::mma_tf32(d, ahi + 2 * k, blo + 2 * k, idesc, k > 0);
#pragma unroll
                    for (int k = 0; k < 4; ++k) ptx::mma_tf32(d, alo + 2 * k, bhi + 2 * k, idesc, 1);
#pragma unroll
                    for (int k = 0; k < 4; ++k) ptx::mma_tf32(d, ahi + 2 * k, bhi + 2 * k, idesc, 1);
                    ptx::mma_commit(&empty[s]);
                    ptx::mma_commit(&acc_full[b]);
                }
            }
            ptx::mma_commit(drain);
            if (!ptx::mbar_wait(drain, 0, kWaitLimit)) ok = false;
            if (!ok) atomicOr(P.err, kErrTimeout);
        }
    } else if (warp >= 10) {
        // A_lo converters: every stage passes through them in order; a stage whose
        // source has an A_lo array is only acknowledged
        const int ct = threadIdx.x - 320;  // 0..127
        int it = 0;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const int tn = t % P.tiles_n;
            const int* tab = P.tab ? P.tab + tn * kTabStride : nullptr;
            const int nseg = tab ? __ldg(tab) : 1;
            for (int sg = 0; sg < nseg && ok; ++sg) {
                const int src = tab ? __ldg(tab + 2 + 4 * sg) : 0;
                const int nch = tab ? __ldg(tab + 5 + 4 * sg) : P.K / kBK;
                const bool chip = P.lo_chip[src] != 0;
                for (int kc = 0; kc < nch; ++kc, ++it) {
                    const int s = it % kStages;
                    if (!ptx::mbar_wait(&full[s], (it / kStages) & 1, kWaitLimit)) { ok = false; break; }
                    if (chip) {
                        const float4* hi = reinterpret_cast<const float4*>(sm + s * T::kStageBytes);
                        float4* lo = reinterpret_cast<float4*>(sm + s * T::kStageBytes + T::kOffAlo);
#pragma unroll
                        for (int e = 0; e < (int)(kSlice / 16 / 128); ++e) {
                            const float4 v = hi[ct + 128 * e];
                            lo[ct + 128 * e] = make_float4(tf32_rem(v.x), tf32_rem(v.y), tf32_rem(v.z), tf32_rem(v.w));
                        }
                        ptx::fence_proxy_async_smem();
                    }
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&lo_full[s]);
                }
            }
        }
        if (!ok && lane == 0) atomicOr(P.err, kErrTimeout);
    } else {
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int r = 32 * q + lane;
        constexpr int WC = T::kWarpCols;
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16) + WC * h;
        float acc[WC];
        uint32_t u[16];
        int it = 0;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const int m0 = (t / P.tiles_n) * kBM, n0 = (t % P.tiles_n) * BN;
            const int nk = tile_chunks(P, t % P.tiles_n);
#pragma unroll
            for (int j = 0; j < WC; ++j) acc[j] = 0.f;
            for (int kc = 0; kc < nk; ++kc, ++it) {
                const int b = it & 1;
                if (!ptx::mbar_wait(&acc_full[b], (it >> 1) & 1, kWaitLimit)) { ok = false; break; }
                ptx::tc_fence_after();
#pragma unroll
                for (int j = 0; j < WC / 16; ++j) {
                    ptx::tmem_ld16(tl + b * BN + 16 * j, u);
                    ptx::tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 16; ++e) acc[16 * j + e] += __uint_as_float(u[e]);
                }
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&acc_empty[b]);
            }
            if (!ok) break;
            unsigned char* ys = sm + T::kOffY + (warp - 2) * 4096;
            for (int part = 0; part < 1 + P.has_lo; ++part) {
#pragma unroll
                for (int c = 0; c < WC / 32; ++c) {
                    // the previous box from this buffer has been read by its store
                    if (lane == 0) ptx::bulk_wait_group_read0();
                    __syncwarp();
#pragma unroll
                    for (int cc = 0; cc < 8; ++cc) {
                        float4 v = make_float4(acc[32 * c + 4 * cc], acc[32 * c + 4 * cc + 1],
                                               acc[32 * c + 4 * cc + 2], acc[32 * c + 4 * cc + 3]);
                        if (part) v = make_float4(tf32_rem(v.x), tf32_rem(v.y), tf32_rem(v.z), tf32_rem(v.w));
                        *reinterpret_cast<float4*>(ys + lane * 128 + ((cc ^ (lane & 7)) << 4)) = v;
                    }
                    ptx::fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        ptx::tma_store_2d(part ? &P.ylo_map : &P.y_map, n0 + WC * h + 32 * c, m0 + 32 * q, ys);
                        ptx::bulk_commit_group();
                    }
                }
            }
        }
        if (lane == 0) ptx::bulk_wait_group0();
        if (!ok && lane == 0) atomicOr(P.err, kErrTimeout);
    }

    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 1) ptx::tmem_dealloc(tmem, T::kTmemCols);
}

}  // namespace gemm

// ----------------------------------------------------------------- host

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn_g() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &f, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

// rows x cols FP32 row-major (leading dimension ld floats), box 32 x box_rows, 128-byte swizzle
static bool encode_rows(CUtensorMap* m, const float* base, int64_t rows, int64_t cols, int64_t ld,
                        int box_rows = 128) {
    auto fn = encode_fn_g();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
    cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

template <int BN>
static dctplus_status gemm_attr(int dev) {
    static bool attr[64] = {};
    if (!attr[dev & 63]) {
        DCTPLUS_CUDA_TRY(cudaFuncSetAttribute(gemm::k_gemm_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)gemm::Tile<BN>::kSmemBytes));
        attr[dev & 63] = true;
    }
    return DCTPLUS_OK;
}

static bool encode_src(gemm::Src* d, int* lo_chip, const GemmSrc& g, int M, int N, int bn) {
    *lo_chip = g.a_lo ? 0 : 1;
    return encode_rows(&d->a_hi, g.a_hi, M, g.Ka, g.lda) &&
           (!g.a_lo || encode_rows(&d->a_lo, g.a_lo, M, g.Ka, g.lda)) &&
           encode_rows(&d->b_hi, g.b_hi, N, g.Kb, g.ldb, bn) && encode_rows(&d->b_lo, g.b_lo, N, g.Kb, g.ldb, bn);
}

template <int BN>
static dctplus_status gemm_run_bn(gemm::Params& P, cudaStream_t s, int dev, const char* name, double bytes,
                                  double flops) {
    dctplus_status r = gemm_attr<BN>(dev);
    if (r != DCTPLUS_OK) return r;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = std::min(P.tiles_m * P.tiles_n, std::max(sms, 1));
    gemm::k_gemm_tc<BN><<<grid, gemm::kThreads, gemm::Tile<BN>::kSmemBytes, s>>>(P);
    note_launch(s, name, bytes, flops);
    DCTPLUS_CUDA_TRY(cudaGetLastError());
    return DCTPLUS_OK;
}

static dctplus_status gemm_run(gemm::Params& P, float* y, float* y_lo, int64_t ldy, int M, int N, int bn,
                               cudaStream_t s, int dev, const char* name, double bytes, double flops) {
    if ((ldy & 3) || !aligned16(y) || (y_lo && !aligned16(y_lo))) return DCTPLUS_ERR_UNSUPPORTED;
    if (!encode_rows(&P.y_map, y, M, N, ldy, 32)) return DCTPLUS_ERR_CUDA;
    if (y_lo && !encode_rows(&P.ylo_map, y_lo, M, N, ldy, 32)) return DCTPLUS_ERR_CUDA;
    P.has_lo = y_lo ? 1 : 0;
    P.M = M;
    P.N = N;
    P.tiles_m = (M + gemm::kBM - 1) / gemm::kBM;
    P.tiles_n = N / bn;
    P.err = device_error_word(dev);
    return bn == 64 ? gemm_run_bn<64>(P, s, dev, name, bytes, flops) : gemm_run_bn<128>(P, s, dev, name, bytes, flops);
}

// y[M x N] = (a_hi + a_lo)[:, band] (b_hi + b_lo)^T (a_lo null: formed on chip
// from a_hi, which then is the FP32 operand itself). A is [M x Ka]; B is
// [N x K]; output column tile tn uses A columns kbeg[tn] .. kbeg[tn] + K - 1
// (nullptr kbeg: all zero, the plain product with Ka = K). K % 32 == 0,
// N % 128 == 0, kbeg multiples of 4, 16-byte aligned bases, leading
// dimensions multiples of 4 floats. kbeg is per 128-column tile; without it a
// small product runs in 64-column tiles.
dctplus_status launch_gemm_tc_band(const float* a_hi, const float* a_lo, int64_t lda, int Ka,
                                   const float* b_hi, const float* b_lo, int64_t ldb, float* y,
                                   int64_t ldy, int M, int N, int K, const int* kbeg,
                                   cudaStream_t s, int dev) {
    if (M <= 0) return DCTPLUS_OK;
    if (K % gemm::kBK || N % kGemmBN || (lda & 3) || (ldb & 3) || N / kGemmBN > gemm::kMaxTilesN)
        return DCTPLUS_ERR_UNSUPPORTED;
    // 64-column tiles when even twice as many tiles fit in one wave over the SMs (small
    // products: dense n = 256, batch 4096, has 64 tiles of 128 x 128), else 128 columns
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t wide_tiles = (int64_t)((M + gemm::kBM - 1) / gemm::kBM) * (N / kGemmBN);
    const int bn = !kbeg && 2 * wide_tiles <= sms ? 64 : kGemmBN;
    gemm::Params P;
    memset(&P, 0, sizeof(P));
    GemmSrc g{a_hi, a_lo, lda, Ka, b_hi, b_lo, ldb, K};
    if (!encode_src(&P.src[0], &P.lo_chip[0], g, M, N, bn)) return DCTPLUS_ERR_CUDA;
    P.K = K;
    P.tab = nullptr;
    const int tiles_n = N / bn;
    for (int t = 0; t < tiles_n; ++t) {
        P.kbeg[t] = kbeg ? kbeg[t] : 0;
        if (P.kbeg[t] & 3) return DCTPLUS_ERR_UNSUPPORTED;
    }
    // A (and its stored remainder) read once over the columns the tiles use, B hi and lo
    // once, Y written
    const double bytes = (a_lo ? 8.0 : 4.0) * (double)M * std::min(Ka, K + (tiles_n - 1) * bn) +
                         8.0 * (double)N * K + 4.0 * (double)M * N;
    return gemm_run(P, y, nullptr, ldy, M, N, bn, s, dev, "k_gemm_tc", bytes, 6.0 * (double)M * N * K);
}

// The same product with a segment table (see the kernel's header): `tab` is a
// device array of kTabStride ints per column tile; `chunks_total` is the sum
// of all tiles' chunk counts and `a_cols` the A columns the tiles read in all
// (both only for the launch's work accounting). y_lo, if not null, receives
// the TF32 remainder of y.
dctplus_status launch_gemm_tc_segs(const GemmSrc* srcs, int nsrc, const int* tab, int64_t chunks_total,
                                   double a_cols, float* y, float* y_lo, int64_t ldy, int M, int N,
                                   cudaStream_t s, int dev, const char* name, int bn) {
    if (M <= 0) return DCTPLUS_OK;
    if ((bn != 64 && bn != 128) || nsrc < 1 || nsrc > gemm::kMaxSrc || !tab || N % bn ||
        N / bn > gemm::kMaxTilesN)
        return DCTPLUS_ERR_UNSUPPORTED;
    gemm::Params P;
    memset(&P, 0, sizeof(P));
    double b_bytes = 0.0, a_bytes_per_col = 0.0;
    for (int i = 0; i < nsrc; ++i) {
        const GemmSrc& g = srcs[i];
        if ((g.lda & 3) || (g.ldb & 3) || !aligned16(g.a_hi) || (g.a_lo && !aligned16(g.a_lo)) ||
            !aligned16(g.b_hi) || !aligned16(g.b_lo))
            return DCTPLUS_ERR_UNSUPPORTED;
        if (!encode_src(&P.src[i], &P.lo_chip[i], g, M, N, bn)) return DCTPLUS_ERR_CUDA;
        b_bytes += 8.0 * (double)N * g.Kb;
        a_bytes_per_col += g.a_lo ? 8.0 : 4.0;
    }
    P.tab = tab;
    P.K = 0;
    const double flops = 6.0 * (double)M * bn * gemm::kBK * (double)chunks_total;
    const double bytes = a_bytes_per_col / nsrc * (double)M * a_cols + b_bytes + (y_lo ? 8.0 : 4.0) * (double)M * N;
    return gemm_run(P, y, y_lo, ldy, M, N, bn, s, dev, name, bytes, flops);
}

}  // namespace dctplus

namespace dctplus {

dctplus_status launch_gemm_tc(const float* a_hi, const float* a_lo, int64_t lda, const float* b_hi,
                              const float* b_lo, int64_t ldb, float* y, int64_t ldy, int M, int N,
                              int K, cudaStream_t s, int dev) {
    return launch_gemm_tc_band(a_hi, a_lo, lda, K, b_hi, b_lo, ldb, y, ldy, M, N, K, nullptr, s, dev);
}

}  // namespace dctplus
