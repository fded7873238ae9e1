// Tensor-core (tcgen05) forward transform for n in {4, 8, 16, 32, 64}.
//
// Data layout: the signals of a segment are contiguous, so the segment is
// also a row-major matrix of "packed rows" of 64 samples, each holding 64/n
// whole signals. The DCT-II of every signal in a packed row is one product
// with the block-diagonal I_{64/n} (x) U^T, and the Cauchy step (Algorithm 1
// steps 2-8, with a and z folded into W = X^T U, Theorem 3.1) one product with
// I_{64/n} (x) W. Per tile of 128 packed rows:
//   S = X B1^T,  Y = S B2^T      (M = 128, N = 64, K = 64)
// on the tensor cores in kind::tf32 with split operands: every FP32 operand
// is a sum hi + lo of two TF32 numbers and each product takes the three terms
// hi*hi + hi*lo + lo*hi, accumulated in FP32 in tensor memory (TMEM).
//
// Roles (192 threads, one persistent CTA per SM):
//   warp 0      TMA producer: x tiles into a 2-stage ring (128-byte swizzle)
//   warp 1      TMEM owner and MMA issuer (one thread)
//   warps 2..5  epilogue: x_lo = x - tf32(x); S from TMEM split into hi/lo
//               tiles; Y from TMEM staged in shared memory and stored by TMA.
// Every mbarrier wait is bounded; a wait that runs out sets the device error
// word and the CTA winds down (no trap, TMEM released).
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace dctplus {

constexpr int kTcMaxSeg = 40;
constexpr int kTcRows = 128;
constexpr uint32_t kWaitLimit = 1u << 22;

// shared-memory map (offsets from a 1024-byte aligned base)
constexpr uint32_t kImgBytes = 16384;               // one 64x64 TF32 operand image
constexpr uint32_t kOffB = 0;                       // B1 hi, B1 lo, B2 hi, B2 lo
constexpr uint32_t kOffX = 4 * kImgBytes;           // 2 stages x 32 KB
constexpr uint32_t kTileBytes = kTcRows * 64 * 4;   // 32 KB
constexpr uint32_t kOffXlo = kOffX + 2 * kTileBytes;
constexpr uint32_t kOffShi = kOffXlo + kTileBytes;
constexpr uint32_t kOffSlo = kOffShi + kTileBytes;
constexpr uint32_t kOffBar = kOffSlo + kTileBytes;
constexpr uint32_t kSmemBytes = kOffBar + 256 + 1024;  // + barriers + alignment slack

struct TcSeg {
    int tile_start;  // first tile index of the segment in this launch
    int rows64;      // packed rows in the segment
};

struct TcParams {
    CUtensorMap xmap[kTcMaxSeg];
    CUtensorMap ymap[kTcMaxSeg];
    const float* images[kTcMaxSeg];  // 4 operand images of the segment's plan (64 KB)
    TcSeg seg[kTcMaxSeg];
    int nseg;
    int ntiles;
    unsigned* err;
};

__device__ __forceinline__ int find_seg(const TcParams& P, int tile) {
    int s = 0;
    for (int i = 1; i < P.nseg; ++i)
        if (P.seg[i].tile_start <= tile) s = i;
    return s;
}

// thread (row r) writes 64 FP32 values in the 128-byte-swizzled K-major layout
__device__ __forceinline__ void store_row_sw128(unsigned char* base, int r, const float* v) {
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        int kb = c >> 3, cc = c & 7;
        float4 q = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
        *reinterpret_cast<float4*>(base + kb * kTileBytes / 2 + r * 128 + ((cc ^ (r & 7)) << 4)) = q;
    }
}

__device__ __forceinline__ void load_tmem_row64(uint32_t taddr, float* v) {
    uint32_t r[16];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        ptx::tmem_ld16(taddr + 16 * j, r);
        ptx::tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 16; ++e) v[16 * j + e] = __uint_as_float(r[e]);
    }
}

__global__ void __launch_bounds__(192, 1) k_small_tc(const __grid_constant__ TcParams P) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* Bimg = sm + kOffB;
    unsigned char* xbuf = sm + kOffX;
    unsigned char* xlo = sm + kOffXlo;
    unsigned char* Shi = sm + kOffShi;
    unsigned char* Slo = sm + kOffSlo;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kOffBar);
    uint64_t* x_full = bars + 0;      // [2]
    uint64_t* x_empty = bars + 2;     // [2]
    uint64_t* d1_full = bars + 4;     // [2]
    uint64_t* d2_full = bars + 6;     // [2]
    uint64_t* tmem_empty = bars + 8;  // [2]
    uint64_t* xlo_full = bars + 10;
    uint64_t* s_full = bars + 11;
    uint64_t* b_full = bars + 12;
    uint64_t* drain = bars + 13;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 16);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // contiguous chunk of tiles for this CTA
    const int G = gridDim.x, c = blockIdx.x;
    const int base = P.ntiles / G, rem = P.ntiles % G;
    const int t0 = c * base + min(c, rem);
    const int count = base + (c < rem ? 1 : 0);

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&x_full[i], 1);
            ptx::mbar_init(&x_empty[i], 1);
            ptx::mbar_init(&d1_full[i], 1);
            ptx::mbar_init(&d2_full[i], 1);
            ptx::mbar_init(&tmem_empty[i], 4);
        }
        ptx::mbar_init(xlo_full, 4);
        ptx::mbar_init(s_full, 4);
        ptx::mbar_init(b_full, 1);
        ptx::mbar_init(drain, 1);
        ptx::fence_mbar_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc(tmem_slot, 256);
        ptx::tmem_relinquish();
        ptx::tc_fence_before();
    }
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < count && ok; ++i) {
                const int tile = t0 + i, s = i & 1;
                if (!ptx::mbar_wait(&x_empty[s], ((i >> 1) & 1) ^ 1, kWaitLimit)) { ok = false; break; }
                const int sg = find_seg(P, tile);
                const int row0 = (tile - P.seg[sg].tile_start) * kTcRows;
                ptx::mbar_expect_tx(&x_full[s], kTileBytes);
                ptx::tma_load_2d(xbuf + s * kTileBytes, &P.xmap[sg], 0, row0, &x_full[s]);
                ptx::tma_load_2d(xbuf + s * kTileBytes + kTileBytes / 2, &P.xmap[sg], 32, row0, &x_full[s]);
                issued = i + 1;
            }
            if (!ok) {
                atomicOr(P.err, kErrTimeout);
                // let the loads already in flight land before the CTA exits
                for (int i = max(0, issued - 2); i < issued; ++i)
                    ptx::mbar_wait(&x_full[i & 1], (i >> 1) & 1, kWaitLimit);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = ptx::idesc_tf32(128, 64);
            const uint32_t sB = ptx::smem_u32(Bimg), sX = ptx::smem_u32(xbuf),
                           sXlo = ptx::smem_u32(xlo), sShi = ptx::smem_u32(Shi),
                           sSlo = ptx::smem_u32(Slo);
            const float* cur = nullptr;
            uint32_t nb = 0, nd = 0;
            for (int i = 0; i < count && ok; ++i) {
                const int tile = t0 + i, s = i & 1, b = i & 1;
                const int sg = find_seg(P, tile);
                if (P.images[sg] != cur) {
                    if (i > 0) {  // all MMAs reading the old operands must finish first
                        ptx::mma_commit(drain);
                        if (!ptx::mbar_wait(drain, nd & 1, kWaitLimit)) { ok = false; break; }
                        ++nd;
                    }
                    ptx::mbar_expect_tx(b_full, 4 * kImgBytes);
                    ptx::bulk_load(Bimg, P.images[sg], 4 * kImgBytes, b_full);
                    if (!ptx::mbar_wait(b_full, nb & 1, kWaitLimit)) { ok = false; break; }
                    ++nb;
                    cur = P.images[sg];
                }
                if (!ptx::mbar_wait(&tmem_empty[b], ((i >> 1) & 1) ^ 1, kWaitLimit)) { ok = false; break; }
                if (!ptx::mbar_wait(xlo_full, i & 1, kWaitLimit)) { ok = false; break; }
                ptx::tc_fence_after();
                const uint32_t d1 = tmem + b * 128, d2 = d1 + 64;
                const uint32_t sA = sX + s * kTileBytes;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t ka = (k >> 2) * (kTileBytes / 2) + (k & 3) * 32;
                    const uint32_t kbb = (k >> 2) * (kImgBytes / 2) + (k & 3) * 32;
                    const uint64_t ah = ptx::desc_sw128(sA + ka), al = ptx::desc_sw128(sXlo + ka);
                    const uint64_t bh = ptx::desc_sw128(sB + 0 * kImgBytes + kbb);
                    const uint64_t bl = ptx::desc_sw128(sB + 1 * kImgBytes + kbb);
                    ptx::mma_tf32(d1, ah, bh, idesc, k > 0);
                    ptx::mma_tf32(d1, ah, bl, idesc, 1);
                    ptx::mma_tf32(d1, al, bh, idesc, 1);
                }
                ptx::mma_commit(&x_empty[s]);
                ptx::mma_commit(&d1_full[b]);
                if (!ptx::mbar_wait(s_full, i & 1, kWaitLimit)) { ok = false; break; }
                ptx::tc_fence_after();
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t ka = (k >> 2) * (kTileBytes / 2) + (k & 3) * 32;
                    const uint32_t kbb = (k >> 2) * (kImgBytes / 2) + (k & 3) * 32;
                    const uint64_t ah = ptx::desc_sw128(sShi + ka), al = ptx::desc_sw128(sSlo + ka);
                    const uint64_t bh = ptx::desc_sw128(sB + 2 * kImgBytes + kbb);
                    const uint64_t bl = ptx::desc_sw128(sB + 3 * kImgBytes + kbb);
                    ptx::mma_tf32(d2, ah, bh, idesc, k > 0);
                    ptx::mma_tf32(d2, ah, bl, idesc, 1);
                    ptx::mma_tf32(d2, al, bh, idesc, 1);
                }
                ptx::mma_commit(&d2_full[b]);
            }
            // every MMA done before TMEM is released
            ptx::mma_commit(drain);
            if (!ptx::mbar_wait(drain, nd & 1, kWaitLimit)) ok = false;
            if (!ok) atomicOr(P.err, kErrTimeout);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int etid = threadIdx.x - 64;  // 0..127
        const int q = warp & 3;             // TMEM lane quarter this warp may access
        const int r = 32 * q + lane;        // tile row = TMEM lane
        const uint32_t lane_off = (uint32_t)(32 * q) << 16;
        float v[64];

        auto conv = [&](int i) -> bool {
            const int s = i & 1;
            if (!ptx::mbar_wait(&x_full[s], (i >> 1) & 1, kWaitLimit)) return false;
            const unsigned char* src = xbuf + s * kTileBytes;
            for (int off = etid * 16; off < (int)kTileBytes; off += 128 * 16) {
                float4 a = *reinterpret_cast<const float4*>(src + off);
                float4 lo;
                // the MMA reads x truncated to TF32; x_lo carries the rest, rounded to TF32
                lo.x = ptx::tf32_round(a.x - __uint_as_float(__float_as_uint(a.x) & ~0x1FFFu));
                lo.y = ptx::tf32_round(a.y - __uint_as_float(__float_as_uint(a.y) & ~0x1FFFu));
                lo.z = ptx::tf32_round(a.z - __uint_as_float(__float_as_uint(a.z) & ~0x1FFFu));
                lo.w = ptx::tf32_round(a.w - __uint_as_float(__float_as_uint(a.w) & ~0x1FFFu));
                *reinterpret_cast<float4*>(xlo + off) = lo;
            }
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(xlo_full);
            return true;
        };

        if (count > 0) ok = conv(0);
        for (int i = 0; i < count && ok; ++i) {
            const int tile = t0 + i, b = i & 1;
            const int sg = find_seg(P, tile);
            const int row0 = (tile - P.seg[sg].tile_start) * kTcRows;
            // S = D1: split into TF32 hi / lo operand tiles
            if (!ptx::mbar_wait(&d1_full[b], (i >> 1) & 1, kWaitLimit)) { ok = false; break; }
            ptx::tc_fence_after();
            if (etid == 0) ptx::bulk_wait_group_read0();  // previous Y store has read its staging
            ptx::named_bar_sync(1, 128);
            load_tmem_row64(tmem + lane_off + b * 128, v);
            {
                float lo[64];
#pragma unroll
                for (int e = 0; e < 64; ++e) {
                    float h = ptx::tf32_round(v[e]);
                    lo[e] = ptx::tf32_round(v[e] - h);
                    v[e] = h;
                }
                store_row_sw128(Shi, r, v);
                store_row_sw128(Slo, r, lo);
            }
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(s_full);
            if (i + 1 < count && !conv(i + 1)) { ok = false; break; }
            // Y = D2: stage in shared memory, store with TMA
            if (!ptx::mbar_wait(&d2_full[b], (i >> 1) & 1, kWaitLimit)) { ok = false; break; }
            ptx::tc_fence_after();
            load_tmem_row64(tmem + lane_off + b * 128 + 64, v);
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&tmem_empty[b]);
            store_row_sw128(Shi, r, v);
            ptx::fence_proxy_async_smem();
            ptx::named_bar_sync(1, 128);
            if (etid == 0) {
                ptx::tma_store_2d(&P.ymap[sg], 0, row0, Shi);
                ptx::tma_store_2d(&P.ymap[sg], 32, row0, Shi + kTileBytes / 2);
                ptx::bulk_commit_group();
            }
        }
        if (etid == 0) ptx::bulk_wait_group0();
        if (!ok && lane == 0) atomicOr(P.err, kErrTimeout);
    }

    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 1) ptx::tmem_dealloc(tmem, 256);
}

// --------------------------------------------------------- operand images

// The four 64x64 B operands (N rows x K, K-major) of a plan, block diagonal
// over 64/n copies: B1 = I (x) U^T, B2 = I (x) W; each split into TF32 hi and
// lo, written in the 128-byte-swizzled layout the MMA reads from shared memory.
__global__ void k_tc_images(int n, const double* ct64, const double* w64, float* img) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;  // r * 64 + k
    if (idx >= 64 * 64) return;
    int r = idx / 64, k = idx % 64;
    bool same = (r / n) == (k / n);
    double b1 = same ? ct64[(r % n) * n + (k % n)] : 0.0;
    double b2 = same ? w64[(r % n) * n + (k % n)] : 0.0;
    int kb = k / 32, c = (k % 32) / 4, e = k % 4;
    int off = (kb * 8192 + r * 128 + ((c ^ (r & 7)) << 4) + e * 4) / 4;  // in floats
    float h1 = ptx::tf32_round((float)b1);
    float l1 = ptx::tf32_round((float)(b1 - (double)h1));
    float h2 = ptx::tf32_round((float)b2);
    float l2 = ptx::tf32_round((float)(b2 - (double)h2));
    img[0 * 4096 + off] = h1;
    img[1 * 4096 + off] = l1;
    img[2 * 4096 + off] = h2;
    img[3 * 4096 + off] = l2;
}

static bool tc_size(int n) { return n == 4 || n == 8 || n == 16 || n == 32 || n == 64; }

dctplus_status setup_small_tc(dctplus_plan_t p) {
    if (!tc_size(p->n) || !p->d_ct64 || !p->d_w64) return DCTPLUS_OK;
    DCTPLUS_CUDA_TRY(cudaMalloc((void**)&p->tc.images, 4 * kImgBytes));
    k_tc_images<<<16, 256>>>(p->n, p->d_ct64, p->d_w64, p->tc.images);
    count_launch();
    DCTPLUS_CUDA_TRY(cudaGetLastError());
    return DCTPLUS_OK;
}

bool small_tc_capable(dctplus_plan_t p) { return tc_size(p->n) && p->tc.images != nullptr; }

// ------------------------------------------------------------- host launch

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// [rows64 x 64] FP32 row-major at `base`, box 32 x 128, 128-byte swizzle.
static bool encode_map(CUtensorMap* m, const float* base, int64_t rows64) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {64, (cuuint64_t)rows64};
    cuuint64_t strides[1] = {256};
    cuuint32_t box[2] = {32, (cuuint32_t)kTcRows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

static int sm_count_tc(int dev) {
    static int cached[64] = {0};
    int d = dev & 63;
    if (!cached[d]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[d] = v > 0 ? v : 148;
    }
    return cached[d];
}

// Launches the tensor-core kernel over packed-row segments. x/y of every
// segment must be 16-byte aligned; rows64 = number of full 64-sample rows.
dctplus_status launch_tc_segments(const std::vector<TcSegHost>& segs, cudaStream_t s, int dev) {
    static bool attr[64] = {};
    if (!attr[dev & 63]) {
        DCTPLUS_CUDA_TRY(cudaFuncSetAttribute(k_small_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
        attr[dev & 63] = true;
    }
    size_t i0 = 0;
    while (i0 < segs.size()) {
        TcParams P;
        memset(&P, 0, sizeof(P));
        int tiles = 0, ns = 0;
        for (; i0 < segs.size() && ns < kTcMaxSeg; ++i0) {
            const TcSegHost& g = segs[i0];
            if (g.rows64 <= 0) continue;
            if (!encode_map(&P.xmap[ns], g.x, g.rows64) || !encode_map(&P.ymap[ns], g.y, g.rows64))
                return DCTPLUS_ERR_CUDA;
            P.images[ns] = g.plan->tc.images;
            P.seg[ns].tile_start = tiles;
            P.seg[ns].rows64 = (int)g.rows64;
            tiles += (int)((g.rows64 + kTcRows - 1) / kTcRows);
            ++ns;
        }
        if (ns == 0) continue;
        P.nseg = ns;
        P.ntiles = tiles;
        P.err = device_error_word(dev);
        int grid = std::min(tiles, sm_count_tc(dev));
        k_small_tc<<<grid, 192, kSmemBytes, s>>>(P);
        count_launch();
        DCTPLUS_CUDA_TRY(cudaGetLastError());
    }
    return DCTPLUS_OK;
}

static bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

bool small_tc_available(dctplus_plan_t p) { return small_tc_capable(p); }

// One plan: the packed body goes to the tensor cores, the < 64/n leftover
// signals to the CUDA-core kernel.
dctplus_status launch_small_tc(dctplus_plan_t p, const float* x, int64_t ldx, float* y,
                               int64_t ldy, int64_t batch, cudaStream_t s) {
    const int n = p->n;
    if (!small_tc_capable(p) || ldx != n || ldy != n || !aligned16(x) || !aligned16(y))
        return launch_small_simt_f32(p, x, ldx, y, ldy, batch, s);
    const int64_t rows64 = batch * n / 64;
    const int64_t body = rows64 * 64 / n;  // signals in full packed rows
    if (rows64 > 0) {
        std::vector<TcSegHost> segs = {{p, x, y, rows64}};
        dctplus_status st = launch_tc_segments(segs, s, p->device);
        if (st != DCTPLUS_OK) return st;
    }
    if (batch > body)
        return launch_small_simt_f32(p, x + body * n, n, y + body * n, n, batch - body, s);
    return DCTPLUS_OK;
}

}  // namespace dctplus
