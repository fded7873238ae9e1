// Tensor-core (tcgen05) forward transform for n in {4, 8, 16, 32, 64}.
//
// Data layout: the signals of a segment are contiguous, so the segment is
// also a row-major matrix of "packed rows" of 64 samples, each holding 64/n
// whole signals. The DCT-II of every signal in a packed row is one product
// with the block-diagonal I_{64/n} (x) U^T, and the Cauchy step (Algorithm 1
// steps 2-8, with a and z folded into W = X^T U, Theorem 3.1) one product with
// I_{64/n} (x) W. Per tile of 128 packed rows:
//   S = X B1^T,  Y = S B2^T      (M = 128, N = 64, K = 64)
// on the tensor cores in kind::tf32 with split operands: an FP32 operand is
// hi + lo with hi, lo TF32, and a product takes hi*hi + hi*lo + lo*hi,
// accumulated in FP32 in tensor memory (TMEM). For x and S the hi part is the
// FP32 value itself, which the MMA reads truncated to TF32 (S straight from
// TMEM), and lo = rn_tf32(v - trunc_tf32(v)); for the plan's matrices hi and
// lo are both rounded. The plan's hi and lo are stacked into one 128-row B
// operand, so hi*[B_hi; B_lo] is a single N = 128 MMA per K step (an N = 64
// MMA runs at about half the rate of an N = 128 one): it writes the main
// term hi*B_hi into columns 0..63 of a 128-column accumulator and hi*B_lo
// into columns 64..127, where the N = 64 MMA lo*B_hi then accumulates. The
// two halves are added in FP32 (round to nearest) by the warps that read
// them: for S by the S_lo warps, which write S and S_lo back in place, for Y
// by the Y warps.
//
// Pipeline: x_lo is double buffered, so x_lo of tile t+1 is formed while the
// DCT GEMM of tile t runs, and so is the DCT accumulator (which then holds S
// and S_lo), so the DCT GEMM of tile t+1 runs while tile t's S is split.
// Shared memory holds the plan's operand images and a 4-stage ring of x tiles
// (a stage is held from its TMA load until the DCT GEMM has read it, so the
// ring depth bounds the loads in flight); all A-side operands the epilogue
// forms live in TMEM.
// Roles (512 threads, one persistent CTA per SM):
//   warp 0       TMA producer: x tiles into a 4-stage ring (128-byte swizzle)
//   warp 1       TMEM owner; one thread issues the DCT GEMMs and loads the
//                DCT operand images (they depend on n only)
//   warp 15      one thread issues the Cauchy GEMMs and loads the W images
//   warps 2..9   x_lo and S_lo into TMEM; two warps per TMEM lane quarter,
//                32 columns each
//   warps 10..13 Y (TMEM) through registers into a shared-memory staging
//                tile (128-byte swizzle), written out by TMA. Stores of rows
//                straight from registers would touch 32 rows per instruction:
//                their many small L2 writes queue in the load/store unit ahead
//                of the shared-memory loads of the x_lo and S_lo warps.
//   warp 14      the < 64/n signals of each segment that do not fill a packed
//                row, on CUDA cores from the plan's FP32 tables
// The two GEMM streams are issued from two threads, so that one thread's
// barrier waits do not leave the tensor pipe idle while the other has work;
// each thread's commits track only its own MMAs, and every buffer two GEMMs
// share is handed over through an mbarrier. At a segment boundary each
// thread drains only its own GEMMs before replacing its half of the operand
// images (the DCT half only when n changes), so the other GEMM stream keeps
// the tensor pipe busy during the reload.
// TMEM columns: D1[2] 0..255 (128 each: S | S_lo after the split), D2 256..383,
// x_lo[2] 384..511. (The Y accumulator D2 is single buffered: its reader
// drains it right after each Cauchy GEMM.)
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
constexpr int kStages = 4;
constexpr int kTcThreads = 512;
constexpr uint32_t kWaitLimit = 1u << 22;

// shared-memory map (offsets from a 1024-byte aligned base)
constexpr uint32_t kImgBytes = 16384;               // one 64x64 TF32 operand (hi or lo)
constexpr uint32_t kTileBytes = kTcRows * 64 * 4;   // 32 KB
constexpr uint32_t kOffB = 0;                       // [B1 hi; B1 lo], [B2 hi; B2 lo]
constexpr uint32_t kOffX = 4 * kImgBytes;           // kStages x 32 KB
constexpr uint32_t kOffY = kOffX + kStages * kTileBytes;  // Y staging tile
constexpr uint32_t kOffBar = kOffY + kTileBytes;
constexpr uint32_t kSmemBytes = kOffBar + 256 + 1024;  // + barriers + alignment slack

// TMEM column map
constexpr uint32_t kColD1 = 0, kColD2 = 256, kColXlo = 384;

struct TcSeg {
    int tile_start;     // first tile index of the segment in this launch
    int rows64;         // packed rows in the segment
    int n;
    int tail;           // signals after the last full packed row
    const float* xt;    // first tail signal
    float* yt;
    float* y;           // first packed row of the segment's output
    const float* ct;    // n x n FP32 U^T
    const float* w;     // n x n FP32 W
};

struct TcParams {
    CUtensorMap xmap[kTcMaxSeg];
    CUtensorMap ymap[kTcMaxSeg];
    const float* images[kTcMaxSeg];  // the segment's plan's operand images (64 KB)
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

// Segment of a non-decreasing sequence of tiles: one search, then O(1) steps
// (each role walks its own contiguous tile range in order).
struct SegCursor {
    int s;
    __device__ __forceinline__ SegCursor(const TcParams& P, int tile) : s(find_seg(P, tile)) {}
    __device__ __forceinline__ int at(const TcParams& P, int tile) {
        while (s + 1 < P.nseg && P.seg[s + 1].tile_start <= tile) ++s;
        return s;
    }
};

// byte offset of the 16-byte chunk c (0..15) of row r in a 128-row tile in the
// 128-byte-swizzled K-major layout (K-block c / 8)
__device__ __forceinline__ uint32_t sw128_off(int r, int c) {
    return (uint32_t)((c >> 3) * (kTileBytes / 2) + r * 128 + (((c & 7) ^ (r & 7)) << 4));
}

// the MMA reads v truncated to TF32; this is the rest, rounded to TF32
__device__ __forceinline__ uint32_t lo_tf32(float v) {
    return ptx::cvt_rna_tf32(v - __uint_as_float(__float_as_uint(v) & ~0x1FFFu));
}

__global__ void __launch_bounds__(kTcThreads, 1) k_small_tc(const __grid_constant__ TcParams P) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* Bimg = sm + kOffB;
    unsigned char* xbuf = sm + kOffX;
    unsigned char* ybuf = sm + kOffY;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kOffBar);
    uint64_t* x_full = bars + 0;                // [kStages]
    uint64_t* x_empty = bars + kStages;         // [kStages]
    uint64_t* d1_full = bars + 2 * kStages;     // [2] DCT GEMM of the tile in D1[d] done
    uint64_t* d1_free = d1_full + 2;            // [2] Cauchy GEMM that read D1[d] done
    uint64_t* s_full = d1_free + 2;             // [2] S and S_lo written into D1[d]
    uint64_t* xlo_full = s_full + 2;            // [2] x_lo[b] written
    uint64_t* d2_full = xlo_full + 2;           // Cauchy GEMM of the tile in D2 done
    uint64_t* d2_empty = d2_full + 1;           // D2 read out
    uint64_t* b_full = d2_empty + 1;
    uint64_t* drain = b_full + 1;               // DCT GEMM issuer's own MMAs done
    uint64_t* drain2 = drain + 1;               // Cauchy GEMM issuer's own MMAs done
    uint64_t* b2_full = drain2 + 1;             // W images loaded
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(b2_full + 1);
    static_assert(8 * (2 * kStages + 15) <= 256, "barrier block");

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // contiguous chunk of tiles for this CTA
    const int G = gridDim.x, c = blockIdx.x;
    const int base = P.ntiles / G, rem = P.ntiles % G;
    const int t0 = c * base + min(c, rem);
    const int count = base + (c < rem ? 1 : 0);

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            ptx::mbar_init(&x_full[i], 1);
            ptx::mbar_init(&x_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&d1_full[i], 1);
            ptx::mbar_init(&d1_free[i], 1);
            ptx::mbar_init(&s_full[i], 8);
            ptx::mbar_init(&xlo_full[i], 8);
        }
        ptx::mbar_init(d2_full, 1);
        ptx::mbar_init(d2_empty, 4);
        ptx::mbar_init(b_full, 1);
        ptx::mbar_init(drain, 1);
        ptx::mbar_init(drain2, 1);
        ptx::mbar_init(b2_full, 1);
        ptx::fence_mbar_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc(tmem_slot, 512);
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
            SegCursor cursor(P, t0);
            for (int i = 0; i < count && ok; ++i) {
                const int tile = t0 + i, s = i % kStages;
                if (!ptx::mbar_wait(&x_empty[s], ((i / kStages) & 1) ^ 1, kWaitLimit)) { ok = false; break; }
                const int sg = cursor.at(P, tile);
                const int row0 = (tile - P.seg[sg].tile_start) * kTcRows;
                ptx::mbar_expect_tx(&x_full[s], kTileBytes);
                ptx::tma_load_2d(xbuf + s * kTileBytes, &P.xmap[sg], 0, row0, &x_full[s]);
                ptx::tma_load_2d(xbuf + s * kTileBytes + kTileBytes / 2, &P.xmap[sg], 32, row0, &x_full[s]);
                issued = i + 1;
            }
            if (!ok) {
                atomicOr(P.err, kErrTimeout);
                // let the loads already in flight land before the CTA exits
                for (int i = max(0, issued - kStages); i < issued; ++i)
                    ptx::mbar_wait(&x_full[i % kStages], (i / kStages) & 1, kWaitLimit);
            }
        }
    } else if (warp == 1 || warp == 15) {
        // ---------------------------------------------------------- MMA issuers
        if (lane == 0) {
            constexpr uint32_t idesc64 = ptx::idesc_tf32(128, 64);
            constexpr uint32_t idesc128 = ptx::idesc_tf32(128, 128);
            // descriptors of the operand bases; a K step or another stage or
            // matrix only moves the start address (field in 16-byte units)
            const uint64_t dB0 = ptx::desc_sw128(ptx::smem_u32(Bimg));
            // K step k = 8 TF32 = 32 bytes inside a 128-byte swizzle row; K
            // block k / 4 is the next 128 rows (16 KB) of an A tile or a
            // stacked [hi; lo] B operand, whose first 64 rows are hi
            auto k16 = [](int k) -> uint64_t { return (uint64_t)((k >> 2) * (kTileBytes / 32) + (k & 3) * 2); };
            constexpr uint64_t kB2 = (2 * kImgBytes) >> 4;   // [B2 hi; B2 lo]
            if (warp == 1) {
                // DCT GEMMs, S = X B1^T, corrections first and hi*hi last
                const uint64_t dX0 = ptx::desc_sw128(ptx::smem_u32(xbuf));
                int cur_n = 0;
                uint32_t nb = 0, nd = 0;
                SegCursor cursor(P, t0);
                for (int i = 0; i < count && ok; ++i) {
                    const int sg = cursor.at(P, t0 + i);
                    if (P.seg[sg].n != cur_n) {
                        // B1 = I (x) U^T depends on n only; the old one is free once
                        // this thread's own MMAs are done
                        if (cur_n) {
                            ptx::mma_commit(drain);
                            if (!ptx::mbar_wait(drain, nd & 1, kWaitLimit)) { ok = false; break; }
                            ++nd;
                        }
                        ptx::mbar_expect_tx(b_full, 2 * kImgBytes);
                        ptx::bulk_load(Bimg, P.images[sg], 2 * kImgBytes, b_full);
                        if (!ptx::mbar_wait(b_full, nb & 1, kWaitLimit)) { ok = false; break; }
                        ++nb;
                        cur_n = P.seg[sg].n;
                    }
                    const int st = i % kStages, d = i & 1;
                    // D1[d] held S and S_lo of tile i - 2 for its Cauchy GEMM
                    if (i >= 2 && !ptx::mbar_wait(&d1_free[d], ((i >> 1) - 1) & 1, kWaitLimit)) { ok = false; break; }
                    if (!ptx::mbar_wait(&xlo_full[i & 1], (i >> 1) & 1, kWaitLimit)) { ok = false; break; }
                    ptx::tc_fence_after();
                    const uint32_t d1 = tmem + kColD1 + d * 128;
                    const uint64_t dA = dX0 + (uint64_t)(st * (kTileBytes >> 4));
                    const uint32_t xl = tmem + kColXlo + (i & 1) * 64;
                    // x_hi [B1 hi; B1 lo]^T into both halves, then x_lo B1_hi^T into the second
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        ptx::mma_tf32(d1, dA + k16(k), dB0 + k16(k), idesc128, k > 0);
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        ptx::mma_tf32_ts(d1 + 64, xl + 8 * k, dB0 + k16(k), idesc64, 1);
                    ptx::mma_commit(&x_empty[st]);
                    ptx::mma_commit(&d1_full[d]);
                }
                // every MMA of this thread done before TMEM is released
                ptx::mma_commit(drain);
                if (!ptx::mbar_wait(drain, nd & 1, kWaitLimit)) ok = false;
            } else {
                // Cauchy GEMMs, Y = S B2^T: S hi straight from the D1 accumulator,
                // S_lo from TMEM
                const float* cur = nullptr;
                uint32_t nb2 = 0, nd2 = 0;
                bool pending = false;  // a W image copy not yet waited for
                SegCursor cursor(P, t0);
                for (int i = 0; i < count && ok; ++i) {
                    const int bf = i & 1;
                    const float* img = P.images[cursor.at(P, t0 + i)];
                    const bool load = img != cur;
                    if (load) {
                        // the old W images are free once this thread's own MMAs are done;
                        // the copy overlaps the wait for tile i's S_lo
                        if (cur) {
                            ptx::mma_commit(drain2);
                            if (!ptx::mbar_wait(drain2, nd2 & 1, kWaitLimit)) { ok = false; break; }
                            ++nd2;
                        }
                        ptx::mbar_expect_tx(b2_full, 2 * kImgBytes);
                        ptx::bulk_load(Bimg + 2 * kImgBytes, img + 2 * (kImgBytes / 4), 2 * kImgBytes, b2_full);
                        pending = true;
                        cur = img;
                    }
                    if (!ptx::mbar_wait(&s_full[bf], (i >> 1) & 1, kWaitLimit)) { ok = false; break; }
                    if (!ptx::mbar_wait(d2_empty, (i & 1) ^ 1, kWaitLimit)) { ok = false; break; }
                    if (load) {
                        if (!ptx::mbar_wait(b2_full, nb2 & 1, kWaitLimit)) { ok = false; break; }
                        ++nb2;
                        pending = false;
                    }
                    ptx::tc_fence_after();
                    const uint32_t d2 = tmem + kColD2;
                    const uint32_t sh = tmem + kColD1 + bf * 128, sl = sh + 64;
                    // S [B2 hi; B2 lo]^T into both halves, then S_lo B2_hi^T into the second
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        ptx::mma_tf32_ts(d2, sh + 8 * k, dB0 + kB2 + k16(k), idesc128, k > 0);
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        ptx::mma_tf32_ts(d2 + 64, sl + 8 * k, dB0 + kB2 + k16(k), idesc64, 1);
                    ptx::mma_commit(d2_full);
                    ptx::mma_commit(&d1_free[bf]);
                }
                // a copy still in flight after a failed wait lands before the CTA exits
                if (pending) ptx::mbar_wait(b2_full, nb2 & 1, kWaitLimit);
                ptx::mma_commit(drain2);
                if (!ptx::mbar_wait(drain2, nd2 & 1, kWaitLimit)) ok = false;
            }
            if (!ok) atomicOr(P.err, kErrTimeout);
        }
    } else if (warp < 10) {
        // ------------------------------------------- x_lo and S_lo (8 warps)
        const int q = warp & 3;                 // TMEM lane quarter this warp may access
        const int h = (warp - 2) >> 2;          // column half: K-block h of the tile
        const int r = 32 * q + lane;            // tile row = TMEM lane
        const uint32_t lanes = (uint32_t)(32 * q) << 16;
        uint32_t u[32];

        auto conv = [&](int i) -> bool {
            const int s = i % kStages;
            if (!ptx::mbar_wait(&x_full[s], (i / kStages) & 1, kWaitLimit)) return false;
            const unsigned char* src = xbuf + s * kTileBytes;
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                float4 a = *reinterpret_cast<const float4*>(src + sw128_off(r, 8 * h + cc));
                u[4 * cc + 0] = lo_tf32(a.x);
                u[4 * cc + 1] = lo_tf32(a.y);
                u[4 * cc + 2] = lo_tf32(a.z);
                u[4 * cc + 3] = lo_tf32(a.w);
            }
            const uint32_t xcol = tmem + lanes + kColXlo + (i & 1) * 64 + 32 * h;
            ptx::tmem_st16(xcol, *reinterpret_cast<uint32_t(*)[16]>(u));
            ptx::tmem_st16(xcol + 16, *reinterpret_cast<uint32_t(*)[16]>(u + 16));
            ptx::tmem_wait_st();
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&xlo_full[i & 1]);
            return true;
        };

        if (count > 0) ok = conv(0);
        uint32_t v[32];
        for (int i = 0; i < count && ok; ++i) {
            const int d = i & 1;
            // x_lo buffer (i + 1) & 1 was read by the DCT GEMM of tile i - 1,
            // complete since the previous iteration waited on it
            if (i + 1 < count && !conv(i + 1)) { ok = false; break; }
            if (!ptx::mbar_wait(&d1_full[d], (i >> 1) & 1, kWaitLimit)) { ok = false; break; }
            ptx::tc_fence_after();
            // S = main + correction half (round to nearest), then split it in place:
            // S over the main half, S_lo over the correction half
            const uint32_t mcol = tmem + lanes + kColD1 + d * 128 + 32 * h, ccol = mcol + 64;
            ptx::tmem_ld16(mcol, *reinterpret_cast<uint32_t(*)[16]>(u));
            ptx::tmem_ld16(mcol + 16, *reinterpret_cast<uint32_t(*)[16]>(u + 16));
            ptx::tmem_ld16(ccol, *reinterpret_cast<uint32_t(*)[16]>(v));
            ptx::tmem_ld16(ccol + 16, *reinterpret_cast<uint32_t(*)[16]>(v + 16));
            ptx::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float sv = __uint_as_float(u[j]) + __uint_as_float(v[j]);
                u[j] = __float_as_uint(sv);
                v[j] = lo_tf32(sv);
            }
            ptx::tmem_st16(mcol, *reinterpret_cast<uint32_t(*)[16]>(u));
            ptx::tmem_st16(mcol + 16, *reinterpret_cast<uint32_t(*)[16]>(u + 16));
            ptx::tmem_st16(ccol, *reinterpret_cast<uint32_t(*)[16]>(v));
            ptx::tmem_st16(ccol + 16, *reinterpret_cast<uint32_t(*)[16]>(v + 16));
            ptx::tmem_wait_st();
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&s_full[i & 1]);
        }
        if (!ok && lane == 0) atomicOr(P.err, kErrTimeout);
    } else if (warp < 14) {
        // ------------------------------------------------- Y out (4 warps)
        const int q = warp & 3;
        const int r = 32 * q + lane;
        const uint32_t lanes = (uint32_t)(32 * q) << 16;
        const int gtid = threadIdx.x - 320;     // 0..127
        uint32_t u[64];
        SegCursor cursor(P, t0);
        for (int i = 0; i < count && ok; ++i) {
            const int tile = t0 + i;
            const int sg = cursor.at(P, tile);
            const int row0 = (tile - P.seg[sg].tile_start) * kTcRows;
            // every Y thread reaches both named barriers of the iteration; a
            // wait that ran out ends the loop for all four warps together
            const bool got = __all_sync(0xffffffffu, ptx::mbar_wait(d2_full, i & 1, kWaitLimit));
            if (got) {
                ptx::tc_fence_after();
                // Y = main + correction half (round to nearest); the correction
                // half comes in 8 columns at a time to bound the registers
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    ptx::tmem_ld16(tmem + lanes + kColD2 + 16 * j, *reinterpret_cast<uint32_t(*)[16]>(u + 16 * j));
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    uint32_t w[8];
                    ptx::tmem_ld8(tmem + lanes + kColD2 + 64 + 8 * j, w);
                    ptx::tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        u[8 * j + e] = __float_as_uint(__uint_as_float(u[8 * j + e]) + __uint_as_float(w[e]));
                }
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(d2_empty);
            }
            // the previous tile's store has read the staging tile
            if (gtid == 0) ptx::bulk_wait_group_read0();
            if (!ptx::named_bar_and(2, 128, got)) { ok = false; break; }
#pragma unroll
            for (int cc = 0; cc < 16; ++cc)
                *reinterpret_cast<uint4*>(ybuf + sw128_off(r, cc)) =
                    make_uint4(u[4 * cc], u[4 * cc + 1], u[4 * cc + 2], u[4 * cc + 3]);
            ptx::fence_proxy_async_smem();
            ptx::named_bar_sync(2, 128);
            if (gtid == 0) {
                // rows past the segment's end are clipped by the tensor map
                ptx::tma_store_2d(&P.ymap[sg], 0, row0, ybuf);
                ptx::tma_store_2d(&P.ymap[sg], 32, row0, ybuf + kTileBytes / 2);
                ptx::bulk_commit_group();
            }
        }
        if (gtid == 0) ptx::bulk_wait_group0();
        if (!ok && lane == 0) atomicOr(P.err, kErrTimeout);
    } else {
        // ------------------------------------------- leftover signals (warp 14)
        // y = W (U^T x) per signal: lanes own output coefficients k, k + 32
        for (int sg = c; sg < P.nseg; sg += G) {
            const TcSeg& S = P.seg[sg];
            const int n = S.n;
            for (int t = 0; t < S.tail; ++t) {
                const float* xs = S.xt + (int64_t)t * n;
                float s0 = 0.f, s1 = 0.f;
                for (int j = 0; j < n; ++j) {
                    const float xj = xs[j];
                    if (lane < n) s0 = fmaf(S.ct[lane * n + j], xj, s0);
                    if (lane + 32 < n) s1 = fmaf(S.ct[(lane + 32) * n + j], xj, s1);
                }
                float y0 = 0.f, y1 = 0.f;
                for (int k = 0; k < n; ++k) {
                    const float sk = __shfl_sync(0xffffffffu, k < 32 ? s0 : s1, k & 31);
                    if (lane < n) y0 = fmaf(S.w[lane * n + k], sk, y0);
                    if (lane + 32 < n) y1 = fmaf(S.w[(lane + 32) * n + k], sk, y1);
                }
                float* ys = S.yt + (int64_t)t * n;
                if (lane < n) ys[lane] = y0;
                if (lane + 32 < n) ys[lane + 32] = y1;
            }
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 1) ptx::tmem_dealloc(tmem, 512);
}

// --------------------------------------------------------- operand images

// The two B operands of a plan, block diagonal over 64/n copies: B1 = I (x)
// U^T, B2 = I (x) W, each split into TF32 hi and lo and stacked as one 128 x 64
// operand [hi; lo] (N rows x K, K-major), in the 128-byte-swizzled layout the
// MMA reads from shared memory: per matrix two K blocks of 128 rows x 128 B.
__global__ void k_tc_images(int n, const double* ct64, const double* w64, float* img) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;  // r * 64 + k
    if (idx >= 64 * 64) return;
    int r = idx / 64, k = idx % 64;
    bool same = (r / n) == (k / n);
    double b1 = same ? ct64[(r % n) * n + (k % n)] : 0.0;
    double b2 = same ? w64[(r % n) * n + (k % n)] : 0.0;
    int kb = k / 32, c = (k % 32) / 4, e = k % 4;
    // byte offset of (row R, k) inside one stacked operand; R = r (hi) or 64 + r (lo)
    auto off = [&](int R) { return (kb * 16384 + R * 128 + ((c ^ (R & 7)) << 4) + e * 4) / 4; };
    float h1 = ptx::tf32_round((float)b1);
    float l1 = ptx::tf32_round((float)(b1 - (double)h1));
    float h2 = ptx::tf32_round((float)b2);
    float l2 = ptx::tf32_round((float)(b2 - (double)h2));
    img[off(r)] = h1;
    img[off(64 + r)] = l1;
    img[8192 + off(r)] = h2;
    img[8192 + off(64 + r)] = l2;
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

bool small_tc_capable(dctplus_plan_t p) {
    return tc_size(p->n) && p->tc.images != nullptr && p->d_ct32 && p->d_w32;
}

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

// Launches the tensor-core kernel over segments of whole signals. x and y of
// every segment must be 16-byte aligned. Full packed rows go to the tensor
// cores; the leftover signals of each segment to the kernel's CUDA-core warp.
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
        int tiles = 0, ns = 0, tails = 0;
        double samples = 0.0;
        for (; i0 < segs.size() && ns < kTcMaxSeg; ++i0) {
            const TcSegHost& g = segs[i0];
            const int n = g.plan->n;
            const int64_t rows64 = g.rows * n / 64;
            const int64_t body = rows64 * 64 / n;
            if (g.rows <= 0) continue;
            samples += (double)g.rows * n;
            if (rows64 > 0 && (!encode_map(&P.xmap[ns], g.x, rows64) || !encode_map(&P.ymap[ns], g.y, rows64)))
                return DCTPLUS_ERR_CUDA;
            P.images[ns] = g.plan->tc.images;
            TcSeg& t = P.seg[ns];
            t.tile_start = tiles;
            t.rows64 = (int)rows64;
            t.n = n;
            t.tail = (int)(g.rows - body);
            t.xt = g.x + body * n;
            t.yt = g.y + body * n;
            t.y = g.y;
            t.ct = g.plan->d_ct32;
            t.w = g.plan->d_w32;
            tiles += (int)((rows64 + kTcRows - 1) / kTcRows);
            tails += t.tail > 0;
            ++ns;
        }
        if (ns == 0) continue;
        P.nseg = ns;
        P.ntiles = tiles;
        P.err = device_error_word(dev);
        int grid = std::min(std::max(tiles, tails > 0 ? ns : 0), sm_count_tc(dev));
        if (grid <= 0) continue;
        k_small_tc<<<grid, kTcThreads, kSmemBytes, s>>>(P);
        // executed tensor work per 64-sample packed row: two GEMMs of K = 64, each an
        // N = 128 (stacked hi | lo) and an N = 64 product: 2 x 192 x 64 multiply-adds
        note_launch(s, "k_small_tc", 8.0 * samples, 2.0 * 384.0 * samples);
        DCTPLUS_CUDA_TRY(cudaGetLastError());
    }
    return DCTPLUS_OK;
}

static bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

bool small_tc_available(dctplus_plan_t p) { return small_tc_capable(p); }

// One plan over a contiguous batch: one launch of the tensor-core kernel.
dctplus_status launch_small_tc(dctplus_plan_t p, const float* x, int64_t ldx, float* y,
                               int64_t ldy, int64_t batch, cudaStream_t s) {
    const int n = p->n;
    if (!small_tc_capable(p) || ldx != n || ldy != n || !aligned16(x) || !aligned16(y))
        return launch_small_simt_f32(p, x, ldx, y, ldy, batch, s);
    if (batch <= 0) return DCTPLUS_OK;
    std::vector<TcSegHost> segs = {{p, x, y, batch}};
    return launch_tc_segments(segs, s, p->device);
}

}  // namespace dctplus
