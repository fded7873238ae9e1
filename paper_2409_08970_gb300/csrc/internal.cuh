// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "../../include/dctplus.h"

namespace dctplus {

constexpr int kMaxN = 16384;
constexpr int kSmallMax = 64;      // n <= 64: fused small-n kernels
constexpr int kTableMax = 4096;    // n <= 4096: a stored FP32 Cauchy table is allowed
constexpr int kF64Max = 1024;      // FP64 execute path
constexpr int kCauchySimtSigTile = 64;  // signals per CTA tile of the CUDA-core Cauchy product

// Device error word bits (dctplus_sync_check).
constexpr unsigned kErrIndex = 1u;    // an index guard fired
constexpr unsigned kErrTimeout = 2u;  // a bounded wait gave up

extern std::atomic<int64_t> g_launches;

// Every kernel launch goes through this so dctplus_launch_count is exact.
inline void count_launch(int k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Execute-path launches also report themselves for the kernel timing trace
// (dctplus_trace_begin / dctplus_trace_end): `name` is the kernel, `bytes` the
// algorithmic global-memory traffic of the launch (inputs read once, outputs
// written once), `flops` its arithmetic (tensor-core products counted as
// executed, split operands included). When a trace is open on stream s and s is
// not capturing, an event is recorded after the launch. Always counts it.
void note_launch(cudaStream_t s, const char* name, double bytes, double flops);

unsigned* device_error_word(int device);  // lazily allocated per device

// Device tables of the hierarchical Cauchy evaluation (hier.cu) and of the
// backward pass (backward.cu).
struct HierTables;
struct BackwardTables;
struct NfstFastTables;

// Tables consumed by the tensor-core small-n kernel (see small_tc.cu).
struct SmallTcTables {
    // 64x64 block-diagonal operands, each as an FP32 image already in the
    // K-major 128-byte-swizzled shared-memory layout the MMA reads:
    // [0] DCT hi, [1] DCT lo, [2] W hi, [3] W lo; 16 KB each.
    float* images = nullptr;
};

}  // namespace dctplus

struct dctplus_plan_s {
    int n = 0;
    double rho = 0.0;
    int device = 0;
    int cauchy_mode = DCTPLUS_CAUCHY_AUTO;
    int far_field = 0;  // hierarchical mode: 1 = leaf level, 2 = tree (resolved at plan time)
    std::vector<double> v;

    // host copies of the setup stage, per output row r (ascending eigenvalue)
    std::vector<double> eig, z, row_tau, row_a;
    std::vector<int> row_kind, row_pole;
    int K = 0;  // number of secular roots (non-deflated poles)

    // device tables
    double* d_z = nullptr;         // n
    double* d_sin = nullptr;       // n+1: sin(pi m / 2n), m = 0..n
    double* d_row_tau = nullptr;   // n
    double* d_row_a = nullptr;     // n
    int* d_row_kind = nullptr;     // n
    int* d_row_pole = nullptr;     // n
    float* d_ct32 = nullptr;       // n x n, U^T row-major (n <= 64)
    double* d_ct64 = nullptr;      // n x n, U^T row-major (F64 path, n <= 1024)
    float* d_w32 = nullptr;        // n x n, W = X^T U row-major (n <= 4096)
    double* d_w64 = nullptr;       // n x n (F64 path, n <= 1024)
    float* d_twiddle = nullptr;    // FFT DCT tables (n >= 128)
    float* d_whi = nullptr;        // n x n W split into TF32 hi / lo (dense tensor-core mode)
    float* d_wlo = nullptr;
    float* d_xthi = nullptr;       // n x n X^T split into TF32 hi / lo (dense-GFT baseline)
    float* d_xtlo = nullptr;
    // per-row generator data for on-chip Cauchy tiles (FP32): pole, tau, -a
    int* d_gen_pole = nullptr;
    float* d_gen_tau = nullptr;
    float* d_gen_na = nullptr;
    float* d_gen_z = nullptr;      // z_k in FP32 (0 where deflated)
    float* d_gen_sin = nullptr;    // sin(pi m / 2n), FP32, m = 0..2n
    dctplus::SmallTcTables tc;
    dctplus::HierTables* hier = nullptr;
    dctplus::BackwardTables* bwd = nullptr;  // built on the first dctplus_backward call
    // the paper's trigonometric route (cauchy mode DCTPLUS_CAUCHY_NFST)
    int* d_nfst_kind = nullptr;
    void* d_nfst_rows = nullptr;
    double* d_nfst_znd = nullptr;
    dctplus::NfstFastTables* nfst = nullptr;  // O(n log n) route tables (n a power of two <= 8192)

    // staging for dctplus_execute_host
    void* d_stage = nullptr;
    size_t stage_bytes = 0;
};

struct dctplus_group_s {
    int device = 0;
    std::vector<dctplus_plan_t> plans;
    // device table of plan pointers for the persistent kernel
    void* d_plan_tables = nullptr;
    int64_t* d_seg = nullptr;
    int seg_cap = 0;
    std::vector<int64_t> seg_cache;
    int* d_tiles = nullptr;  // per-tile work list (see small kernels)
    int tile_cap = 0;
    int ntiles = 0;
    void* d_stage = nullptr;
    size_t stage_bytes = 0;
    // streams and events of the pipelined host-buffer path (created on first use)
    cudaStream_t pipe_compute = nullptr, pipe_d2h = nullptr;
    std::vector<cudaEvent_t> pipe_events;
};

#define DCTPLUS_CUDA_TRY(expr)                                  \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) return DCTPLUS_ERR_CUDA;         \
    } while (0)

namespace dctplus {

// One segment of contiguous signals for the tensor-core kernel.
struct TcSegHost {
    dctplus_plan_t plan;
    const float* x;
    float* y;
    int64_t rows;  // signals
};

// small_tc.cu
bool small_tc_capable(dctplus_plan_t p);
dctplus_status launch_tc_segments(const std::vector<TcSegHost>& segs, cudaStream_t s, int dev);

// autotune.cu: the cache entry for (device, n, batch bucket), if any
int64_t tune_bucket(int64_t batch);
bool tune_lookup(const char* path, const char* device, int n, int64_t batch, int* mode, int* far);

// plan.cu
dctplus_status build_plan(dctplus_plan_t p, const dctplus_opts& o);
void free_plan_tables(dctplus_plan_t p);

// hier.cu
constexpr int kHierAutoMin = 1024;  // AUTO picks the hierarchical product from this n on
constexpr int kTreeAutoMin = 8192;  // the far field's default form: the tree from this n on
bool hier_shape(int n);
dctplus_status setup_hier(dctplus_plan_t p, const double* d_znd);
void free_hier(HierTables* h);
dctplus_status launch_hier(dctplus_plan_t p, const float* x, int64_t ldx, float* y, int64_t ldy,
                           int64_t batch, cudaStream_t st);
// K <= kFarMaxPlans hierarchical plans of one length over the same signals: one DCT-II,
// then plan k's output into ys[k] (row stride ldy)
dctplus_status launch_hier_multi(const dctplus_plan_t* plans, int K, const float* x, int64_t ldx,
                                 float* const* ys, int64_t ldy, int64_t batch, cudaStream_t st);

// gemm_tc.cu: split-TF32 tensor-core product y = A B^T over K segments
struct GemmSrc {
    const float* a_hi;
    const float* a_lo;
    int64_t lda;
    int Ka;              // A columns (TMA reads beyond read as zero)
    const float* b_hi;
    const float* b_lo;
    int64_t ldb;
    int Kb;              // B columns
};
constexpr int kGemmTabStride = 34;  // ints per column tile of a segment table
constexpr int kGemmMaxSeg = 8;
// y[M x N] = (a_hi + a_lo) (b_hi + b_lo)^T, K columns (a_lo null: formed on chip)
dctplus_status launch_gemm_tc(const float* a_hi, const float* a_lo, int64_t lda, const float* b_hi,
                              const float* b_lo, int64_t ldb, float* y, int64_t ldy, int M, int N, int K,
                              cudaStream_t s, int dev);
constexpr int kGemmBN = 128;         // output columns per tile (bn: 128, or 64 for products with few tiles)
dctplus_status launch_gemm_tc_segs(const GemmSrc* srcs, int nsrc, const int* tab, int64_t chunks_total,
                                   double a_cols, float* y, float* y_lo, int64_t ldy, int M, int N,
                                   cudaStream_t s, int dev, const char* name, int bn = kGemmBN);

// pruned.cu
void pruned_forget(dctplus_plan_t p);  // drop cached stacked tables that use p
// y[b][r] = sum_{k < Kd} a[b][k] w[r][k] for r < N on CUDA cores (any sizes)
dctplus_status launch_rows_gemm(const float* a, int64_t lda, const float* w, int64_t ldw, float* y,
                                int64_t ldy, int64_t batch, int N, int Kd, cudaStream_t st);

// backward.cu
void free_backward(BackwardTables* b);

// nfst.cu
bool nfst_fast_shape(int n);  // n a power of two, 16 <= n <= 8192: the O(n log n) route applies
dctplus_status setup_nfst(dctplus_plan_t p);
void free_nfst(NfstFastTables* t);
template <typename T>
dctplus_status launch_nfst(dctplus_plan_t p, const T* x, int64_t ldx, T* y, int64_t ldy, int64_t batch,
                           cudaStream_t st);

// small_simt.cu
dctplus_status launch_small_simt_f32(dctplus_plan_t p, const float* x, int64_t ldx, float* y,
                                     int64_t ldy, int64_t batch, cudaStream_t s);

// Far-field outputs of the DCT-II kernel for the hierarchical Cauchy product
// (hier.cu): with s in shared memory the kernel also forms, per signal, the
// leaf moments of the far field (P2M) and the values of the dense rows.
constexpr int kFarR = 12;     // Chebyshev degree (moments per box)
constexpr int kFarTqLd = 24;  // row pitch of the P2M and M2M tables (conflict-free fragment loads)
constexpr int kFarMaxLev = 8; // tree levels (leaf level included), nleaf <= 256
struct DctFar {
    const float* zf;      // n: z_j, 0 where deflated
    const float* tq_hi;   // 64 x kFarTqLd: S_a(u_jj) at the 64 source positions of a leaf
    const float* tq_lo;   // (a < 12; other columns 0), TF32 hi and remainder
    float* mc;            // moments of the tree boxes: leaf level (P2M) mc[b * ldm + leaf * 12 + a]
    int64_t ldm;          //   = sum_jj S_a(u_jj) z_j s_j, level l at lev_off[l] (M2M)
    const float* tm_hi;   // M2M re-expansion [24][kFarTqLd]: row k = child * 12 + b, column a
    const float* tm_lo;   //   holds S_a^parent(child's node b), TF32 hi and remainder
    int nlev;             // levels formed here (1: leaf moments only)
    int lev_off[kFarMaxLev];
    const float* out_g;   // nout x n: for the rows whose eigenvalue mu_o lies outside [0, 4],
    int nout;             // g_oj = -a_o / (mu_o - lambda_j) (0 where z_j = 0)
    float* dv;            // 32 dense-row slots per signal: dv[b * ldd + dbase + o] = sum_j g_oj z_j s_j
    int64_t ldd;
    int dbase;            // the plan's first slot (even; its nout <= 2 slots follow)
    int dzero;            // 1: also write zeros to the other slots (the first plan to use dv)
    int moments;          // 1: form the moments (and M2M); 0: the previous plan of the set
                          //   has the same zf and formed them (this plan: dense rows only)
};

// The far-field inputs of up to kFarMaxPlans plans of one length over the same signals: the
// DCT-II is formed once, the moments and dense rows per plan.
constexpr int kFarMaxPlans = 4;
struct DctFarSet {
    int K;
    DctFar f[kFarMaxPlans];
};

// api.cu: streams on which plans 1 .. K - 1 of a multi-plan call run their own products, forked
// from the caller's stream after the shared DCT-II (event `fork`) and joined back (`join`).
// One set per (device, caller stream), created on first use outside stream capture; null while
// the caller's stream is being captured before the set exists, or while it is traced.
struct SideStreams {
    cudaStream_t side[kFarMaxPlans - 1];
    cudaEvent_t fork;
    cudaEvent_t join[kFarMaxPlans - 1];
};
const SideStreams* side_streams(int dev, cudaStream_t caller);

// Runs body(k, stream) for k = 0 .. K - 1 (K <= kFarMaxPlans) where the K bodies are independent:
// body 0 on the caller's stream, the others on side streams forked from it (after the work it
// already holds) and joined back, also after an error, so that a stream capture stays whole. All
// on the caller's stream when side_streams gives none.
template <class Body>
dctplus_status run_forked(int dev, cudaStream_t st, int K, Body body) {
    const SideStreams* ss = K > 1 ? side_streams(dev, st) : nullptr;
    dctplus_status r = DCTPLUS_OK;
    if (!ss) {
        for (int k = 0; k < K && r == DCTPLUS_OK; ++k) r = body(k, st);
        return r;
    }
    if (cudaEventRecord(ss->fork, st) != cudaSuccess) return DCTPLUS_ERR_CUDA;
    for (int k = 1; k < K; ++k) {
        cudaStream_t sk = ss->side[k - 1];
        const dctplus_status rk = cudaStreamWaitEvent(sk, ss->fork, 0) == cudaSuccess ? body(k, sk) : DCTPLUS_ERR_CUDA;
        if (r == DCTPLUS_OK) r = rk;
    }
    const dctplus_status r0 = body(0, st);
    for (int k = 1; k < K; ++k)
        if (cudaEventRecord(ss->join[k - 1], ss->side[k - 1]) != cudaSuccess ||
            cudaStreamWaitEvent(st, ss->join[k - 1], 0) != cudaSuccess)
            r = DCTPLUS_ERR_CUDA;
    return r != DCTPLUS_OK ? r : r0;
}

// large.cu
// DCT-II with the far-field outputs above (n a power of two in [256, 16384])
dctplus_status launch_dct_far(dctplus_plan_t p, const float* x, int64_t ldx, float* s_out, int64_t lds,
                              int64_t batch, const DctFar& far, cudaStream_t st);
dctplus_status launch_dct_far_multi(dctplus_plan_t p, const float* x, int64_t ldx, float* s_out, int64_t lds,
                                    int64_t batch, const DctFarSet& far, cudaStream_t st);
dctplus_status launch_dct_fft(dctplus_plan_t p, const float* x, int64_t ldx, float* s_out,
                              int64_t lds, int64_t batch, cudaStream_t st);
// DCT-III (inverse of the orthonormal DCT-II), n a power of two in [128, 16384]
dctplus_status launch_idct_fft(dctplus_plan_t p, const float* s, int64_t lds, float* x, int64_t ldx,
                               int64_t batch, cudaStream_t st);
dctplus_status launch_cauchy_simt(dctplus_plan_t p, const float* s_in, int64_t lds, float* y,
                                  int64_t ldy, int64_t batch, cudaStream_t st);
// FP64, n <= 64: a warp per signal
dctplus_status launch_small_f64(dctplus_plan_t p, const double* x, int64_t ldx, double* y,
                                int64_t ldy, int64_t batch, cudaStream_t st);
dctplus_status launch_dense_f64(dctplus_plan_t p, const double* x, int64_t ldx, double* y,
                                int64_t ldy, int64_t batch, cudaStream_t st);
dctplus_status launch_large_f32(dctplus_plan_t p, const float* x, int64_t ldx, float* y,
                                int64_t ldy, int64_t batch, cudaStream_t st);

}  // namespace dctplus
