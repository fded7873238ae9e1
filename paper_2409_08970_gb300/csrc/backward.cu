// Backward pass of the forward transform y_b = X^T x_b (reverse mode).
//
// Given upstream gradients g_b = dLoss/dy_b:
//   dLoss/dx_b = X g_b = U W^T g_b                 (the inverse transform, undone
//                                                   step by step: the transposed
//                                                   Cauchy product, then DCT-III)
//   dLoss/drho = sum_b sum_i g_bi w_i (K (y_b * w))_i
//   dLoss/dv   = rho X sum_b r_b,
//   r_b        = y_b * (K^T (g_b * w)) + g_b * (K (y_b * w)),
// with w = X^T v (w_i = -a_i / rho for a secular root, z_j for a deflated
// row) and K_ik = 1 / (mu_i - mu_k), K_ii = 0, from first-order perturbation of
// the eigenvectors of L~ + rho v v^T (Def. 2.3). K is antisymmetric, so
// K^T u = -K u and both products are one contraction with K over the stacked
// rows [y * w; g * w].
//
// Tables (built on the first call for a plan, FP64 then split): W^T and K as
// TF32 hi/lo pairs for the tensor-core GEMM and in FP32 for the CUDA-core
// path, and U for the DCT-III when no FFT length applies. Every plan length (n <= 16384).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace dctplus {

dctplus_status launch_gemm_tc(const float* a_hi, const float* a_lo, int64_t lda, const float* b_hi,
                              const float* b_lo, int64_t ldb, float* y, int64_t ldy, int M, int N,
                              int K, cudaStream_t s, int dev);  // gemm_tc.cu
void* plan_workspace(dctplus_plan_t p, cudaStream_t st, size_t bytes);  // api.cu

constexpr int kBwdMaxN = 16384;  // dense n x n tables: 7 x 4 n^2 bytes, 7.5 GB at n = 16384

struct BackwardTables {
    float* wt_hi = nullptr;  // n x n, W^T, TF32 hi / lo
    float* wt_lo = nullptr;
    float* wt32 = nullptr;   // n x n, W^T, FP32
    float* k_hi = nullptr;   // n x n, K, TF32 hi / lo
    float* k_lo = nullptr;
    float* k32 = nullptr;    // n x n, K, FP32
    float* u32 = nullptr;    // n x n, U (row k: c_j cos(pi j (2k + 1) / 2n)), when no FFT applies
    double* znd = nullptr;   // n: z with deflated entries zero
    double* w64 = nullptr;   // n: w = X^T v
    float* w32 = nullptr;
};

void free_backward(BackwardTables* b) {
    if (!b) return;
    void* ptrs[] = {b->wt_hi, b->wt_lo, b->wt32, b->k_hi, b->k_lo, b->k32, b->u32, b->znd, b->w64, b->w32};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete b;
}

namespace {

std::mutex g_bwd_mu;

__device__ __forceinline__ float tf32_rn(float v) { return __uint_as_float(ptx::cvt_rna_tf32(v)); }

// lambda_a - lambda_b = 4 sin(pi (a + b) / 2n) sin(pi (a - b) / 2n), from the table sin(pi m / 2n)
__device__ __forceinline__ double pole_gap(int a, int b, int n, const double* S) {
    int m = a + b;
    if (m > 2 * n - m) m = 2 * n - m;
    const int q = a - b;
    return 4.0 * S[m] * (q >= 0 ? S[q] : -S[-q]);
}

// W entry of row i at column j (FP64), as in the forward tables
__device__ __forceinline__ double w_entry(int i, int j, int n, const double* S, const int* kind,
                                          const int* pole, const double* tau, const double* a,
                                          const double* znd) {
    if (kind[i] == 0) return pole[i] == j ? 1.0 : 0.0;
    if (znd[j] == 0.0) return 0.0;
    return -a[i] * znd[j] / (tau[i] - pole_gap(j, pole[i], n, S));
}

__global__ void k_bwd_tables(int n, const double* __restrict__ S, const int* __restrict__ kind,
                             const int* __restrict__ pole, const double* __restrict__ tau,
                             const double* __restrict__ a, const double* __restrict__ znd,
                             float* wt_hi, float* wt_lo, float* wt32, float* k_hi, float* k_lo,
                             float* k32, float* u32) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * n) return;
    const int r = (int)(idx / n), c = (int)(idx % n);
    const double w = w_entry(c, r, n, S, kind, pole, tau, a, znd);  // W^T[r][c] = W[c][r]
    float h = tf32_rn((float)w);
    wt_hi[idx] = h;
    wt_lo[idx] = tf32_rn((float)(w - (double)h));
    wt32[idx] = (float)w;
    double kv = 0.0;
    if (r != c) kv = 1.0 / (pole_gap(pole[r], pole[c], n, S) + (tau[r] - tau[c]));  // mu_r - mu_c
    h = tf32_rn((float)kv);
    k_hi[idx] = h;
    k_lo[idx] = tf32_rn((float)(kv - (double)h));
    k32[idx] = (float)kv;
    if (u32) {
        const long long m = ((long long)c * (2 * r + 1)) % (4LL * n);  // exact phase reduction
        const double ck = c == 0 ? sqrt(1.0 / n) : sqrt(2.0 / n);
        u32[idx] = (float)(ck * cospi((double)m / (2.0 * n)));
    }
}

dctplus_status ensure_tables(dctplus_plan_t p) {
    std::lock_guard<std::mutex> lk(g_bwd_mu);
    if (p->bwd) return DCTPLUS_OK;
    const int n = p->n;
    BackwardTables* b = new BackwardTables();
    std::vector<double> znd(p->z), w64(n);
    for (int r = 0; r < n; ++r)
        if (p->row_kind[r] == 0) znd[p->row_pole[r]] = 0.0;
    for (int r = 0; r < n; ++r)
        w64[r] = p->row_kind[r] == 0 ? p->z[p->row_pole[r]] : -p->row_a[r] / p->rho;
    std::vector<float> w32(w64.begin(), w64.end());
    const bool need_u = !((n & (n - 1)) == 0 && n >= 128 && p->d_twiddle);
    const size_t nn = (size_t)n * n;
    auto fail = [&]() { free_backward(b); return DCTPLUS_ERR_CUDA; };
    float** f32s[] = {&b->wt_hi, &b->wt_lo, &b->wt32, &b->k_hi, &b->k_lo, &b->k32};
    for (float** q : f32s)
        if (cudaMalloc((void**)q, sizeof(float) * nn) != cudaSuccess) return fail();
    if (need_u && cudaMalloc((void**)&b->u32, sizeof(float) * nn) != cudaSuccess) return fail();
    if (cudaMalloc((void**)&b->znd, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc((void**)&b->w64, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc((void**)&b->w32, sizeof(float) * n) != cudaSuccess ||
        cudaMemcpy(b->znd, znd.data(), sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->w64, w64.data(), sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->w32, w32.data(), sizeof(float) * n, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail();
    k_bwd_tables<<<(unsigned)((nn + 255) / 256), 256>>>(n, p->d_sin, p->d_row_kind, p->d_row_pole,
                                                        p->d_row_tau, p->d_row_a, b->znd, b->wt_hi,
                                                        b->wt_lo, b->wt32, b->k_hi, b->k_lo, b->k32,
                                                        b->u32);
    count_launch();
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return fail();
    p->bwd = b;
    return DCTPLUS_OK;
}

// rows [y * w; g * w] (2 batch x n)
__global__ void k_param_prep(const float* __restrict__ y, int64_t ldy, const float* __restrict__ g,
                             int64_t ldg, const float* __restrict__ w, int n, int64_t batch,
                             float* __restrict__ a_hi) {
    const int64_t plane = batch * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < plane;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / n;
        const int i = (int)(e - b * n);
        const float u = y[b * ldy + i] * w[i], v = g[b * ldg + i] * w[i];
        a_hi[e] = u;
        a_hi[plane + e] = v;
    }
}

// pq rows 0..batch-1: K (y_b * w); rows batch..2 batch-1: K (g_b * w).
// rsum_i += sum_b (-y_bi (K (g_b * w))_i + g_bi (K (y_b * w))_i), grho += sum g_bi w_i (K (y_b * w))_i
// Each thread sums kRedRows rows in FP32 (FP64 arithmetic is slow on this part), then the
// partial sums meet in FP64 atomics.
constexpr int kRedRows = 16;
__global__ void k_param_reduce(const float* __restrict__ y, int64_t ldy, const float* __restrict__ g,
                               int64_t ldg, const float* __restrict__ w, const float* __restrict__ pq,
                               int n, int64_t batch, double* __restrict__ rsum,
                               double* __restrict__ grho) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b0 = (int64_t)blockIdx.y * kRedRows;
    double gr = 0.0;
    if (i < n) {
        const float wi = w[i];
        const int64_t b1 = min(batch, b0 + kRedRows);
        float r = 0.f, g32 = 0.f;
#pragma unroll 4
        for (int64_t b = b0; b < b1; ++b) {
            const float p = pq[b * n + i], q = pq[(batch + b) * n + i];
            const float yv = y[b * ldy + i], gv = g[b * ldg + i];
            r = fmaf(gv, p, fmaf(-yv, q, r));
            g32 = fmaf(gv * wi, p, g32);
        }
        atomicAdd(rsum + i, (double)r);
        gr = g32;
    }
    for (int off = 16; off > 0; off >>= 1) gr += __shfl_xor_sync(0xffffffffu, gr, off);
    if ((threadIdx.x & 31) == 0 && gr != 0.0) atomicAdd(grho, gr);
}

// out_j = scale sum_i T[j][i] r_i for a table given as TF32 hi + lo (about 22 bits),
// accumulated in FP64 (one warp per j)
__global__ void k_table_apply(int n, const float* __restrict__ hi, const float* __restrict__ lo,
                              const double* __restrict__ r, double scale, double* __restrict__ out,
                              float* __restrict__ out32) {
    const int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (j >= n) return;
    double acc = 0.0;
    const float* h = hi + (size_t)j * n;
    const float* l = lo ? lo + (size_t)j * n : nullptr;
    for (int i = lane; i < n; i += 32) acc += ((double)h[i] + (l ? (double)l[i] : 0.0)) * r[i];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
        if (out) out[j] = scale * acc;
        if (out32) out32[j] = (float)(scale * acc);
    }
}

__global__ void k_scale_f32_to_f64(int n, const float* __restrict__ v, double scale, double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = scale * (double)v[j];
}

bool aligned16(const void* p, int64_t ld) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0 && (ld & 3) == 0; }

unsigned blocks_for(int64_t work) { return (unsigned)std::min<int64_t>((work + 255) / 256, 152LL * 16); }

}  // namespace

}  // namespace dctplus

using namespace dctplus;

extern "C" dctplus_status dctplus_backward(dctplus_plan_t p, const float* gy, int64_t ldg,
                                           const float* y, int64_t ldy, float* gx, int64_t ldgx,
                                           double* grad_rho, double* grad_v, int64_t batch,
                                           dctplus_stream_t stream) {
    if (!p || batch < 0) return DCTPLUS_ERR_INVALID_ARG;
    const int n = p->n;
    const bool want_params = grad_rho || grad_v;
    if (batch > 0) {
        if (!gy || ldg < n || (want_params && (!y || ldy < n)) || (gx && ldgx < n))
            return DCTPLUS_ERR_INVALID_ARG;
        if ((reinterpret_cast<uintptr_t>(gy) | reinterpret_cast<uintptr_t>(y) |
             reinterpret_cast<uintptr_t>(gx)) & 3)
            return DCTPLUS_ERR_INVALID_ARG;
        if (gx) {  // gx must not overlap the inputs it is computed from
            const uintptr_t xa = (uintptr_t)gx, xe = xa + 4 * (size_t)((batch - 1) * ldgx + n);
            const uintptr_t ga = (uintptr_t)gy, ge = ga + 4 * (size_t)((batch - 1) * ldg + n);
            if (xa < ge && ga < xe) return DCTPLUS_ERR_INVALID_ARG;
            if (y) {
                const uintptr_t ya = (uintptr_t)y, ye = ya + 4 * (size_t)((batch - 1) * ldy + n);
                if (xa < ye && ya < xe) return DCTPLUS_ERR_INVALID_ARG;
            }
        }
    }
    if (n > kBwdMaxN) return DCTPLUS_ERR_UNSUPPORTED;
    if (batch > INT32_MAX / 2) return DCTPLUS_ERR_UNSUPPORTED;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return DCTPLUS_ERR_NO_DEVICE;
    if (cur != p->device) return DCTPLUS_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (grad_rho) DCTPLUS_CUDA_TRY(cudaMemsetAsync(grad_rho, 0, sizeof(double), st));
    if (grad_v) DCTPLUS_CUDA_TRY(cudaMemsetAsync(grad_v, 0, sizeof(double) * n, st));
    if (batch == 0 || (!gx && !want_params)) return DCTPLUS_OK;
    dctplus_status rc = ensure_tables(p);
    if (rc != DCTPLUS_OK) return rc;
    BackwardTables* T = p->bwd;

    const size_t plane = (size_t)batch * n;
    const size_t bytes = sizeof(float) * 4 * plane + sizeof(double) * (2 * n + 2) + sizeof(float) * (2 * n + 8);
    float* ws = static_cast<float*>(plan_workspace(p, st, bytes));
    if (!ws) return DCTPLUS_ERR_CUDA;
    const bool tc_shape = n % 128 == 0;
    const bool fft = (n & (n - 1)) == 0 && n >= 128 && p->d_twiddle;

    if (gx) {  // dLoss/dx = U (W^T g): transposed Cauchy product, then DCT-III
        float* t = ws;
        if (tc_shape && aligned16(gy, ldg)) {  // g split on chip
            rc = launch_gemm_tc(gy, nullptr, ldg, T->wt_hi, T->wt_lo, n, t, n, (int)batch, n, n, st, cur);
        } else {
            rc = launch_rows_gemm(gy, ldg, T->wt32, n, t, n, batch, n, n, st);
        }
        if (rc != DCTPLUS_OK) return rc;
        rc = fft ? launch_idct_fft(p, t, n, gx, ldgx, batch, st)
                 : launch_rows_gemm(t, n, T->u32, n, gx, ldgx, batch, n, n, st);
        if (rc != DCTPLUS_OK) return rc;
    }
    if (!want_params) return DCTPLUS_OK;

    float* a_hi = ws;               // 2 planes
    float* pq = ws + 2 * plane;     // 2 planes
    double* rsum = reinterpret_cast<double*>(ws + 4 * plane);
    double* t64 = rsum + n;
    double* grho = t64 + n;         // scratch when grad_rho is not wanted
    double* grho_out = grad_rho ? grad_rho : grho;
    const bool tc = tc_shape;
    DCTPLUS_CUDA_TRY(cudaMemsetAsync(rsum, 0, sizeof(double) * (n + n + 2), st));
    k_param_prep<<<blocks_for(plane), 256, 0, st>>>(y, ldy, gy, ldg, T->w32, n, batch, a_hi);
    note_launch(st, "k_param_prep", 16.0 * plane, 2.0 * plane);
    DCTPLUS_CUDA_TRY(cudaGetLastError());
    rc = tc ? launch_gemm_tc(a_hi, nullptr, n, T->k_hi, T->k_lo, n, pq, n, (int)(2 * batch), n, n, st, cur)
            : launch_rows_gemm(a_hi, n, T->k32, n, pq, n, 2 * batch, n, n, st);
    if (rc != DCTPLUS_OK) return rc;
    dim3 grid((n + 255) / 256, (unsigned)((batch + kRedRows - 1) / kRedRows));
    if (grid.y > 65535) return DCTPLUS_ERR_UNSUPPORTED;
    k_param_reduce<<<grid, 256, 0, st>>>(y, ldy, gy, ldg, T->w32, pq, n, batch, rsum, grho_out);
    note_launch(st, "k_param_reduce", 16.0 * plane, 6.0 * plane);
    DCTPLUS_CUDA_TRY(cudaGetLastError());
    if (grad_v) {  // rho X rsum = rho U (W^T rsum): W^T from its hi / lo table, FP64 sums
        float* t32 = reinterpret_cast<float*>(grho + 2);  // n floats after the FP64 scratch
        float* v32 = t32 + n;
        k_table_apply<<<(n + 7) / 8, 256, 0, st>>>(n, T->wt_hi, T->wt_lo, rsum, 1.0, t64, t32);
        note_launch(st, "k_table_apply", 8.0 * (double)n * n, 4.0 * (double)n * n);
        DCTPLUS_CUDA_TRY(cudaGetLastError());
        if (fft) {  // DCT-III of the single vector in FP32, scaled by rho into FP64
            rc = launch_idct_fft(p, t32, n, v32, n, 1, st);
            if (rc != DCTPLUS_OK) return rc;
            k_scale_f32_to_f64<<<(n + 255) / 256, 256, 0, st>>>(n, v32, p->rho, grad_v);
            note_launch(st, "k_scale_f32_to_f64", 12.0 * n, (double)n);
        } else {
            k_table_apply<<<(n + 7) / 8, 256, 0, st>>>(n, T->u32, nullptr, t64, p->rho, grad_v, nullptr);
            note_launch(st, "k_table_apply", 4.0 * (double)n * n, 2.0 * (double)n * n);
        }
        DCTPLUS_CUDA_TRY(cudaGetLastError());
    }
    return DCTPLUS_OK;
}
