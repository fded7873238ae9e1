// Progressive multi-transform with output pruning (Theorem 3.4, Fig. 2).
//
// K updates of the same path graph share the DCT-II of a signal (Algorithm 1
// step 1 does not depend on v or rho). Each update then needs only the first
// m rows of its coefficient matrix W_k = -diag(a) C(mu, lambda) diag(z)
// (Theorem 3.1), and with c_p < n only their first c_p columns: C^ keeps the
// upper-left c_p x c_p block (Theorem 3.4). So one call is
//   s   = DCT-II(x)                          (once per signal)
//   y_k = W_k[0:m, 0:c_p] s[0:c_p]           for k = 0..K-1,
// and all K products are one GEMM against the stacked rows
//   B = [W_0[0:m, 0:c_p]; ...; W_{K-1}[0:m, 0:c_p]]   ([K m] x c_p),
// whose output row for a signal is y_0 | y_1 | ... | y_{K-1}.
//
// B is built once per (plans, m, c_p) from the plans' FP64 setup data on the
// host (entries from the pole-gap product form, as in the plan tables), split
// into TF32 hi/lo, uploaded, and cached; dctplus_destroy drops the cache
// entries of a plan.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace dctplus {

dctplus_status launch_gemm_tc_band(const float* a_hi, const float* a_lo, int64_t lda, int Ka,
                                   const float* b_hi, const float* b_lo, int64_t ldb, float* y,
                                   int64_t ldy, int M, int N, int K, const int* kbeg,
                                   cudaStream_t s, int dev);  // gemm_tc.cu
void* plan_workspace(dctplus_plan_t p, cudaStream_t st, size_t bytes);  // api.cu

namespace {

struct PrunedSet {
    std::vector<dctplus_plan_t> plans;
    int m = 0, cp = 0, device = 0;
    float* b_hi = nullptr;  // [K m] x c_p, TF32 hi
    float* b_lo = nullptr;  // TF32 remainder
    float* b32 = nullptr;   // FP32 rounding of the FP64 entries (CUDA-core path)
};

std::mutex g_pr_mu;
std::vector<PrunedSet*> g_pr_cache;

float tf32_rn_host(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return f;
    u += 0xfffu + ((u >> 13) & 1u);
    u &= 0xffffe000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

void free_set(PrunedSet* s) {
    if (s->b_hi) cudaFree(s->b_hi);
    if (s->b_lo) cudaFree(s->b_lo);
    if (s->b32) cudaFree(s->b32);
    delete s;
}

// Rows 0..m-1, columns 0..cp-1 of W for one plan, FP64 (row-major, ld = cp).
void w_block(dctplus_plan_t p, int m, int cp, double* out) {
    const int n = p->n;
    std::vector<double> sn(2 * n + 1);
    for (int k = 0; k <= 2 * n; ++k) sn[k] = std::sin(M_PI * k / (2.0 * n));
    std::vector<double> znd(p->z);
    for (int r = 0; r < n; ++r)
        if (p->row_kind[r] == 0) znd[p->row_pole[r]] = 0.0;
    for (int i = 0; i < m; ++i) {
        double* row = out + (size_t)i * cp;
        if (p->row_kind[i] == 0) {
            for (int j = 0; j < cp; ++j) row[j] = (j == p->row_pole[i]) ? 1.0 : 0.0;
            continue;
        }
        const int pole = p->row_pole[i];
        const double tau = p->row_tau[i], a = p->row_a[i];
        for (int j = 0; j < cp; ++j) {
            if (znd[j] == 0.0) { row[j] = 0.0; continue; }
            int mm = j + pole;
            if (mm > 2 * n - mm) mm = 2 * n - mm;
            const int q = j - pole;
            const double d = 4.0 * sn[mm] * (q >= 0 ? sn[q] : -sn[-q]);  // lambda_j - lambda_pole
            row[j] = -a * znd[j] / (tau - d);
        }
    }
}

dctplus_status get_set(const dctplus_plan_t* plans, int K, int m, int cp, PrunedSet** out) {
    std::lock_guard<std::mutex> lk(g_pr_mu);
    for (PrunedSet* s : g_pr_cache) {
        if (s->m != m || s->cp != cp || (int)s->plans.size() != K) continue;
        if (std::equal(s->plans.begin(), s->plans.end(), plans)) { *out = s; return DCTPLUS_OK; }
    }
    PrunedSet* s = new PrunedSet();
    s->plans.assign(plans, plans + K);
    s->m = m;
    s->cp = cp;
    s->device = plans[0]->device;
    const size_t rows = (size_t)K * m, cnt = rows * cp;
    std::vector<double> w(cnt);
    for (int k = 0; k < K; ++k) w_block(plans[k], m, cp, w.data() + (size_t)k * m * cp);
    std::vector<float> hi(cnt), lo(cnt), f32(cnt);
    for (size_t e = 0; e < cnt; ++e) {
        hi[e] = tf32_rn_host((float)w[e]);
        lo[e] = tf32_rn_host((float)(w[e] - (double)hi[e]));
        f32[e] = (float)w[e];
    }
    const size_t bytes = sizeof(float) * cnt;
    if (cudaMalloc((void**)&s->b_hi, bytes) != cudaSuccess ||
        cudaMalloc((void**)&s->b_lo, bytes) != cudaSuccess ||
        cudaMalloc((void**)&s->b32, bytes) != cudaSuccess ||
        cudaMemcpy(s->b_hi, hi.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->b_lo, lo.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->b32, f32.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        free_set(s);
        return DCTPLUS_ERR_CUDA;
    }
    g_pr_cache.push_back(s);
    *out = s;
    return DCTPLUS_OK;
}

}  // namespace

constexpr int kRB = 64;  // signals per tile
constexpr int kRR = 64;  // output rows per tile
constexpr int kRK = 16;

// y[b][r] = sum_{k < Kd} a[b][k] w[r][k] for r < N (CUDA cores, FP32 with a fresh
// partial per K tile), any sizes.
__global__ void __launch_bounds__(256) k_rows_gemm(const float* __restrict__ a, int64_t lda,
                                                   const float* __restrict__ w, int64_t ldw,
                                                   float* __restrict__ y, int64_t ldy,
                                                   int64_t batch, int N, int Kd) {
    __shared__ float As[kRK][kRB + 4];
    __shared__ float Ws[kRK][kRR + 4];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t b0 = (int64_t)blockIdx.y * kRB;
    const int r0 = blockIdx.x * kRR;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < Kd; k0 += kRK) {
        for (int e = tid; e < kRB * kRK; e += 256) {
            const int bb = e / kRK, kk = e % kRK;
            const int64_t b = b0 + bb;
            const int k = k0 + kk;
            As[kk][bb] = (b < batch && k < Kd) ? a[b * lda + k] : 0.0f;
        }
        for (int e = tid; e < kRR * kRK; e += 256) {
            const int rr = e / kRK, kk = e % kRK;
            const int r = r0 + rr, k = k0 + kk;
            Ws[kk][rr] = (r < N && k < Kd) ? w[(int64_t)r * ldw + k] : 0.0f;
        }
        __syncthreads();
        float part[4][4] = {};
#pragma unroll
        for (int kk = 0; kk < kRK; ++kk) {
            float av[4], wv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) wv[j] = Ws[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) part[i][j] = fmaf(av[i], wv[j], part[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += part[i][j];
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t b = b0 + ty * 4 + i;
        if (b >= batch) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = r0 + tx * 4 + j;
            if (r < N) y[b * ldy + r] = acc[i][j];
        }
    }
}

dctplus_status launch_rows_gemm(const float* a, int64_t lda, const float* w, int64_t ldw, float* y,
                                int64_t ldy, int64_t batch, int N, int Kd, cudaStream_t st) {
    const int64_t by = (batch + kRB - 1) / kRB;
    if (by > 65535) {  // grid.y limit: split the batch
        for (int64_t b = 0; b < batch; b += 65535LL * kRB) {
            const int64_t nb = std::min<int64_t>(batch - b, 65535LL * kRB);
            dctplus_status r = launch_rows_gemm(a + b * lda, lda, w, ldw, y + b * ldy, ldy, nb, N, Kd, st);
            if (r != DCTPLUS_OK) return r;
        }
        return DCTPLUS_OK;
    }
    dim3 grid((N + kRR - 1) / kRR, (unsigned)by);
    k_rows_gemm<<<grid, 256, 0, st>>>(a, lda, w, ldw, y, ldy, batch, N, Kd);
    note_launch(st, "k_rows_gemm", 4.0 * ((double)batch * (Kd + N) + (double)N * Kd),
                2.0 * (double)batch * N * Kd);
    DCTPLUS_CUDA_TRY(cudaGetLastError());
    return DCTPLUS_OK;
}

void pruned_forget(dctplus_plan_t p) {
    std::lock_guard<std::mutex> lk(g_pr_mu);
    for (size_t i = 0; i < g_pr_cache.size();) {
        PrunedSet* s = g_pr_cache[i];
        if (std::find(s->plans.begin(), s->plans.end(), p) != s->plans.end()) {
            free_set(s);
            g_pr_cache.erase(g_pr_cache.begin() + i);
        } else {
            ++i;
        }
    }
}

}  // namespace dctplus

using namespace dctplus;

extern "C" dctplus_status dctplus_execute_pruned(const dctplus_plan_t* plans, int nplans,
                                                 const float* x_dev, int64_t ldx, float* y_dev,
                                                 int64_t ldy, int64_t batch, int m_out, int c_p,
                                                 dctplus_stream_t stream) {
    if (!plans || nplans < 1 || nplans > 64 || batch < 0) return DCTPLUS_ERR_INVALID_ARG;
    for (int k = 0; k < nplans; ++k)
        if (!plans[k]) return DCTPLUS_ERR_INVALID_ARG;
    const int n = plans[0]->n;
    for (int k = 1; k < nplans; ++k)
        if (plans[k]->n != n || plans[k]->device != plans[0]->device) return DCTPLUS_ERR_INVALID_ARG;
    if (m_out < 1 || m_out > c_p || c_p > n) return DCTPLUS_ERR_INVALID_ARG;
    const int64_t width = (int64_t)nplans * m_out;
    if (batch == 0) return DCTPLUS_OK;
    if (!x_dev || !y_dev || ldx < n || ldy < width) return DCTPLUS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(x_dev) | reinterpret_cast<uintptr_t>(y_dev)) & 3)
        return DCTPLUS_ERR_INVALID_ARG;
    const uintptr_t xa = (uintptr_t)x_dev, ya = (uintptr_t)y_dev;
    const uintptr_t xe = xa + 4 * (size_t)((batch - 1) * ldx + n);
    const uintptr_t ye = ya + 4 * (size_t)((batch - 1) * ldy + width);
    if (xa < ye && ya < xe) return DCTPLUS_ERR_INVALID_ARG;
    if (batch > INT32_MAX) return DCTPLUS_ERR_UNSUPPORTED;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return DCTPLUS_ERR_NO_DEVICE;
    if (cur != plans[0]->device) return DCTPLUS_ERR_INVALID_ARG;
    const bool fft = n > kSmallMax && (n & (n - 1)) == 0 && plans[0]->d_twiddle;
    if (!fft && !plans[0]->d_ct32) return DCTPLUS_ERR_UNSUPPORTED;

    PrunedSet* set = nullptr;
    dctplus_status st = get_set(plans, nplans, m_out, c_p, &set);
    if (st != DCTPLUS_OK) return st;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const size_t plane = (size_t)batch * n;
    float* s = static_cast<float*>(plan_workspace(plans[0], cs, sizeof(float) * plane));
    if (!s) return DCTPLUS_ERR_CUDA;

    const bool tc = fft && width % 128 == 0 && width / 128 <= 128 && c_p % 32 == 0 &&
                    (reinterpret_cast<uintptr_t>(y_dev) & 15) == 0 && (ldy & 3) == 0;
    // Algorithm 1 step 1, once for all K updates
    if (fft) {
        st = launch_dct_fft(plans[0], x_dev, ldx, s, n, batch, cs);
    } else {
        st = launch_rows_gemm(x_dev, ldx, plans[0]->d_ct32, n, s, n, batch, n, n, cs);
    }
    if (st != DCTPLUS_OK) return st;
    // Theorem 3.4's pruned Cauchy products of all K updates in one contraction
    if (tc)
        return launch_gemm_tc_band(s, nullptr, n, c_p, set->b_hi, set->b_lo, c_p, y_dev, ldy,
                                   (int)batch, (int)width, c_p, nullptr, cs, cur);
    return launch_rows_gemm(s, n, set->b32, c_p, y_dev, ldy, batch, (int)width, c_p, cs);
}
