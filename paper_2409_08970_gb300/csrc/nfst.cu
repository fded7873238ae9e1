// The paper's own evaluation of the Cauchy product (Algorithm 1 steps 3-7,
// Sec. 4), as an alternative Cauchy mode (DCTPLUS_CAUCHY_NFST), FP64 inside.
//
// With s = z * DCT-II(x), the zero pole's column stays explicit (s_0 / mu_i) and
// the rest of the product is a rational function of x = 1 - mu / 2 whose poles
// are the zeros cos(pi j / n) of U_{n-1}. By Gastinel's proposition and
// Lemma 4.3 (d_n cancelled, so never formed) it equals a sine series over
// sin(n theta), mu = 2 - 2 cos(theta):
//   c_l = 2 sum_{j=1}^{n-1} (-1)^(j+1) s_j sin(pi l j / n) / sin(pi j / n)  (DST-I)
//   p_i = s_0 / mu_i - 1/2 sum_l c_l sin(l theta_i) / sin(n theta_i)
//   y_i = -a_i p_i.
// Roots outside (0, 4) (the root the paper isolates) are plain sums; deflated
// rows are the DCT coefficient. The paper evaluates the sine series with an
// NFST; here it is a Clenshaw recurrence per root (O(n) each), and the DCT-II
// and DST-I are direct sums, so the route is O(n^2) per signal: it reproduces
// the paper's arithmetic, not its speed. Its accuracy degrades like
// eps / |sin(n theta)| when a root sits next to a pole, which is why the
// tensor-core and hierarchical modes use the pole + offset form instead.
// One CTA per signal, n <= 1024.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace dctplus {

// per-row route data (FP64): kind (0 deflated, 1 sine series, 2 plain sum),
// 2 cos(theta), sin(theta), 1 / sin(n theta), mu
struct NfstRow {
    double c2, sn, isn, mu;
};

dctplus_status setup_nfst(dctplus_plan_t p) {
    const int n = p->n;
    if (n > kF64Max || !p->d_ct64) return DCTPLUS_ERR_UNSUPPORTED;
    std::vector<int> kind(n);
    std::vector<NfstRow> rows(n);
    std::vector<double> znd(p->z);
    for (int r = 0; r < n; ++r)
        if (p->row_kind[r] == 0) znd[p->row_pole[r]] = 0.0;
    for (int r = 0; r < n; ++r) {
        rows[r] = {0.0, 0.0, 0.0, 0.0};
        if (p->row_kind[r] == 0) { kind[r] = 0; continue; }
        const double half = M_PI * p->row_pole[r] / (2.0 * n);
        const double sh = std::sin(half), ch = std::cos(half);
        const double mu = 4.0 * sh * sh + p->row_tau[r];         // lambda_pole + tau
        const double mc = 4.0 * ch * ch - p->row_tau[r];         // 4 - mu without cancellation
        rows[r].mu = mu;
        if (mu > 0.0 && mc > 0.0) {
            const double th = 2.0 * std::atan2(std::sqrt(mu), std::sqrt(mc));
            kind[r] = 1;
            rows[r].c2 = 2.0 * std::cos(th);
            rows[r].sn = std::sin(th);
            rows[r].isn = 1.0 / std::sin(n * th);
        } else {
            kind[r] = 2;
        }
    }
    DCTPLUS_CUDA_TRY(cudaMalloc((void**)&p->d_nfst_kind, sizeof(int) * n));
    DCTPLUS_CUDA_TRY(cudaMalloc((void**)&p->d_nfst_rows, sizeof(NfstRow) * n));
    DCTPLUS_CUDA_TRY(cudaMalloc((void**)&p->d_nfst_znd, sizeof(double) * n));
    DCTPLUS_CUDA_TRY(cudaMemcpy(p->d_nfst_kind, kind.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    DCTPLUS_CUDA_TRY(cudaMemcpy(p->d_nfst_rows, rows.data(), sizeof(NfstRow) * n, cudaMemcpyHostToDevice));
    DCTPLUS_CUDA_TRY(cudaMemcpy(p->d_nfst_znd, znd.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    return DCTPLUS_OK;
}

// sin(pi k / 2n) for 0 <= k <= 2n from the plan's table S[m] = sin(pi m / 2n), m = 0..n
__device__ __forceinline__ double sin_half(long long k, int n, const double* S) {
    return S[k <= n ? k : 2LL * n - k];
}

// sin(pi m / n) for any integer m >= 0
__device__ __forceinline__ double sin_pi_over_n(long long m, int n, const double* S) {
    m %= 2LL * n;
    return m <= n ? sin_half(2 * m, n, S) : -sin_half(2 * (m - n), n, S);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_nfst_route(int n, const T* __restrict__ x, int64_t ldx,
                                                     T* __restrict__ y, int64_t ldy, int64_t batch,
                                                     const double* __restrict__ ct64,
                                                     const double* __restrict__ S,
                                                     const double* __restrict__ znd,
                                                     const int* __restrict__ kind,
                                                     const NfstRow* __restrict__ rows,
                                                     const int* __restrict__ pole,
                                                     const double* __restrict__ tau,
                                                     const double* __restrict__ a) {
    extern __shared__ double nsm[];
    double* xs = nsm;        // n
    double* sd = xs + n;     // n: DCT-II coefficients
    double* s = sd + n;      // n: z * sd
    double* c = s + n;       // n: DST-I coefficients c_l (index l)
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
        __syncthreads();
        for (int j = tid; j < n; j += nt) xs[j] = (double)x[b * ldx + j];
        __syncthreads();
        // Algorithm 1 step 1: sd_k = sum_j (U^T)_kj x_j, one warp per k
        for (int k = warp; k < n; k += nw) {
            double acc = 0.0;
            for (int j = lane; j < n; j += 32) acc += ct64[(size_t)k * n + j] * xs[j];
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) {
                sd[k] = acc;
                s[k] = znd[k] * acc;  // step 2
            }
        }
        __syncthreads();
        // steps 4-5: c_l = 2 sum_j (-1)^(j+1) s_j sin(pi l j / n) / sin(pi j / n), one warp per l
        for (int l = 1 + warp; l < n; l += nw) {
            double acc = 0.0;
            for (int j = 1 + lane; j < n; j += 32) {
                const double h = ((j & 1) ? 1.0 : -1.0) * s[j] / sin_half(2 * j, n, S);
                acc += h * sin_pi_over_n((long long)l * j, n, S);
            }
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) c[l] = 2.0 * acc;
        }
        __syncthreads();
        // steps 6-7 per output row, then the normalisation
        for (int r = tid; r < n; r += nt) {
            const int kd = kind[r];
            double out;
            if (kd == 0) {
                out = sd[pole[r]];
            } else if (kd == 1) {
                // Clenshaw: sum_{l=1}^{n-1} c_l sin(l theta) = b_1 sin(theta)
                const NfstRow R = rows[r];
                double b1 = 0.0, b2 = 0.0;
                for (int l = n - 1; l >= 1; --l) {
                    const double b0 = c[l] + R.c2 * b1 - b2;
                    b2 = b1;
                    b1 = b0;
                }
                const double f = b1 * R.sn * R.isn;
                out = -a[r] * (s[0] / R.mu - 0.5 * f);
            } else {
                // the isolated root: -a_r sum_j s_j / (mu_r - lambda_j), gaps from the pole form
                const int p0 = pole[r];
                double acc = 0.0;
                for (int j = 0; j < n; ++j) {
                    int m = j + p0;
                    if (m > 2 * n - m) m = 2 * n - m;
                    const int q = j - p0;
                    const double gap = tau[r] - 4.0 * S[m] * (q >= 0 ? S[q] : -S[-q]);
                    acc += s[j] / gap;
                }
                out = -a[r] * acc;
            }
            y[b * ldy + r] = (T)out;
        }
    }
}

template <typename T>
dctplus_status launch_nfst(dctplus_plan_t p, const T* x, int64_t ldx, T* y, int64_t ldy, int64_t batch,
                           cudaStream_t st) {
    const int n = p->n;
    if (!p->d_nfst_rows || n > kF64Max) return DCTPLUS_ERR_UNSUPPORTED;
    if (batch <= 0) return DCTPLUS_OK;
    const int threads = std::min(1024, std::max(64, (n + 31) / 32 * 32));
    const size_t smem = sizeof(double) * 4 * (size_t)n;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    const int64_t grid = std::min<int64_t>(batch, (int64_t)std::max(sms, 1) * 4);
    k_nfst_route<T><<<(unsigned)grid, threads, smem, st>>>(n, x, ldx, y, ldy, batch, p->d_ct64, p->d_sin,
                                                           p->d_nfst_znd, p->d_nfst_kind,
                                                           reinterpret_cast<const NfstRow*>(p->d_nfst_rows),
                                                           p->d_row_pole, p->d_row_tau, p->d_row_a);
    note_launch(st, "k_nfst_route", 2.0 * sizeof(T) * (double)batch * n, 6.0 * (double)batch * n * n);
    DCTPLUS_CUDA_TRY(cudaGetLastError());
    return DCTPLUS_OK;
}

template dctplus_status launch_nfst<float>(dctplus_plan_t, const float*, int64_t, float*, int64_t,
                                           int64_t, cudaStream_t);
template dctplus_status launch_nfst<double>(dctplus_plan_t, const double*, int64_t, double*, int64_t,
                                            int64_t, cudaStream_t);

}  // namespace dctplus
