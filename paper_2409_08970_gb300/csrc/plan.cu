// Setup stage of Fast DCT+ (Remark in Sec. 3): lambda, z, deflation, secular
// roots mu (FP64, on the GPU), normalisation a, and the tables the execute
// kernels read.
//
// Root representation. Every root is held as mu_i = lambda_o + tau_i with o
// the nearer pole of its Lemma 4.1 bracket, and every gap is formed as
//   lambda_j - mu_i = (lambda_j - lambda_o) - tau_i,
//   lambda_j - lambda_o = 4 sin(pi (j+o)/2n) sin(pi (j-o)/2n),
// from a table of sin(pi m / 2n), m = 0..n, with the first argument reflected
// to m = min(j+o, 2n-j-o). No gap is the difference of two rounded eigenvalues.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace dctplus {

std::atomic<int64_t> g_launches{0};

// ------------------------------------------------------------------ tables

__global__ void k_sin_table(int n, double* S) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m <= n) S[m] = sinpi((double)m / (2.0 * n));  // m <= n: argument <= 1/2, exact reduction
}

// cos(pi m / 2n) for any m >= 0 from the sine table (exact integer reduction).
__device__ __forceinline__ double cos_half_pi_over_n(long long m, int n, const double* S) {
    long long q = m % (4LL * n);
    if (q > 2LL * n) q = 4LL * n - q;  // cos(2 pi - t) = cos t
    double sgn = 1.0;
    if (q > n) { q = 2LL * n - q; sgn = -1.0; }  // cos(pi - t) = -cos t
    return sgn * S[n - q];                        // cos(t) = sin(pi/2 - t)
}

// lambda_j - lambda_p without cancellation.
__device__ __forceinline__ double pole_diff(int j, int p, int n, const double* S) {
    int m = j + p;
    if (m > 2 * n - m) m = 2 * n - m;
    int q = j - p;
    double s2 = q >= 0 ? S[q] : -S[-q];
    return 4.0 * S[m] * s2;
}

// z_k = c_k sum_j v_j cos(pi k (2j+1) / 2n) over the nonzero entries of v; one warp per k.
__global__ void k_z(int n, const int* vidx, const double* vval, int nnz, const double* S,
                    double* z) {
    int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (k >= n) return;
    double acc = 0.0;
    for (int t = lane; t < nnz; t += 32) {
        long long m = (long long)k * (2LL * vidx[t] + 1);
        acc += vval[t] * cos_half_pi_over_n(m, n, S);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) z[k] = (k == 0 ? sqrt(1.0 / n) : sqrt(2.0 / n)) * acc;
}

// ---------------------------------------------------------- secular solver

struct SecularSums {
    double g;     // 1/rho + sum z_j^2 / (lambda_j - mu)
    double dpsi;  // sum over lambda_j < mu of z_j^2 / (lambda_j - mu)^2
    double dphi;  // sum over lambda_j > mu of the same
    double sabs;  // sum |z_j^2 / (lambda_j - mu)|
};

__device__ SecularSums secular_eval(int n, double rho, int K, const int* poles, const double* zsq,
                                    const double* S, int origin, double tau) {
    double g = 0.0, dpsi = 0.0, dphi = 0.0, sabs = 0.0;
    int lane = threadIdx.x & 31;
    for (int t = lane; t < K; t += 32) {
        double delta = pole_diff(poles[t], origin, n, S) - tau;  // lambda_j - mu
        double r = 1.0 / delta;
        double term = zsq[t] * r;
        g += term;
        sabs += fabs(term);
        double d2 = term * r;
        if (delta < 0.0) dpsi += d2; else dphi += d2;
    }
    for (int o = 16; o > 0; o >>= 1) {
        g += __shfl_xor_sync(0xffffffffu, g, o);
        dpsi += __shfl_xor_sync(0xffffffffu, dpsi, o);
        dphi += __shfl_xor_sync(0xffffffffu, dphi, o);
        sabs += __shfl_xor_sync(0xffffffffu, sabs, o);
    }
    // lanes may differ in the last bit after the butterfly: take lane 0's values
    SecularSums r;
    r.g = 1.0 / rho + __shfl_sync(0xffffffffu, g, 0);
    r.dpsi = __shfl_sync(0xffffffffu, dpsi, 0);
    r.dphi = __shfl_sync(0xffffffffu, dphi, 0);
    r.sabs = __shfl_sync(0xffffffffu, sabs, 0);
    return r;
}

// One warp per root. Root i of K lies in (pole[i], pole[i+1]) for rho > 0 (the
// last one above pole[K-1]) and in (pole[i-1], pole[i]) for rho < 0 (the first
// one below pole[0]), Lemma 4.1. The iteration fits g by two poles at the
// bracket ends, g ~ c + s_l/(d_l - t) + s_r/(d_r - t), matching g and the
// derivative contributed by each side at the current point, and moves to the
// model's root; a step that leaves the current sign-change bracket is replaced
// by bisection, so every iteration shrinks the bracket.
__global__ void k_secular(int n, double rho, int K, const int* poles, const double* zsq,
                          const double* zsign, double znorm2, const double* S, int max_iter,
                          int* out_origin, double* out_tau, double* out_a, int* out_iters) {
    int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= K) return;
    const double eps = 1.1102230246251565e-16;
    int left = -1, right = -1;  // indices into poles[]
    if (rho > 0) { left = i; right = (i + 1 < K) ? i + 1 : -1; }
    else { right = i; left = (i >= 1) ? i - 1 : -1; }

    int origin;
    double lo, hi;
    if (left >= 0 && right >= 0) {
        double gap = pole_diff(poles[right], poles[left], n, S);
        SecularSums m = secular_eval(n, rho, K, poles, zsq, S, poles[left], 0.5 * gap);
        if (m.g >= 0.0) { origin = poles[left]; lo = 0.0; hi = 0.5 * gap; }
        else { origin = poles[right]; lo = -0.5 * gap; hi = 0.0; }
    } else if (right < 0) {  // rho > 0, above the largest pole
        origin = poles[left]; lo = 0.0; hi = rho * znorm2;
    } else {                 // rho < 0, below the smallest pole
        origin = poles[right]; lo = rho * znorm2; hi = 0.0;
    }
    double dl = left >= 0 ? pole_diff(poles[left], origin, n, S) : 0.0;
    double dr = right >= 0 ? pole_diff(poles[right], origin, n, S) : 0.0;

    double tau = 0.5 * (lo + hi);
    SecularSums f;
    int it = 0;
    bool converged = false;
    for (; it < max_iter; ++it) {
        f = secular_eval(n, rho, K, poles, zsq, S, origin, tau);
        if (f.g == 0.0) { converged = true; break; }
        if (f.g > 0.0) hi = tau; else lo = tau;
        double tol = 8.0 * eps * (fabs(1.0 / rho) + f.sabs);
        if (fabs(f.g) <= tol) { converged = true; break; }

        double eta;
        bool ok = false;
        if (left >= 0 && right >= 0) {
            double Dl = dl - tau, Dr = dr - tau;  // < 0, > 0
            double sl = f.dpsi * Dl * Dl, sr = f.dphi * Dr * Dr;
            double c = f.g - sl / Dl - sr / Dr;
            double a2 = c, a1 = -(c * (Dl + Dr) + sl + sr), a0 = Dl * Dr * f.g;
            if (fabs(a2) <= 1e-300 * fabs(a1)) {
                eta = -a0 / a1;
                ok = true;
            } else {
                double disc = fmax(a1 * a1 - 4.0 * a2 * a0, 0.0);
                double q = -0.5 * (a1 + copysign(sqrt(disc), a1));
                double e1 = (q != 0.0) ? a0 / q : 0.0;
                double e2 = q / a2;
                if (e1 > Dl && e1 < Dr) { eta = e1; ok = true; }
                else if (e2 > Dl && e2 < Dr) { eta = e2; ok = true; }
            }
        } else if (right < 0) {
            double Dl = dl - tau;
            double sl = f.dpsi * Dl * Dl;
            double c = f.g - sl / Dl;
            if (c > 0.0) { eta = Dl + sl / c; ok = true; }
        } else {
            double Dr = dr - tau;
            double sr = f.dphi * Dr * Dr;
            double c = f.g - sr / Dr;
            if (c < 0.0) { eta = Dr + sr / c; ok = true; }
        }
        double next = ok ? tau + eta : 0.5 * (lo + hi);
        if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
        if (fabs(next - tau) <= 2.0 * eps * fabs(tau) || !(hi - lo > 2.0 * eps * fmax(fabs(lo), fabs(hi)))) {
            converged = true;
            break;
        }
        tau = next;
    }
    if ((threadIdx.x & 31) == 0) {
        out_origin[i] = origin;
        out_tau[i] = tau;
        // a_i = sign / sqrt(sum_j z_j^2 / (mu_i - lambda_j)^2), sign = -sign(rho) sign(z_pi(i))
        double sgn = (rho > 0 ? -1.0 : 1.0) * zsign[i];
        out_a[i] = sgn / sqrt(f.dpsi + f.dphi);
        out_iters[i] = converged ? it + 1 : -1;
    }
}

// ---------------------------------------------------------- execute tables

// FP64 value -> TF32 hi + TF32 lo (both nearest)
__device__ __forceinline__ void split_tf32(double w, float* hi, float* lo) {
    float h = ptx::tf32_round((float)w);
    *hi = h;
    *lo = ptx::tf32_round((float)(w - (double)h));
}

// W[r][k] = -a_r z_k / (mu_r - lambda_k) for root rows, e_pole for deflated rows.
__global__ void k_w_table(int n, const int* row_kind, const int* row_pole, const double* row_tau,
                          const double* row_a, const double* znd, const double* S, float* w32,
                          double* w64, float* whi, float* wlo) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    int r = (int)(idx / n), k = (int)(idx % n);
    double w;
    if (row_kind[r] == 0) {
        w = (k == row_pole[r]) ? 1.0 : 0.0;
    } else if (znd[k] == 0.0) {
        w = 0.0;
    } else {
        double gap = row_tau[r] - pole_diff(k, row_pole[r], n, S);  // mu_r - lambda_k
        w = -row_a[r] * znd[k] / gap;
    }
    if (w32) w32[idx] = (float)w;
    if (w64) w64[idx] = w;
    if (whi) split_tf32(w, &whi[idx], &wlo[idx]);
}

// Dense X^T = W U^T (row r = eigenvector r in signal coordinates), split into
// TF32 hi / lo: the table of the dense-GFT comparison baseline.
__global__ void k_xt_table(int n, const double* w64, const double* ct64, float* hi, float* lo) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    int r = (int)(idx / n), j = (int)(idx % n);
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc = fma(w64[(long long)r * n + k], ct64[(long long)k * n + j], acc);
    split_tf32(acc, &hi[idx], &lo[idx]);
}

// Rows of U (U[c][k] = c_k cos(pi k (2c + 1) / 2n)) as TF32 hi / lo: the B operand of
// X^T = W U^T on the tensor cores (dense-GFT comparator for n > 1024).
__global__ void k_u_rows(int n, const double* S, float* hi, float* lo) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    int c = (int)(idx / n), k = (int)(idx % n);
    double ck = (k == 0 ? sqrt(1.0 / n) : sqrt(2.0 / n));
    split_tf32(ck * cos_half_pi_over_n((long long)k * (2LL * c + 1), n, S), &hi[idx], &lo[idx]);
}

// FP32 table to TF32 hi / lo (both rounded)
__global__ void k_split_table(long long count, const float* v, float* hi, float* lo) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= count) return;
    split_tf32((double)v[idx], &hi[idx], &lo[idx]);
}

// Ct[k][j] = c_k cos(pi k (2j+1) / 2n): the orthonormal DCT-II as a row-major matrix.
__global__ void k_ct_table(int n, const double* S, float* ct32, double* ct64) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    int k = (int)(idx / n), j = (int)(idx % n);
    double c = (k == 0 ? sqrt(1.0 / n) : sqrt(2.0 / n));
    double v = c * cos_half_pi_over_n((long long)k * (2LL * j + 1), n, S);
    if (ct32) ct32[idx] = (float)v;
    if (ct64) ct64[idx] = v;
}

// Per-row generator data for on-chip Cauchy tiles (FP32).
__global__ void k_gen_tables(int n, const int* row_kind, const int* row_pole,
                             const double* row_tau, const double* row_a, const double* znd,
                             const double* S, int* gpole, float* gtau, float* gna, float* gz,
                             float* gsin) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) {
        gpole[r] = row_kind[r] ? row_pole[r] : -1 - row_pole[r];  // deflated: -1 - j
        gtau[r] = (float)row_tau[r];
        gna[r] = (float)(-row_a[r]);
        gz[r] = (float)znd[r];
    }
    if (r <= n) gsin[r] = (float)S[r];
}

// ------------------------------------------------------------------ driver

template <typename T>
static cudaError_t dalloc(T** p, size_t count) {
    return cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(count, 1));
}

void free_plan_tables(dctplus_plan_t p) {
    void* ptrs[] = {p->d_z, p->d_sin, p->d_row_tau, p->d_row_a, p->d_row_kind, p->d_row_pole,
                    p->d_ct32, p->d_ct64, p->d_w32, p->d_w64, p->d_twiddle, p->d_gen_pole,
                    p->d_gen_tau, p->d_gen_na, p->d_gen_z, p->d_gen_sin, p->tc.images, p->d_stage,
                    p->d_whi, p->d_wlo, p->d_xthi, p->d_xtlo, p->d_nfst_kind, p->d_nfst_rows,
                    p->d_nfst_znd};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    free_hier(p->hier);
    p->hier = nullptr;
    free_backward(p->bwd);
    p->bwd = nullptr;
    free_nfst(p->nfst);
    p->nfst = nullptr;
}

dctplus_status setup_small_tc(dctplus_plan_t p);   // small_tc.cu
dctplus_status launch_gemm_tc(const float* a_hi, const float* a_lo, int64_t lda, const float* b_hi,
                              const float* b_lo, int64_t ldb, float* y, int64_t ldy, int M, int N,
                              int K, cudaStream_t s, int dev);  // gemm_tc.cu
dctplus_status setup_large(dctplus_plan_t p);      // large.cu

dctplus_status build_plan(dctplus_plan_t p, const dctplus_opts& o) {
    const int n = p->n;
    const double rho = p->rho;
    cudaStream_t s = 0;

    // nonzero entries of v
    std::vector<int> vidx;
    std::vector<double> vval;
    for (int j = 0; j < n; ++j)
        if (p->v[j] != 0.0) { vidx.push_back(j); vval.push_back(p->v[j]); }
    int nnz = (int)vidx.size();

    int* d_vidx = nullptr;
    double* d_vval = nullptr;
    DCTPLUS_CUDA_TRY(dalloc(&p->d_sin, n + 1));
    DCTPLUS_CUDA_TRY(dalloc(&p->d_z, n));
    DCTPLUS_CUDA_TRY(dalloc(&d_vidx, nnz));
    DCTPLUS_CUDA_TRY(dalloc(&d_vval, nnz));
    if (nnz) {
        DCTPLUS_CUDA_TRY(cudaMemcpy(d_vidx, vidx.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice));
        DCTPLUS_CUDA_TRY(cudaMemcpy(d_vval, vval.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice));
    }
    k_sin_table<<<(n + 1 + 255) / 256, 256, 0, s>>>(n, p->d_sin);
    k_z<<<(n * 32 + 255) / 256, 256, 0, s>>>(n, d_vidx, d_vval, nnz, p->d_sin, p->d_z);
    count_launch(2);
    DCTPLUS_CUDA_TRY(cudaGetLastError());
    p->z.assign(n, 0.0);
    DCTPLUS_CUDA_TRY(cudaMemcpy(p->z.data(), p->d_z, sizeof(double) * n, cudaMemcpyDeviceToHost));
    cudaFree(d_vidx);
    cudaFree(d_vval);

    // deflation (Sec. 4): |rho| |z_j| ||z|| <= 2^-48 max(1, |rho| ||z||^2, 4)
    double nz2 = 0.0;
    for (double zz : p->z) nz2 += zz * zz;
    const double scale = std::max({1.0, std::fabs(rho) * nz2, 4.0});
    const double thr = std::ldexp(1.0, -48) * scale;
    const double nzn = std::sqrt(nz2);
    std::vector<int> poles;
    std::vector<double> zsq, zsign, znd(n, 0.0);
    double znorm2 = 0.0;
    for (int j = 0; j < n; ++j) {
        bool defl = std::fabs(rho) * std::fabs(p->z[j]) * nzn <= thr;
        if (!defl) {
            poles.push_back(j);
            zsq.push_back(p->z[j] * p->z[j]);
            zsign.push_back(p->z[j] > 0 ? 1.0 : -1.0);
            znd[j] = p->z[j];
            znorm2 += p->z[j] * p->z[j];
        }
    }
    const int K = (int)poles.size();
    p->K = K;

    std::vector<int> origin(K);
    std::vector<double> tau(K), a(K);
    if (K > 0) {
        int *d_poles, *d_origin, *d_iters;
        double *d_zsq, *d_zsign, *d_tau, *d_a;
        DCTPLUS_CUDA_TRY(dalloc(&d_poles, K));
        DCTPLUS_CUDA_TRY(dalloc(&d_origin, K));
        DCTPLUS_CUDA_TRY(dalloc(&d_iters, K));
        DCTPLUS_CUDA_TRY(dalloc(&d_zsq, K));
        DCTPLUS_CUDA_TRY(dalloc(&d_zsign, K));
        DCTPLUS_CUDA_TRY(dalloc(&d_tau, K));
        DCTPLUS_CUDA_TRY(dalloc(&d_a, K));
        DCTPLUS_CUDA_TRY(cudaMemcpy(d_poles, poles.data(), sizeof(int) * K, cudaMemcpyHostToDevice));
        DCTPLUS_CUDA_TRY(cudaMemcpy(d_zsq, zsq.data(), sizeof(double) * K, cudaMemcpyHostToDevice));
        DCTPLUS_CUDA_TRY(cudaMemcpy(d_zsign, zsign.data(), sizeof(double) * K, cudaMemcpyHostToDevice));
        int max_iter = o.max_secular_iter > 0 ? o.max_secular_iter : 200;
        k_secular<<<(K * 32 + 127) / 128, 128, 0, s>>>(n, rho, K, d_poles, d_zsq, d_zsign, znorm2,
                                                      p->d_sin, max_iter, d_origin, d_tau, d_a,
                                                      d_iters);
        count_launch();
        DCTPLUS_CUDA_TRY(cudaGetLastError());
        std::vector<int> iters(K);
        DCTPLUS_CUDA_TRY(cudaMemcpy(origin.data(), d_origin, sizeof(int) * K, cudaMemcpyDeviceToHost));
        DCTPLUS_CUDA_TRY(cudaMemcpy(tau.data(), d_tau, sizeof(double) * K, cudaMemcpyDeviceToHost));
        DCTPLUS_CUDA_TRY(cudaMemcpy(a.data(), d_a, sizeof(double) * K, cudaMemcpyDeviceToHost));
        DCTPLUS_CUDA_TRY(cudaMemcpy(iters.data(), d_iters, sizeof(int) * K, cudaMemcpyDeviceToHost));
        cudaFree(d_poles); cudaFree(d_origin); cudaFree(d_iters); cudaFree(d_zsq);
        cudaFree(d_zsign); cudaFree(d_tau); cudaFree(d_a);
        for (int i = 0; i < K; ++i)
            if (iters[i] < 0 || !std::isfinite(tau[i]) || !std::isfinite(a[i]))
                return DCTPLUS_ERR_NOT_CONVERGED;
    }

    // merge root rows and deflated rows by ascending eigenvalue (deflated first on a tie)
    auto lam = [n](int j) { double t = std::sin(M_PI * j / (2.0 * n)); return 4.0 * t * t; };
    struct Row { double val; int kind; int pole; double tau; double a; };
    std::vector<Row> rows;
    rows.reserve(n);
    for (int j = 0; j < n; ++j)
        if (znd[j] == 0.0) rows.push_back({lam(j), 0, j, 0.0, 0.0});
    for (int i = 0; i < K; ++i) rows.push_back({lam(origin[i]) + tau[i], 1, origin[i], tau[i], a[i]});
    std::stable_sort(rows.begin(), rows.end(), [](const Row& x, const Row& y) {
        if (x.val != y.val) return x.val < y.val;
        return x.kind < y.kind;
    });
    p->eig.resize(n); p->row_kind.resize(n); p->row_pole.resize(n);
    p->row_tau.resize(n); p->row_a.resize(n);
    for (int r = 0; r < n; ++r) {
        p->eig[r] = rows[r].val; p->row_kind[r] = rows[r].kind; p->row_pole[r] = rows[r].pole;
        p->row_tau[r] = rows[r].tau; p->row_a[r] = rows[r].a;
    }

    double* d_znd;
    DCTPLUS_CUDA_TRY(dalloc(&d_znd, n));
    DCTPLUS_CUDA_TRY(cudaMemcpy(d_znd, znd.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    DCTPLUS_CUDA_TRY(dalloc(&p->d_row_tau, n));
    DCTPLUS_CUDA_TRY(dalloc(&p->d_row_a, n));
    DCTPLUS_CUDA_TRY(dalloc(&p->d_row_kind, n));
    DCTPLUS_CUDA_TRY(dalloc(&p->d_row_pole, n));
    DCTPLUS_CUDA_TRY(cudaMemcpy(p->d_row_tau, p->row_tau.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    DCTPLUS_CUDA_TRY(cudaMemcpy(p->d_row_a, p->row_a.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    DCTPLUS_CUDA_TRY(cudaMemcpy(p->d_row_kind, p->row_kind.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    DCTPLUS_CUDA_TRY(cudaMemcpy(p->d_row_pole, p->row_pole.data(), sizeof(int) * n, cudaMemcpyHostToDevice));

    const long long nn = (long long)n * n;
    const int blocks_nn = (int)((nn + 255) / 256);
    // Cauchy evaluation for FP32 data with n > 64 (n <= 64 always runs the fused small-n kernels)
    const bool gemm_shape = n > kSmallMax && n % 128 == 0 && n <= kTableMax;
    if (n > kSmallMax) {
        int m = p->cauchy_mode;
        if (m == DCTPLUS_CAUCHY_AUTO) {
            // a measured choice from the autotune cache, if one applies
            const char* cache = o.tune_cache ? o.tune_cache : std::getenv("DCTPLUS_TUNE_CACHE");
            int tm = -1, tf = 0;
            cudaDeviceProp prop;
            if (cache && *cache && cudaGetDeviceProperties(&prop, p->device) == cudaSuccess &&
                tune_lookup(cache, prop.name, n, o.batch_hint > 0 ? o.batch_hint : 4096, &tm, &tf) &&
                ((tm == DCTPLUS_CAUCHY_DENSE && gemm_shape) || (tm == DCTPLUS_CAUCHY_HIER && hier_shape(n) && tf > 0) ||
                 tm == DCTPLUS_CAUCHY_SIMT)) {
                m = tm;
                if (m == DCTPLUS_CAUCHY_HIER && p->far_field == 0) p->far_field = tf;
            } else if (hier_shape(n) && n >= kHierAutoMin) {
                m = DCTPLUS_CAUCHY_HIER;
            } else {
                m = gemm_shape ? DCTPLUS_CAUCHY_DENSE : DCTPLUS_CAUCHY_SIMT;
            }
        }
        if ((m == DCTPLUS_CAUCHY_NFST && n > kF64Max && !nfst_fast_shape(n)) ||
            (m == DCTPLUS_CAUCHY_DENSE && !gemm_shape) ||
            (m == DCTPLUS_CAUCHY_DENSE_GFT && !gemm_shape) ||
            (m == DCTPLUS_CAUCHY_HIER && !hier_shape(n)))
            return DCTPLUS_ERR_UNSUPPORTED;
        p->cauchy_mode = m;
        if (m == DCTPLUS_CAUCHY_HIER && p->far_field == 0) p->far_field = n >= kTreeAutoMin ? 2 : 1;
    }
    const bool want_xt = p->cauchy_mode == DCTPLUS_CAUCHY_DENSE_GFT;
    // W split is also the operand that builds X^T for the comparator beyond the FP64 table size
    const bool want_split = p->cauchy_mode == DCTPLUS_CAUCHY_DENSE || (want_xt && n > kF64Max);
    if (n <= kTableMax) {
        DCTPLUS_CUDA_TRY(dalloc(&p->d_w32, nn));
        if (n <= kF64Max) DCTPLUS_CUDA_TRY(dalloc(&p->d_w64, nn));
        if (want_split) {
            DCTPLUS_CUDA_TRY(dalloc(&p->d_whi, nn));
            DCTPLUS_CUDA_TRY(dalloc(&p->d_wlo, nn));
        }
        k_w_table<<<blocks_nn, 256, 0, s>>>(n, p->d_row_kind, p->d_row_pole, p->d_row_tau,
                                            p->d_row_a, d_znd, p->d_sin, p->d_w32, p->d_w64,
                                            p->d_whi, p->d_wlo);
        count_launch();
    }
    // U^T in FP32 for the small kernels and for lengths without an FFT (n > 64 not a power of two)
    const bool want_ct32 = n <= kSmallMax || ((n & (n - 1)) != 0 && n <= kTableMax);
    if (n <= kF64Max || want_ct32) {
        if (want_ct32) DCTPLUS_CUDA_TRY(dalloc(&p->d_ct32, nn));
        if (n <= kF64Max) DCTPLUS_CUDA_TRY(dalloc(&p->d_ct64, nn));
        k_ct_table<<<blocks_nn, 256, 0, s>>>(n, p->d_sin, p->d_ct32, p->d_ct64);
        count_launch();
    }
    if (want_xt) {
        DCTPLUS_CUDA_TRY(dalloc(&p->d_xthi, nn));
        DCTPLUS_CUDA_TRY(dalloc(&p->d_xtlo, nn));
        if (n <= kF64Max) {
            k_xt_table<<<blocks_nn, 256, 0, s>>>(n, p->d_w64, p->d_ct64, p->d_xthi, p->d_xtlo);
            count_launch();
        } else {
            // X^T = W U^T with the split-TF32 tensor-core GEMM (FP32 accurate), then split
            float *uhi = nullptr, *ulo = nullptr, *xt = nullptr;
            dctplus_status st = DCTPLUS_OK;
            if (dalloc(&uhi, nn) != cudaSuccess || dalloc(&ulo, nn) != cudaSuccess ||
                dalloc(&xt, nn) != cudaSuccess) {
                st = DCTPLUS_ERR_CUDA;
            } else {
                k_u_rows<<<blocks_nn, 256, 0, s>>>(n, p->d_sin, uhi, ulo);
                count_launch();
                st = launch_gemm_tc(p->d_whi, p->d_wlo, n, uhi, ulo, n, xt, n, n, n, n, s, p->device);
                if (st == DCTPLUS_OK) {
                    k_split_table<<<blocks_nn, 256, 0, s>>>(nn, xt, p->d_xthi, p->d_xtlo);
                    count_launch();
                    if (cudaStreamSynchronize(s) != cudaSuccess) st = DCTPLUS_ERR_CUDA;
                }
            }
            cudaFree(uhi);
            cudaFree(ulo);
            cudaFree(xt);
            cudaFree(p->d_whi);
            cudaFree(p->d_wlo);
            p->d_whi = p->d_wlo = nullptr;
            if (st != DCTPLUS_OK) return st;
        }
    }
    DCTPLUS_CUDA_TRY(dalloc(&p->d_gen_pole, n));
    DCTPLUS_CUDA_TRY(dalloc(&p->d_gen_tau, n));
    DCTPLUS_CUDA_TRY(dalloc(&p->d_gen_na, n));
    DCTPLUS_CUDA_TRY(dalloc(&p->d_gen_z, n));
    DCTPLUS_CUDA_TRY(dalloc(&p->d_gen_sin, n + 1));
    k_gen_tables<<<(n + 1 + 255) / 256, 256, 0, s>>>(n, p->d_row_kind, p->d_row_pole, p->d_row_tau,
                                                     p->d_row_a, d_znd, p->d_sin, p->d_gen_pole,
                                                     p->d_gen_tau, p->d_gen_na, p->d_gen_z,
                                                     p->d_gen_sin);
    count_launch();
    DCTPLUS_CUDA_TRY(cudaGetLastError());
    DCTPLUS_CUDA_TRY(cudaStreamSynchronize(s));
    if (p->cauchy_mode == DCTPLUS_CAUCHY_HIER && n > kSmallMax) {
        dctplus_status hs = setup_hier(p, d_znd);
        if (hs != DCTPLUS_OK) { cudaFree(d_znd); return hs; }
    }
    cudaFree(d_znd);

    dctplus_status st = DCTPLUS_OK;
    if (n <= kSmallMax) st = setup_small_tc(p);
    else st = setup_large(p);
    if (st != DCTPLUS_OK) return st;
    if (p->cauchy_mode == DCTPLUS_CAUCHY_NFST && (st = setup_nfst(p)) != DCTPLUS_OK) return st;
    DCTPLUS_CUDA_TRY(cudaDeviceSynchronize());
    return DCTPLUS_OK;
}

}  // namespace dctplus
