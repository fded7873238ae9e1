// The paper's own evaluation of the Cauchy product (Algorithm 1 steps 3-7,
// Sec. 4): cauchy mode DCTPLUS_CAUCHY_NFST, FP64 inside for both dtypes.
//
// With s = z * DCT-II(x), the zero pole's column stays explicit (s_0 / mu_i) and
// the rest of the product is a rational function of x = 1 - mu / 2 whose poles
// are the zeros cos(pi j / n) of U_{n-1}. By Gastinel's proposition and
// Lemma 4.3 (d_n cancelled, so never formed) it equals a sine series over
// sin(n theta), mu = 2 - 2 cos(theta) (eq. trigo):
//   h_j = (-1)^(j+1) s_j / sin(pi j / n)
//   c_l = 2 sum_{j=1}^{n-1} h_j sin(pi l j / n)                      (DST-I)
//   p_i = s_0 / mu_i - 1/2 sum_l c_l sin(l theta_i) / sin(n theta_i)
//   y_i = -a_i p_i.
// Roots outside (0, 4) (the root the paper isolates) are plain sums; deflated
// rows are the DCT coefficient.
//
// Two kernels compute it:
//  * k_nfst_fast (n a power of two, 16 <= n <= 8192) is the O(n log n) route
//    of Algorithm 1. One CTA per signal keeps everything in one shared-memory
//    buffer of n complex doubles:
//      - the DCT-II by Makhoul's reordering and a complex FFT of length n/2;
//      - the DST-I by a complex FFT of length n/2 on a symmetrised sequence
//        (even outputs read directly, odd outputs as a prefix sum);
//      - the sine series at the n root angles by a type-2 nonuniform sine
//        transform. The coefficients are divided by the Fourier transform of a
//        Kaiser-Bessel window, a DST-I of length 2n (same method) puts the
//        series on the grid theta_k = pi k / 2n (oversampled twice), and each
//        root sums 16 grid values times the window, with weights fixed per plan.
//  * k_nfst_route (any other n <= 1024) does the same arithmetic by direct sums:
//    the DCT-II and DST-I as matrix products, the series by a Clenshaw recurrence
//    per root. That is O(n^2) per signal.
// The route's accuracy degrades like eps / |sin(n theta)| when a root sits next
// to a pole, which is why the tensor-core and hierarchical modes use the
// pole + offset form instead.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace dctplus {

constexpr int kNfstFastMin = 16;
constexpr int kNfstFastMax = 8192;
constexpr int kNfstTaps = 16;      // window width in grid steps
constexpr int kNfstMaxDense = 4;   // rows whose root lies outside (0, 4): at most one in exact arithmetic

bool nfst_fast_shape(int n) { return n >= kNfstFastMin && n <= kNfstFastMax && (n & (n - 1)) == 0; }

// Rows with a root outside (0, 4), summed directly by the fast kernel.
struct NfstDenseRows {
    int count;
    double a[kNfstMaxDense];
};

// Plan tables of k_nfst_fast. Device blobs:
//   f: znd[n] | hfac[n] | dec[n] | arow[n] | wt[kNfstTaps][n] | dinv[dense.count][n]
//   i: kind[n] | k0[n] | drow[n]
// znd_j = z_j (0 where deflated); hfac_j = (-1)^(j+1) znd_j / sin(pi j / n);
// dec_l = 2 hg / phi^(l) (the DST-I's factor 2 and the window's deconvolution,
// hg = pi / 2n the grid step); for a root row r: arow_r = -a_r / mu_r,
// wt[t][r] = a_r / (2 sin(n theta_r)) * phi(theta_r - (k0_r + t) hg), kind 1;
// a dense row has kind 2 and k0 = its index d in the dense list, whose
// reciprocal gaps dinv[d][j] = 1 / (mu - lambda_j) come from the pole + offset
// form; drow_j is the row of the deflated pole j, else -1.
struct NfstFastTables {
    double* f = nullptr;
    int* i = nullptr;
    NfstDenseRows dense{};
};

void free_nfst(NfstFastTables* t) {
    if (!t) return;
    if (t->f) cudaFree(t->f);
    if (t->i) cudaFree(t->i);
    delete t;
}

namespace {

// I0 by its power series sum_k ((x/2)^k / k!)^2 (all terms positive, so the
// partial sums converge without cancellation for every x used here, x < 40).
double bessel_i0(double x) {
    const double q = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 1000; ++k) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

// The root angle theta = 2 atan(sqrt(mu / (4 - mu))) of row r with mu = lambda_pole + tau;
// 4 - mu is formed from cos^2 so that it keeps its digits near 4. Returns false when the
// root lies outside (0, 4).
bool root_angle(dctplus_plan_t p, int r, double* mu_out, double* theta) {
    const int n = p->n;
    const double half = M_PI * p->row_pole[r] / (2.0 * n);
    const double sh = std::sin(half), ch = std::cos(half);
    const double mu = 4.0 * sh * sh + p->row_tau[r];
    const double mc = 4.0 * ch * ch - p->row_tau[r];
    *mu_out = mu;
    if (!(mu > 0.0 && mc > 0.0)) return false;
    *theta = 2.0 * std::atan2(std::sqrt(mu), std::sqrt(mc));
    return true;
}

std::vector<double> nondeflated_z(dctplus_plan_t p) {
    std::vector<double> znd(p->z);
    for (int r = 0; r < p->n; ++r)
        if (p->row_kind[r] == 0) znd[p->row_pole[r]] = 0.0;
    return znd;
}

dctplus_status setup_nfst_fast(dctplus_plan_t p) {
    const int n = p->n;
    // Kaiser-Bessel window of kNfstTaps grid steps, phi(x) = I0(beta sqrt(1 - (x/alpha)^2)),
    // with the shape parameter of Beatty, Nishimura and Pauly (IEEE TMI 2005) for
    // oversampling ratio 2: beta = pi sqrt((w/2)^2 (2 - 1/2)^2 - 0.8). Its Fourier transform
    // is 2 alpha sinh(sqrt(beta^2 - (alpha xi)^2)) / sqrt(beta^2 - (alpha xi)^2). Both are
    // divided by I0(beta), which cancels in the route.
    const double hg = M_PI / (2.0 * n);
    const double alpha = 0.5 * kNfstTaps * hg;
    const double half_w = 0.5 * kNfstTaps;
    const double beta = M_PI * std::sqrt(half_w * half_w * 2.25 - 0.8);
    const double i0b = bessel_i0(beta);
    auto window = [&](double xv) {
        const double t = 1.0 - (xv / alpha) * (xv / alpha);
        return t > 0.0 ? bessel_i0(beta * std::sqrt(t)) / i0b : 0.0;
    };
    auto window_hat = [&](double xi) {
        const double q = std::sqrt(beta * beta - (alpha * xi) * (alpha * xi));  // alpha xi < 4 pi < beta
        return 2.0 * alpha * std::sinh(q) / q / i0b;
    };
    std::vector<double> f((size_t)(4 + kNfstTaps + kNfstMaxDense) * n, 0.0);
    double* znd = f.data();
    double* hfac = znd + n;
    double* dec = hfac + n;
    double* arow = dec + n;
    double* wt = arow + n;
    std::vector<int> iv(3 * (size_t)n, 0);
    int* kind = iv.data();
    int* k0 = kind + n;
    int* drow = k0 + n;
    const std::vector<double> z = nondeflated_z(p);
    for (int j = 0; j < n; ++j) {
        znd[j] = z[j];
        drow[j] = -1;
    }
    for (int j = 1; j < n; ++j) hfac[j] = ((j & 1) ? 1.0 : -1.0) * znd[j] / std::sin(M_PI * j / n);
    for (int l = 1; l < n; ++l) dec[l] = 2.0 * hg / window_hat((double)l);
    NfstFastTables* t = new NfstFastTables();
    for (int r = 0; r < n; ++r) {
        if (p->row_kind[r] == 0) {
            kind[r] = 0;
            drow[p->row_pole[r]] = r;
            continue;
        }
        double mu = 0.0, th = 0.0;
        if (root_angle(p, r, &mu, &th)) {
            kind[r] = 1;
            const int kb = (int)std::ceil(th / hg - half_w);
            k0[r] = kb;
            arow[r] = -p->row_a[r] / mu;
            const double br = p->row_a[r] / (2.0 * std::sin(n * th));
            for (int q = 0; q < kNfstTaps; ++q) wt[(size_t)q * n + r] = br * window(th - (kb + q) * hg);
        } else {
            if (t->dense.count == kNfstMaxDense) {
                delete t;
                return DCTPLUS_ERR_UNSUPPORTED;
            }
            const int d = t->dense.count++;
            kind[r] = 2;
            k0[r] = d;
            t->dense.a[d] = p->row_a[r];
            // mu - lambda_j = tau - (lambda_j - lambda_p), the difference of eigenvalues as
            // 4 sin(pi (j + p) / 2n) sin(pi (j - p) / 2n)
            double* dinv = wt + (size_t)(kNfstTaps + d) * n;
            const int pole = p->row_pole[r];
            for (int j = 0; j < n; ++j) {
                const int m = std::min(j + pole, 2 * n - j - pole);  // same sine, argument <= pi / 2
                dinv[j] = 1.0 / (p->row_tau[r] - 4.0 * std::sin(M_PI * m / (2.0 * n)) *
                                                      std::sin(M_PI * (j - pole) / (2.0 * n)));
            }
        }
    }
    f.resize((size_t)(4 + kNfstTaps + t->dense.count) * n);
    p->nfst = t;  // owned by the plan from here on (freed with its tables)
    DCTPLUS_CUDA_TRY(cudaMalloc((void**)&t->f, sizeof(double) * f.size()));
    DCTPLUS_CUDA_TRY(cudaMalloc((void**)&t->i, sizeof(int) * iv.size()));
    DCTPLUS_CUDA_TRY(cudaMemcpy(t->f, f.data(), sizeof(double) * f.size(), cudaMemcpyHostToDevice));
    DCTPLUS_CUDA_TRY(cudaMemcpy(t->i, iv.data(), sizeof(int) * iv.size(), cudaMemcpyHostToDevice));
    return DCTPLUS_OK;
}

}  // namespace

// per-row data of the direct route (FP64): 2 cos(theta), sin(theta), 1 / sin(n theta), mu
struct NfstRow {
    double c2, sn, isn, mu;
};

dctplus_status setup_nfst(dctplus_plan_t p) {
    const int n = p->n;
    if (nfst_fast_shape(n)) return setup_nfst_fast(p);
    if (n > kF64Max || !p->d_ct64) return DCTPLUS_ERR_UNSUPPORTED;
    std::vector<int> kind(n);
    std::vector<NfstRow> rows(n);
    const std::vector<double> znd = nondeflated_z(p);
    for (int r = 0; r < n; ++r) {
        rows[r] = {0.0, 0.0, 0.0, 0.0};
        if (p->row_kind[r] == 0) {
            kind[r] = 0;
            continue;
        }
        double mu = 0.0, th = 0.0;
        const bool inside = root_angle(p, r, &mu, &th);
        rows[r].mu = mu;
        if (inside) {
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

// ------------------------------------------------------------------ fast route

namespace {

struct NfstFastArgs {
    const double* S;  // sin(pi m / 2n), m = 0..n
    const double* f;  // NfstFastTables::f
    const int* iv;    // NfstFastTables::i
    NfstDenseRows dense;
    double scale0, scale;  // orthonormal DCT-II factors sqrt(1/n), sqrt(2/n)
};

// Threads per CTA: n / 16 between one warp and 512; the launch bound asks for 512 threads per SM,
// so 128 registers at most per thread.
__host__ __device__ constexpr int nfst_threads(int n) { return n >= 8192 ? 512 : (n / 16 > 32 ? n / 16 : 32); }
__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }

// Complex slot i of the shared buffer, one pad slot every 8 (keeps the strided
// FFT passes off a single bank group).
__device__ __forceinline__ int cpad(int i) { return i + (i >> 3); }

// Real element r of the buffer read as packed complex values (r = 2 slot + part).
__device__ __forceinline__ double& packed_re(double2* buf, int r) {
    return reinterpret_cast<double*>(&buf[cpad(r >> 1)])[r & 1];
}

// (cos, sin) of pi m / 2n for 0 <= m < 2n from the table S[m] = sin(pi m / 2n), m <= n.
__device__ __forceinline__ double2 cis_half(int m, int n, const double* __restrict__ S) {
    return m <= n ? make_double2(S[n - m], S[m]) : make_double2(-S[m - n], S[2 * n - m]);
}

__device__ __forceinline__ int bitrev(int k, int bits) { return (int)(__brev((unsigned)k) >> (32 - bits)); }

// R radix-2 decimation-in-frequency stages, half sizes 2^lgh, 2^(lgh-1), ...,
// of a forward (exp(-i ...)) complex FFT of length 2^lgL, in place; each thread
// takes groups of 2^R points that the R stages combine only among themselves.
template <int R>
__device__ __forceinline__ void fft_stages(double2* buf, int lgL, int lgh, int n, int lg2n,
                                           const double* __restrict__ S) {
    constexpr int P = 1 << R;
    const int lgs = lgh - (R - 1);  // distance between a group's points: 2^lgs
    const int s = 1 << lgs;
    const int groups = 1 << (lgL - R);
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {
        const int base = ((g >> lgs) << (lgh + 1)) + (g & (s - 1));
        double2 v[P];
#pragma unroll
        for (int q = 0; q < P; ++q) v[q] = buf[cpad(base + q * s)];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int lghi = lgh - i;   // this stage pairs points 2^lghi apart
            const int qs = P >> (i + 1);
#pragma unroll
            for (int q = 0; q < P; ++q) {
                if (q & qs) continue;
                const int t = (base + q * s) & ((2 << lghi) - 1);  // offset in its block, < 2^lghi
                const double2 a = v[q], b = v[q + qs];
                v[q] = make_double2(a.x + b.x, a.y + b.y);
                const double2 d = make_double2(a.x - b.x, a.y - b.y);
                const double2 w = cis_half(t << (lg2n - lghi), n, S);  // angle pi t / 2^lghi
                v[q + qs] = make_double2(d.x * w.x + d.y * w.y, d.y * w.x - d.x * w.y);
            }
        }
#pragma unroll
        for (int q = 0; q < P; ++q) buf[cpad(base + q * s)] = v[q];
    }
}

// Forward complex FFT of length 2^lgL in place; output k at slot bitrev(k).
__device__ void fft_forward(double2* buf, int lgL, int n, int lg2n, const double* __restrict__ S) {
    int lgh = lgL - 1;
    for (int rem = lgL; rem > 0;) {
        if (rem >= 3) {
            fft_stages<3>(buf, lgL, lgh, n, lg2n, S);
            lgh -= 3;
            rem -= 3;
        } else if (rem == 2) {
            fft_stages<2>(buf, lgL, lgh, n, lg2n, S);
            lgh -= 2;
            rem -= 2;
        } else {
            fft_stages<1>(buf, lgL, lgh, n, lg2n, S);
            lgh -= 1;
            rem -= 1;
        }
        __syncthreads();
    }
}

// Bin k of the forward DFT of a real sequence of length 2L, from the complex FFT Z
// of length L of its packed pairs: Y_k = E_k + exp(-i a) O_k with
// E_k = (Z_k + conj Z_{L-k}) / 2, O_k = (Z_k - conj Z_{L-k}) / 2i, a = pi k / L,
// w = (cos a, sin a).
__device__ __forceinline__ double2 real_bin(double2 zk, double2 zm, double2 w) {
    const double ex = 0.5 * (zk.x + zm.x), ey = 0.5 * (zk.y - zm.y);
    const double ox = 0.5 * (zk.y + zm.y), oy = -0.5 * (zk.x - zm.x);
    return make_double2(ex + w.x * ox + w.y * oy, ey + w.x * oy - w.y * ox);
}

// Exclusive prefix sum of v over the block's threads in thread order.
__device__ __forceinline__ double block_exclusive_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) red[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        double w = lane < nw ? red[lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nw) red[lane] = w;
    }
    __syncthreads();
    const double out = (warp > 0 ? red[warp - 1] : 0.0) + incl - v;
    __syncthreads();
    return out;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    __syncthreads();
    return t;
}

template <typename T, int N>
__global__ void __launch_bounds__(nfst_threads(N), 512 / nfst_threads(N)) k_nfst_fast(const T* __restrict__ x, int64_t ldx,
                                                               T* __restrict__ y, int64_t ldy,
                                                               int64_t batch, NfstFastArgs g) {
    constexpr int NT = nfst_threads(N);
    constexpr int L1 = N / 2;                 // complex FFT length of the DCT-II and the DST-I
    constexpr int LG1 = ilog2c(L1), LGN = ilog2c(N), LG2N = LGN + 1;
    constexpr int C1 = (L1 + NT - 1) / NT;    // bins per thread of the length-n transforms
    constexpr int CG = (N + NT - 1) / NT;     // bins per thread of the grid transform
    extern __shared__ double2 nbuf[];
    double* nre = reinterpret_cast<double*>(nbuf);  // the buffer as plain reals (grid values)
    __shared__ double red[NT / 32];
    __shared__ double dense_sum[kNfstMaxDense];
    __shared__ double s0_sh, r0_sh;
    const int tid = threadIdx.x;
    const double* __restrict__ S = g.S;
    const double* __restrict__ znd = g.f;
    const double* __restrict__ hfac = znd + N;
    const double* __restrict__ dec = hfac + N;
    const double* __restrict__ arow = dec + N;
    const double* __restrict__ wt = arow + N;
    const double* __restrict__ dinv = wt + (size_t)kNfstTaps * N;
    const int* __restrict__ kind = g.iv;
    const int* __restrict__ k0 = kind + N;
    const int* __restrict__ drow = k0 + N;
    const int nd = g.dense.count;

    for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
        const T* xb = x + b * ldx;
        T* yb = y + b * ldy;
        // Algorithm 1 step 1, DCT-II: Makhoul's order v_q = x_2q, v_{n-1-q} = x_{2q+1},
        // packed as n/2 complex values v_2m + i v_2m+1.
        for (int j = tid; j < N; j += NT) {
            const int q = (j & 1) ? N - 1 - (j >> 1) : (j >> 1);
            packed_re(nbuf, q) = (double)xb[j];
        }
        __syncthreads();
        fft_forward(nbuf, LG1, N, LG2N, S);

        // X_k = c_k Re(exp(-i pi k / 2n) V_k), X_{n-k} = -c_k Im(...), k = 0..n/2, where V is the
        // length-n DFT of v. Each coefficient j then gives s_j = z_j X_j (step 2), the deflated
        // rows (y = X_j), the dense rows' sums, and h_j for the DST-I of steps 4-5, which enters
        // it through the symmetrised sequence u_j = sin(pi j / n)(h_j + h_{n-j}) + (h_j - h_{n-j}) / 2.
        double u[C1][2];
        double dacc[kNfstMaxDense];
#pragma unroll
        for (int d = 0; d < kNfstMaxDense; ++d) dacc[d] = 0.0;
        double u_half = 0.0;  // u_{n/2}, from bin n/2 (thread 0)
        auto coefficient = [&](int j, double X) -> double {
            const double sj = znd[j] * X;
            if (j == 0) s0_sh = sj;
            const int dr = drow[j];
            if (dr >= 0) yb[dr] = (T)X;
#pragma unroll
            for (int d = 0; d < kNfstMaxDense; ++d)
                if (d < nd) dacc[d] += sj * dinv[(size_t)d * N + j];
            return hfac[j] * X;
        };
#pragma unroll
        for (int i = 0; i < C1; ++i) {
            const int k = tid * C1 + i;
            u[i][0] = u[i][1] = 0.0;
            if (k < L1) {
                const double2 zk = nbuf[cpad(bitrev(k, LG1))];
                const double2 zm = nbuf[cpad(bitrev((L1 - k) & (L1 - 1), LG1))];
                const double2 V = real_bin(zk, zm, cis_half(4 * k, N, S));
                const double2 w = cis_half(k, N, S);
                const double qx = w.x * V.x + w.y * V.y, qy = w.x * V.y - w.y * V.x;
                if (k == 0) {
                    coefficient(0, g.scale0 * qx);
                    // bin n/2: V_{n/2} = Re Z_0 - Im Z_0, rotated by pi / 4
                    const double Xh = g.scale * S[N / 2] * (zk.x - zk.y);
                    u_half = 2.0 * coefficient(L1, Xh);
                } else {
                    const double hk = coefficient(k, g.scale * qx);
                    const double hm = coefficient(N - k, -g.scale * qy);
                    const double sk = S[2 * k];
                    u[i][0] = sk * (hk + hm) + 0.5 * (hk - hm);
                    u[i][1] = sk * (hk + hm) - 0.5 * (hk - hm);
                }
            }
        }
#pragma unroll
        for (int d = 0; d < kNfstMaxDense; ++d) {
            if (d < nd) {  // uniform over the block
                const double t = block_sum(dacc[d], red);
                if (tid == 0) dense_sum[d] = t;
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < C1; ++i) {
            const int k = tid * C1 + i;
            if (k < L1) {
                packed_re(nbuf, k) = u[i][0];  // u_0 = 0
                if (k > 0) packed_re(nbuf, N - k) = u[i][1];
            }
        }
        if (tid == 0) packed_re(nbuf, L1) = u_half;
        __syncthreads();
        fft_forward(nbuf, LG1, N, LG2N, S);

        // DST-I: with U the length-n DFT of u, sum_j h_j sin(pi l j / n) is -Im U_{l/2} for even l
        // and Re U_0 / 2 + Re U_1 + ... + Re U_{(l-1)/2} for odd l. Then the coefficients are
        // deconvolved (d_l = dec_l F_l) and symmetrised again for the grid's DST-I of length 2n:
        // g_l = (sin(pi l / 2n) + 1/2) d_l, g_{2n-l} = (sin(pi l / 2n) - 1/2) d_l, g_0 = g_n = 0.
        {
            double fe[C1], rr[C1];
            double tsum = 0.0;
#pragma unroll
            for (int i = 0; i < C1; ++i) {
                const int k = tid * C1 + i;
                fe[i] = rr[i] = 0.0;
                if (k < L1) {
                    const double2 zk = nbuf[cpad(bitrev(k, LG1))];
                    const double2 zm = nbuf[cpad(bitrev((L1 - k) & (L1 - 1), LG1))];
                    const double2 Y = real_bin(zk, zm, cis_half(4 * k, N, S));
                    fe[i] = -Y.y;
                    rr[i] = Y.x;
                    tsum += Y.x;
                }
            }
            if (tid == 0) r0_sh = rr[0];
            double run = block_exclusive_sum(tsum, red);
            const double r0h = 0.5 * r0_sh;
#pragma unroll
            for (int i = 0; i < C1; ++i) {
                const int k = tid * C1 + i;
                if (k < L1) {
                    run += rr[i];
                    if (k > 0) {
                        const int l = 2 * k;
                        const double dl = dec[l] * fe[i];
                        packed_re(nbuf, l) = (S[l] + 0.5) * dl;
                        packed_re(nbuf, 2 * N - l) = (S[l] - 0.5) * dl;
                    }
                    const int l = 2 * k + 1;
                    const double dl = dec[l] * (run - r0h);
                    packed_re(nbuf, l) = (S[l] + 0.5) * dl;
                    packed_re(nbuf, 2 * N - l) = (S[l] - 0.5) * dl;
                }
            }
            if (tid == 0) {
                packed_re(nbuf, 0) = 0.0;
                packed_re(nbuf, N) = 0.0;
            }
        }
        __syncthreads();
        fft_forward(nbuf, LGN, N, LG2N, S);

        // Grid values G_k = sum_l d_l sin(pi l k / 2n), k = 0..2n, by the same reading of the
        // length-2n DFT, written as plain reals in natural order.
        {
            double ge[CG], gr[CG];
            double tsum = 0.0;
#pragma unroll
            for (int i = 0; i < CG; ++i) {
                const int k = tid * CG + i;
                ge[i] = gr[i] = 0.0;
                if (k < N) {
                    const double2 zk = nbuf[cpad(bitrev(k, LGN))];
                    const double2 zm = nbuf[cpad(bitrev((N - k) & (N - 1), LGN))];
                    const double2 Y = real_bin(zk, zm, cis_half(2 * k, N, S));
                    ge[i] = -Y.y;
                    gr[i] = Y.x;
                    tsum += Y.x;
                }
            }
            if (tid == 0) r0_sh = gr[0];
            double run = block_exclusive_sum(tsum, red);
            const double r0h = 0.5 * r0_sh;
#pragma unroll
            for (int i = 0; i < CG; ++i) {
                const int k = tid * CG + i;
                if (k < N) {
                    run += gr[i];
                    nre[2 * k] = ge[i];
                    nre[2 * k + 1] = run - r0h;
                }
            }
            if (tid == 0) nre[2 * N] = 0.0;
        }
        __syncthreads();

        // Steps 6-7: the series at theta_r from the 16 grid values around it (odd about k = 0
        // and k = 2n), plus the zero pole's column, already scaled by -a_r.
        const double s0 = s0_sh;
        for (int r = tid; r < N; r += NT) {
            const int kd = kind[r];
            if (kd == 0) continue;
            double out;
            if (kd == 1) {
                const int kb = k0[r];
                double acc = arow[r] * s0;
#pragma unroll
                for (int t = 0; t < kNfstTaps; ++t) {
                    const int k = kb + t;
                    const double gv = k < 0 ? -nre[-k] : (k > 2 * N ? -nre[4 * N - k] : nre[k]);
                    acc = fma(wt[(size_t)t * N + r], gv, acc);
                }
                out = acc;
            } else {
                const int d = k0[r];
                out = -g.dense.a[d] * dense_sum[d];
            }
            yb[r] = (T)out;
        }
        __syncthreads();
    }
}

template <typename T, int N>
dctplus_status launch_nfst_fast_n(dctplus_plan_t p, const T* x, int64_t ldx, T* y, int64_t ldy,
                                  int64_t batch, cudaStream_t st) {
    constexpr int NT = nfst_threads(N);
    const size_t smem = sizeof(double2) * (size_t)(N + (N - 1) / 8 + 1);
    // per device, once: the shared-memory opt-in and the resident CTAs per SM it allows
    static int per_sm_dev[64] = {};
    int& per_sm = per_sm_dev[p->device & 63];
    if (per_sm == 0) {
        DCTPLUS_CUDA_TRY(cudaFuncSetAttribute(k_nfst_fast<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        int r = 0;
        DCTPLUS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_nfst_fast<T, N>, NT, smem));
        per_sm = std::max(r, 1);
    }
    int sms = 0;
    DCTPLUS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    const int64_t grid = std::min<int64_t>(batch, (int64_t)std::max(sms, 1) * per_sm);
    NfstFastArgs a;
    a.S = p->d_sin;
    a.f = p->nfst->f;
    a.iv = p->nfst->i;
    a.dense = p->nfst->dense;
    a.scale0 = std::sqrt(1.0 / N);
    a.scale = std::sqrt(2.0 / N);
    k_nfst_fast<T, N><<<(unsigned)grid, NT, smem, st>>>(x, ldx, y, ldy, batch, a);
    // FP64 arithmetic counted as: 10 flops per radix-2 butterfly of the three FFTs (n/2, n/2,
    // n points), about 30 per bin of the three unpacking steps, 32 per root for the window sum.
    const double lg = std::log2((double)N);
    const double per_signal = 10.0 * (2.0 * (N / 4.0) * (lg - 1.0) + (N / 2.0) * lg) + 30.0 * 2.0 * N + 32.0 * N;
    note_launch(st, "k_nfst_fast", 2.0 * sizeof(T) * (double)batch * N, per_signal * (double)batch);
    DCTPLUS_CUDA_TRY(cudaGetLastError());
    return DCTPLUS_OK;
}

template <typename T>
dctplus_status launch_nfst_fast(dctplus_plan_t p, const T* x, int64_t ldx, T* y, int64_t ldy, int64_t batch,
                                cudaStream_t st) {
    switch (p->n) {
        case 16: return launch_nfst_fast_n<T, 16>(p, x, ldx, y, ldy, batch, st);
        case 32: return launch_nfst_fast_n<T, 32>(p, x, ldx, y, ldy, batch, st);
        case 64: return launch_nfst_fast_n<T, 64>(p, x, ldx, y, ldy, batch, st);
        case 128: return launch_nfst_fast_n<T, 128>(p, x, ldx, y, ldy, batch, st);
        case 256: return launch_nfst_fast_n<T, 256>(p, x, ldx, y, ldy, batch, st);
        case 512: return launch_nfst_fast_n<T, 512>(p, x, ldx, y, ldy, batch, st);
        case 1024: return launch_nfst_fast_n<T, 1024>(p, x, ldx, y, ldy, batch, st);
        case 2048: return launch_nfst_fast_n<T, 2048>(p, x, ldx, y, ldy, batch, st);
        case 4096: return launch_nfst_fast_n<T, 4096>(p, x, ldx, y, ldy, batch, st);
        case 8192: return launch_nfst_fast_n<T, 8192>(p, x, ldx, y, ldy, batch, st);
        default: return DCTPLUS_ERR_UNSUPPORTED;
    }
}

}  // namespace

template <typename T>
dctplus_status launch_nfst(dctplus_plan_t p, const T* x, int64_t ldx, T* y, int64_t ldy, int64_t batch,
                           cudaStream_t st) {
    const int n = p->n;
    if (batch <= 0) return DCTPLUS_OK;
    if (p->nfst) return launch_nfst_fast<T>(p, x, ldx, y, ldy, batch, st);
    if (!p->d_nfst_rows || n > kF64Max) return DCTPLUS_ERR_UNSUPPORTED;
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
