// Hierarchical evaluation of the Cauchy product of Theorem 3.1 (the fast
// matrix-vector product Theorem 3.2 relies on, in the Gerasoulis /
// fast-multipole family), for a batch of signals.
//
// The product is y_r = sum_j W_rj s_j with W_rj = -a_r z_j / (mu_r - lambda_j)
// (root rows) or e_j (deflated rows), s = U^T x. Write lambda_j = 2 - 2 cos th_j
// with th_j = pi j / n (uniform) and mu_r = 2 - 2 cos ph_r. Then
//   1 / (mu - lambda) = 1 / (2 cos th - 2 cos ph),
// a kernel of (ph, th) that is analytic away from th = +-ph, so Chebyshev
// interpolation in th over a box of width h is accurate for targets at least
// one box away (convergence factor 3 + sqrt(8) per degree). Sources are
// uniform in th, so equal th-boxes ("leaves") of 64 sources each are
// balanced; targets interlace the sources (Lemma 4.1), about 64 per leaf.
//
//   near field  targets of leaf I against sources of leaves I-1, I, I+1: exact
//               entries of W, a band matrix applied on the tensor cores with
//               the split-TF32 GEMM (each 128-row output tile contracts a
//               K window of s against a compact [n x Kw] slab of W entries);
//   far field   every other source, through Chebyshev interpolation of degree
//               R in both variables at the leaf level: P2M (per leaf, the
//               sources' z-weighted interpolation coefficients, CUDA cores),
//               then one dense product with the kernel sampled at the leaf
//               nodes of every well-separated leaf pair (target leaf I,
//               source leaf J, |I - J| >= 2), a [nleaf R x nleaf R] matrix on
//               the tensor cores (split-TF32 GEMM), then L2P (-a folded into
//               the weights, CUDA cores) added into y. A single level with a
//               dense leaf-to-leaf operator trades a multilevel tree's O(n)
//               translation work for (12 n / 64)^2 tensor-core multiply-adds
//               per signal, fewer than the dense product's n^2 by (64 / 12)^2,
//               and needs no barriers between tree levels.
// Roots outside [0, 4] (at most the largest for rho > 0 or the smallest for
// rho < 0; the paper's pre-processing isolates the same root) have no real
// angle; their rows are dense dot products, formed as per-leaf partial sums
// by P2M and summed by L2P.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace dctplus {

constexpr int kLeaf = 64;
constexpr int kR = 12;  // Chebyshev degree of the far-field expansions

struct HierTables {
    int nleaf = 0, Kw = 0;
    int nc = 0, ncp = 0;         // leaf coefficients nleaf R, padded to a multiple of 128
    std::vector<int> kbeg;       // per 128-row output tile: first source of the K window
    float* slab_hi = nullptr;    // n x Kw
    float* slab_lo = nullptr;
    float* zf = nullptr;         // n: z_j (0 where deflated)
    float* tq = nullptr;         // 64 x R: S_a at the 64 source positions of any leaf
    float* pna = nullptr;        // n: -a_r for far-field targets, 0 otherwise
    float* wl = nullptr;         // R x n: L2P weights -a_r S_a(u_r) (0 for other rows)
    int* row_leaf = nullptr;     // n
    float* kf_hi = nullptr;      // ncp x ncp: leaf-to-leaf kernel samples, TF32 hi
    float* kf_lo = nullptr;      //            and lo (zero for near pairs and padding)
    int nout = 0;
    int out_row[2] = {-1, -1};
    float* out_w = nullptr;      // nout x n dense rows
};

// round to TF32 (10 explicit mantissa bits), nearest-even; finite inputs
static float tf32_host(float v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    u = (u + 0xFFFu + ((u >> 13) & 1u)) & ~0x1FFFu;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// Lagrange basis polynomial a on the degree-R Chebyshev nodes of [-1, 1], at u
static double cheb_lagrange(int a, double u) {
    double ta = std::cos((2 * a + 1) * M_PI / (2.0 * kR));
    double v = 1.0;
    for (int b = 0; b < kR; ++b) {
        if (b == a) continue;
        double tb = std::cos((2 * b + 1) * M_PI / (2.0 * kR));
        v *= (u - tb) / (ta - tb);
    }
    return v;
}

static double cheb_node(int a) { return std::cos((2 * a + 1) * M_PI / (2.0 * kR)); }

// W entry of a root row r (origin pole p, offset tau, normalisation a) at source j
static double w_entry(int n, int p, double tau, double a, double zj, int j) {
    if (zj == 0.0) return 0.0;
    double m = j + p;
    if (m > 2.0 * n - m) m = 2.0 * n - m;
    double d = 4.0 * std::sin(M_PI * m / (2.0 * n)) * std::sin(M_PI * (j - p) / (2.0 * n));
    return -a * zj / (tau - d);
}

__global__ void k_band_slab(int n, int Kw, const int* kbeg_tile, const int* row_kind,
                            const int* row_pole, const double* row_tau, const double* row_a,
                            const double* znd, const int* row_leaf, const double* S, float* hi,
                            float* lo) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * Kw) return;
    int r = (int)(idx / Kw), kk = (int)(idx % Kw);
    int j = kbeg_tile[r / 128] + kk;
    double w = 0.0;
    int lr = row_leaf[r];
    if (lr >= 0 && j >= 0 && j < n && abs(j / kLeaf - lr) <= 1) {
        if (row_kind[r] == 0) {
            w = (j == row_pole[r]) ? 1.0 : 0.0;
        } else if (znd[j] != 0.0) {
            int p = row_pole[r];
            int m = j + p;
            if (m > 2 * n - m) m = 2 * n - m;
            int q = j - p;
            double d = 4.0 * S[m] * (q >= 0 ? S[q] : -S[-q]);
            w = -row_a[r] * znd[j] / (row_tau[r] - d);
        }
    }
    float h = ptx::tf32_round((float)w);
    hi[idx] = h;
    lo[idx] = ptx::tf32_round((float)(w - (double)h));
}

void free_hier(HierTables* h) {
    if (!h) return;
    void* ptrs[] = {h->slab_hi, h->slab_lo, h->zf, h->tq, h->pna, h->wl, h->row_leaf,
                    h->kf_hi, h->kf_lo, h->out_w};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete h;
}

bool hier_shape(int n) { return n >= 4 * kLeaf && (n & (n - 1)) == 0 && n <= kMaxN; }

dctplus_status setup_hier(dctplus_plan_t p, const double* d_znd) {
    const int n = p->n;
    if (!hier_shape(n)) return DCTPLUS_ERR_UNSUPPORTED;
    HierTables* h = new HierTables();
    p->hier = h;
    h->nleaf = n / kLeaf;
    const int nleaf = h->nleaf;
    const double hleaf = M_PI / nleaf;  // th-width of a leaf

    // z with deflated entries zero (host)
    std::vector<double> znd(n, 0.0);
    {
        std::vector<char> defl(n, 0);
        for (int r = 0; r < n; ++r)
            if (p->row_kind[r] == 0) defl[p->row_pole[r]] = 1;
        for (int j = 0; j < n; ++j) znd[j] = defl[j] ? 0.0 : p->z[j];
    }

    // target angles and leaves; rows whose eigenvalue lies outside [0, 4] are dense rows
    std::vector<int> row_leaf(n);
    std::vector<double> ph(n, 0.0);
    for (int r = 0; r < n; ++r) {
        double mu = p->eig[r];
        if (p->row_kind[r] == 0) {
            ph[r] = M_PI * p->row_pole[r] / n;
        } else if (mu < 0.0 || mu > 4.0) {
            if (h->nout >= 2) return DCTPLUS_ERR_UNSUPPORTED;
            h->out_row[h->nout++] = r;
            row_leaf[r] = -1;
            continue;
        } else {
            ph[r] = 2.0 * std::asin(std::sqrt(mu) / 2.0);
        }
        int lf = (int)std::floor(ph[r] / hleaf);
        row_leaf[r] = std::min(std::max(lf, 0), nleaf - 1);
    }

    // band windows per 128-row output tile
    const int ntile = n / 128;
    h->kbeg.assign(ntile, 0);
    int kw = 0;
    for (int t = 0; t < ntile; ++t) {
        int lmin = nleaf, lmax = -1;
        for (int r = 128 * t; r < 128 * t + 128; ++r) {
            if (row_leaf[r] < 0) continue;
            lmin = std::min(lmin, row_leaf[r]);
            lmax = std::max(lmax, row_leaf[r]);
        }
        if (lmax < 0) { lmin = lmax = 0; }
        int k0 = (lmin - 1) * kLeaf, k1 = (lmax + 2) * kLeaf;
        h->kbeg[t] = k0;
        kw = std::max(kw, k1 - k0);
    }
    h->Kw = (kw + 31) / 32 * 32;

    // P2M: every leaf holds 64 sources at the same relative positions, so the
    // weights are z_j S_a(u_jj) with one 64 x R table; L2P: per-row position and -a_r
    std::vector<float> zf(n), tq((size_t)kLeaf * kR), pna(n, 0.0f);
    for (int j = 0; j < n; ++j) zf[j] = (float)znd[j];
    for (int jj = 0; jj < kLeaf; ++jj) {
        double u = (jj + 0.0) / kLeaf * 2.0 - 1.0;  // th_j within its leaf, scaled to [-1, 1)
        for (int a = 0; a < kR; ++a) tq[(size_t)jj * kR + a] = (float)cheb_lagrange(a, u);
    }
    for (int r = 0; r < n; ++r) {
        if (row_leaf[r] < 0 || p->row_kind[r] == 0) continue;
        pna[r] = (float)(-p->row_a[r]);
    }
    std::vector<float> wl((size_t)kR * n, 0.0f);
    for (int r = 0; r < n; ++r) {
        if (pna[r] == 0.0f) continue;
        int b = row_leaf[r];
        double c = (b + 0.5) * hleaf, hw = 0.5 * hleaf;
        for (int a = 0; a < kR; ++a)
            wl[(size_t)a * n + r] = (float)(-p->row_a[r] * cheb_lagrange(a, (ph[r] - c) / hw));
    }
    // leaf-to-leaf kernel 1 / (mu - lambda) = 1 / (2 cos th - 2 cos ph) at the
    // Chebyshev nodes of target leaf I (ph) and source leaf J (th), |I - J| >= 2;
    // rows (I, a), columns (J, b), zero-padded to ncp x ncp
    h->nc = nleaf * kR;
    h->ncp = (h->nc + 127) / 128 * 128;
    const int nc = h->nc, ncp = h->ncp;
    std::vector<float> kf_hi((size_t)ncp * ncp, 0.0f), kf_lo((size_t)ncp * ncp, 0.0f);
    {
        const double hw = 0.5 * hleaf;
        std::vector<double> node(nc);
        for (int I = 0; I < nleaf; ++I)
            for (int a = 0; a < kR; ++a) node[I * kR + a] = (I + 0.5) * hleaf + hw * cheb_node(a);
        for (int ia = 0; ia < nc; ++ia) {
            const int I = ia / kR;
            const double phi = node[ia];
            for (int jb = 0; jb < nc; ++jb) {
                const int J = jb / kR;
                if (std::abs(I - J) <= 1) continue;
                const double th = node[jb];
                const double v = 1.0 / (4.0 * std::sin(0.5 * (phi + th)) * std::sin(0.5 * (phi - th)));
                const float hi = tf32_host((float)v);
                kf_hi[(size_t)ia * ncp + jb] = hi;
                kf_lo[(size_t)ia * ncp + jb] = tf32_host((float)(v - (double)hi));
            }
        }
    }
    // dense rows for eigenvalues outside [0, 4]
    std::vector<float> outw((size_t)std::max(h->nout, 1) * n, 0.0f);
    for (int o = 0; o < h->nout; ++o) {
        int r = h->out_row[o];
        for (int j = 0; j < n; ++j)
            outw[(size_t)o * n + j] =
                (float)w_entry(n, p->row_pole[r], p->row_tau[r], p->row_a[r], znd[j], j);
    }

    auto up = [](auto** dst, const auto& v) -> cudaError_t {
        cudaError_t e = cudaMalloc((void**)dst, sizeof(v[0]) * std::max<size_t>(v.size(), 1));
        if (e != cudaSuccess) return e;
        return cudaMemcpy(*dst, v.data(), sizeof(v[0]) * v.size(), cudaMemcpyHostToDevice);
    };
    DCTPLUS_CUDA_TRY(up(&h->zf, zf));
    DCTPLUS_CUDA_TRY(up(&h->tq, tq));
    DCTPLUS_CUDA_TRY(up(&h->pna, pna));
    DCTPLUS_CUDA_TRY(up(&h->wl, wl));
    DCTPLUS_CUDA_TRY(up(&h->row_leaf, row_leaf));
    DCTPLUS_CUDA_TRY(up(&h->kf_hi, kf_hi));
    DCTPLUS_CUDA_TRY(up(&h->kf_lo, kf_lo));
    DCTPLUS_CUDA_TRY(up(&h->out_w, outw));

    int* d_kbeg = nullptr;
    DCTPLUS_CUDA_TRY(up(&d_kbeg, h->kbeg));
    const size_t slab = (size_t)n * h->Kw;
    DCTPLUS_CUDA_TRY(cudaMalloc((void**)&h->slab_hi, sizeof(float) * slab));
    DCTPLUS_CUDA_TRY(cudaMalloc((void**)&h->slab_lo, sizeof(float) * slab));
    k_band_slab<<<(unsigned)((slab + 255) / 256), 256>>>(n, h->Kw, d_kbeg, p->d_row_kind,
                                                         p->d_row_pole, p->d_row_tau, p->d_row_a,
                                                         d_znd, h->row_leaf, p->d_sin, h->slab_hi,
                                                         h->slab_lo);
    count_launch();
    DCTPLUS_CUDA_TRY(cudaGetLastError());
    DCTPLUS_CUDA_TRY(cudaDeviceSynchronize());
    cudaFree(d_kbeg);
    return DCTPLUS_OK;
}

// ------------------------------------------------------------- far field

// the TF32 remainder of v for an operand whose hi part is v itself (the MMA
// reads v truncated to TF32)
__device__ __forceinline__ float lo_of(float v) {
    return __uint_as_float(ptx::cvt_rna_tf32(v - __uint_as_float(__float_as_uint(v) & ~0x1FFFu)));
}

// P2M: mc[b][lf R + a] = sum over the 64 sources j of leaf lf of z_j S_a(u_j) s_bj
// (and its TF32 remainder), and for each dense row o the partial dot product
// po[b][2 lf + o] = sum over the same sources of out_w[o][j] s_bj. A warp takes
// one leaf of 32 signals: it copies the 32 x 64 source block into shared
// memory with coalesced loads (rows padded to 68 floats, so the per-signal
// reads below are conflict-free), then each lane forms the values of its
// signal; z, the S_a table and the dense rows are broadcast.
constexpr int kP2mPitch = kLeaf + 4;
__global__ void __launch_bounds__(256) k_p2m(int nleaf, const float* __restrict__ zf,
                                             const float* __restrict__ tq, const float* __restrict__ s,
                                             int64_t lds, int64_t batch, float* __restrict__ mc,
                                             float* __restrict__ mc_lo, int ldm, int n, int nout,
                                             const float* __restrict__ out_w, float* __restrict__ po) {
    __shared__ __align__(16) float tqs[kLeaf * kR];
    extern __shared__ __align__(16) float p2m_tile[];  // 8 warps x 32 x kP2mPitch
    for (int e = threadIdx.x; e < kLeaf * kR; e += blockDim.x) tqs[e] = tq[e];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lf = blockIdx.y * 8 + warp;
    if (lf >= nleaf) return;
    const int64_t b0 = (int64_t)blockIdx.x * 32;
    float* tile = p2m_tile + warp * 32 * kP2mPitch;
#pragma unroll
    for (int k = 0; k < 16; ++k) {  // all 16 loads in flight
        const int row = 2 * k + (lane >> 4), c4 = lane & 15;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (b0 + row < batch)
            v = *reinterpret_cast<const float4*>(s + (b0 + row) * lds + (int64_t)lf * kLeaf + 4 * c4);
        *reinterpret_cast<float4*>(tile + row * kP2mPitch + 4 * c4) = v;
    }
    __syncwarp();
    const float4* zp = reinterpret_cast<const float4*>(zf + (int64_t)lf * kLeaf);
    const float* mine = tile + lane * kP2mPitch;
    float acc[kR];
#pragma unroll
    for (int a = 0; a < kR; ++a) acc[a] = 0.f;
    float od[2] = {0.f, 0.f};
#pragma unroll 4
    for (int j4 = 0; j4 < kLeaf / 4; ++j4) {
        const float4 zv = __ldg(zp + j4);
        const float4 sv = *reinterpret_cast<const float4*>(mine + 4 * j4);
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            if (o < nout) {
                const float4 wv = __ldg(reinterpret_cast<const float4*>(out_w + (int64_t)o * n + (int64_t)lf * kLeaf) + j4);
                od[o] = fmaf(wv.x, sv.x, fmaf(wv.y, sv.y, fmaf(wv.z, sv.z, fmaf(wv.w, sv.w, od[o]))));
            }
        }
        const float w[4] = {sv.x * zv.x, sv.y * zv.y, sv.z * zv.z, sv.w * zv.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float4* t = reinterpret_cast<const float4*>(tqs + (4 * j4 + e) * kR);
#pragma unroll
            for (int q = 0; q < kR / 4; ++q) {
                const float4 tv = t[q];
                acc[4 * q + 0] = fmaf(w[e], tv.x, acc[4 * q + 0]);
                acc[4 * q + 1] = fmaf(w[e], tv.y, acc[4 * q + 1]);
                acc[4 * q + 2] = fmaf(w[e], tv.z, acc[4 * q + 2]);
                acc[4 * q + 3] = fmaf(w[e], tv.w, acc[4 * q + 3]);
            }
        }
    }
    const int64_t b = b0 + lane;
    if (b >= batch) return;
    float4* out = reinterpret_cast<float4*>(mc + b * ldm + (int64_t)lf * kR);
    float4* olo = reinterpret_cast<float4*>(mc_lo + b * ldm + (int64_t)lf * kR);
#pragma unroll
    for (int q = 0; q < kR / 4; ++q) {
        out[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
        olo[q] = make_float4(lo_of(acc[4 * q]), lo_of(acc[4 * q + 1]), lo_of(acc[4 * q + 2]),
                             lo_of(acc[4 * q + 3]));
    }
#pragma unroll
    for (int o = 0; o < 2; ++o)
        if (o < nout) po[b * 2 * nleaf + 2 * lf + o] = od[o];
}

// L2P: y[b][r] += sum_a wl[a][r] lc[b][leaf(r) R + a] for the far-field targets.
// A thread keeps row r's weights in registers for 8 signals (block x: 8
// signals, block y: 256 consecutive rows). The extra block row y = n / 256
// writes the dense rows (eigenvalue outside [0, 4]): warp w sums, across its
// lanes, the per-leaf partial dot products of signal 8 x + w.
constexpr int kL2pSig = 8;
__global__ void __launch_bounds__(256) k_l2p(int n, const float* __restrict__ wl,
                                             const int* __restrict__ row_leaf,
                                             const float* __restrict__ pna, const float* __restrict__ lc,
                                             int ldm, float* __restrict__ y, int64_t ldy, int64_t batch,
                                             int nleaf, int out_row0, int out_row1,
                                             const float* __restrict__ po) {
    const int64_t b0 = (int64_t)blockIdx.x * kL2pSig;
    if ((int)blockIdx.y * 256 >= n) {
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int64_t b = b0 + w;
        if (w >= kL2pSig || b >= batch) return;
        for (int o = 0; o < 2; ++o) {
            const int row = o == 0 ? out_row0 : out_row1;
            if (row < 0) continue;
            float t = 0.f;
            for (int lf = lane; lf < nleaf; lf += 32) t += po[b * 2 * nleaf + 2 * lf + o];
            for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
            if (lane == 0) y[b * ldy + row] = t;
        }
        return;
    }
    const int r = blockIdx.y * 256 + threadIdx.x;
    if (pna[r] == 0.f) return;
    float w[kR];
#pragma unroll
    for (int a = 0; a < kR; ++a) w[a] = __ldg(wl + (int64_t)a * n + r);
    const int leaf = row_leaf[r];
#pragma unroll 4
    for (int g = 0; g < kL2pSig; ++g) {
        const int64_t b = b0 + g;
        if (b >= batch) break;
        const float4* l4 = reinterpret_cast<const float4*>(lc + b * ldm + (int64_t)leaf * kR);
        float acc = 0.f;
#pragma unroll
        for (int q = 0; q < kR / 4; ++q) {
            const float4 l = l4[q];
            acc = fmaf(w[4 * q], l.x, fmaf(w[4 * q + 1], l.y, fmaf(w[4 * q + 2], l.z, fmaf(w[4 * q + 3], l.w, acc))));
        }
        y[b * ldy + r] += acc;
    }
}

dctplus_status launch_gemm_tc_band(const float* a_hi, const float* a_lo, int64_t lda, int Ka,
                                   const float* b_hi, const float* b_lo, int64_t ldb, float* y,
                                   int64_t ldy, int M, int N, int K, const int* kbeg,
                                   cudaStream_t s, int dev);  // gemm_tc.cu
void* plan_workspace(dctplus_plan_t p, cudaStream_t st, size_t bytes);

dctplus_status launch_hier(dctplus_plan_t p, const float* x, int64_t ldx, float* y, int64_t ldy,
                           int64_t batch, cudaStream_t st) {
    HierTables* h = p->hier;
    const int n = p->n;
    if (!h || batch > INT32_MAX || (reinterpret_cast<uintptr_t>(y) & 15) || (ldy & 3))
        return DCTPLUS_ERR_UNSUPPORTED;
    if (batch <= 0) return DCTPLUS_OK;
    const size_t plane = (size_t)batch * n, cplane = (size_t)batch * h->ncp;
    const size_t pplane = (size_t)batch * 2 * h->nleaf;
    float* ws = static_cast<float*>(plan_workspace(p, st, sizeof(float) * (2 * plane + 3 * cplane + pplane)));
    if (!ws) return DCTPLUS_ERR_CUDA;
    float* s_hi = ws;
    float* s_lo = ws + plane;
    float* mc = ws + 2 * plane;
    float* mc_lo = mc + cplane;
    float* lc = mc_lo + cplane;
    float* po = lc + cplane;  // batch x 2 nleaf: the dense rows' per-leaf partial sums
    dctplus_status r = launch_dct_fft(p, x, ldx, s_hi, s_lo, n, batch, st);
    if (r != DCTPLUS_OK) return r;
    // far field first, while s is still in L2: leaf coefficients (and the dense
    // rows' per-leaf partial sums), then the leaf-to-leaf product
    const size_t p2m_smem = sizeof(float) * 8 * 32 * kP2mPitch;  // 69.6 KB
    static bool p2m_attr[64] = {};
    if (!p2m_attr[p->device & 63]) {
        DCTPLUS_CUDA_TRY(cudaFuncSetAttribute(k_p2m, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p2m_smem));
        p2m_attr[p->device & 63] = true;
    }
    k_p2m<<<dim3((unsigned)((batch + 31) / 32), (unsigned)((h->nleaf + 7) / 8)), 256, p2m_smem, st>>>(
        h->nleaf, h->zf, h->tq, s_hi, n, batch, mc, mc_lo, h->ncp, n, h->nout, h->out_w, po);
    note_launch(st, "k_p2m", 4.0 * plane + 8.0 * cplane + 4.0 * pplane, 2.0 * kR * plane);
    DCTPLUS_CUDA_TRY(cudaGetLastError());
    r = launch_gemm_tc_band(mc, mc_lo, h->ncp, h->nc, h->kf_hi, h->kf_lo, h->ncp, lc, h->ncp,
                            (int)batch, h->ncp, h->ncp, nullptr, st, p->device);
    if (r != DCTPLUS_OK) return r;
    // near field: y = band of W applied to s (dense rows get 0 here)
    r = launch_gemm_tc_band(s_hi, s_lo, n, n, h->slab_hi, h->slab_lo, h->Kw, y, ldy, (int)batch, n,
                            h->Kw, h->kbeg.data(), st, p->device);
    if (r != DCTPLUS_OK) return r;
    // far field added into y; the dense rows from their partial sums
    k_l2p<<<dim3((unsigned)((batch + kL2pSig - 1) / kL2pSig), (unsigned)(n / 256 + (h->nout > 0))), 256, 0, st>>>(
        n, h->wl, h->row_leaf, h->pna, lc, h->ncp, y, ldy, batch, h->nleaf,
        h->nout > 0 ? h->out_row[0] : -1, h->nout > 1 ? h->out_row[1] : -1, po);
    note_launch(st, "k_l2p", 8.0 * plane + 4.0 * cplane + 4.0 * pplane, 2.0 * kR * plane);
    DCTPLUS_CUDA_TRY(cudaGetLastError());
    return DCTPLUS_OK;
}

}  // namespace dctplus
