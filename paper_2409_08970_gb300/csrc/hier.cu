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
    int ldl = 0;                 // row pitch of the leaf-local array: ncp + 32 (dense-row slots)
    int Kx = 0;                  // far-field (L2P) columns per 128-row output tile, multiple of 32
    std::vector<int> kbeg;       // per 128-row output tile: first source of the K window
    float* slab_hi = nullptr;    // n x Kw
    float* slab_lo = nullptr;
    float* zf = nullptr;         // n: z_j (0 where deflated)
    float* tq_hi = nullptr;      // 64 x kFarTqLd: S_a at the 64 source positions of any leaf
    float* tq_lo = nullptr;
    int* row_leaf = nullptr;     // n
    float* ext_hi = nullptr;     // n x (Kx + 32): L2P weights -a_r S_a(u_r) against the leaf-local
    float* ext_lo = nullptr;     //   coefficients of the row's tile window, then the dense-row slots
    float* kf_hi = nullptr;      // ncp x ncp: leaf-to-leaf kernel samples, TF32 hi
    float* kf_lo = nullptr;      //            and lo (zero for near pairs and padding)
    int* tab_l2l = nullptr;      // K-segment tables of the leaf-to-leaf and the output products
    int* tab_out = nullptr;
    int64_t chunks_l2l = 0, chunks_out = 0;
    double acols_out = 0.0;
    int nout = 0;
    int out_row[2] = {-1, -1};
    float* out_g = nullptr;      // nout x n: -a_o / (mu_o - lambda_j) of the dense rows
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
    void* ptrs[] = {h->slab_hi, h->slab_lo, h->zf,     h->tq_hi,   h->tq_lo,   h->row_leaf, h->ext_hi,
                    h->ext_lo,  h->kf_hi,   h->kf_lo, h->tab_l2l, h->tab_out, h->out_g};
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

    // band windows per 128-row output tile, and each tile's range of target leaves
    const int ntile = n / 128;
    h->kbeg.assign(ntile, 0);
    std::vector<int> tile_lmin(ntile, 0), tile_lmax(ntile, -1);
    int kw = 0;
    for (int t = 0; t < ntile; ++t) {
        int lmin = nleaf, lmax = -1;
        for (int r = 128 * t; r < 128 * t + 128; ++r) {
            if (row_leaf[r] < 0) continue;
            lmin = std::min(lmin, row_leaf[r]);
            lmax = std::max(lmax, row_leaf[r]);
        }
        if (lmax < 0) { lmin = lmax = 0; }
        tile_lmin[t] = lmin;
        tile_lmax[t] = lmax;
        int k0 = (lmin - 1) * kLeaf, k1 = (lmax + 2) * kLeaf;
        h->kbeg[t] = k0;
        kw = std::max(kw, k1 - k0);
    }
    h->Kw = (kw + 31) / 32 * 32;

    // P2M: every leaf holds 64 sources at the same relative positions, so the
    // weights are z_j S_a(u_jj) with one 64 x R table (split into TF32 hi / lo for
    // the DCT kernel's tensor-core contraction); L2P: per-row position and -a_r
    std::vector<float> zf(n), tq_hi((size_t)kLeaf * kFarTqLd, 0.0f), tq_lo((size_t)kLeaf * kFarTqLd, 0.0f);
    for (int j = 0; j < n; ++j) zf[j] = (float)znd[j];
    for (int jj = 0; jj < kLeaf; ++jj) {
        double u = (jj + 0.0) / kLeaf * 2.0 - 1.0;  // th_j within its leaf, scaled to [-1, 1)
        for (int a = 0; a < kR; ++a) {
            const double v = cheb_lagrange(a, u);
            const float hi = tf32_host((float)v);
            tq_hi[(size_t)jj * kFarTqLd + a] = hi;
            tq_lo[(size_t)jj * kFarTqLd + a] = tf32_host((float)(v - (double)hi));
        }
    }
    // leaf-local array per signal: nleaf R coefficients (leaf I at I R), padding to
    // ncp, then 32 slots of which the first nout hold the dense rows' values
    h->nc = nleaf * kR;
    h->ncp = (h->nc + 127) / 128 * 128;
    h->ldl = h->ncp + 32;
    // L2P weights of each far-field target row against the leaf-local coefficients of
    // its tile's window (leaves lmin .. lmax of the tile, starting at column lmin R)
    int kx = 0;
    for (int t = 0; t < ntile; ++t) kx = std::max(kx, (tile_lmax[t] - tile_lmin[t] + 1) * kR);
    h->Kx = (kx + 31) / 32 * 32;
    const int kxb = h->Kx + 32;
    std::vector<float> ext_hi((size_t)n * kxb, 0.0f), ext_lo((size_t)n * kxb, 0.0f);
    for (int r = 0; r < n; ++r) {
        const int t = r / 128;
        if (row_leaf[r] < 0) {  // dense row o: its value sits in slot o after the leaf window
            for (int o = 0; o < h->nout; ++o)
                if (h->out_row[o] == r) ext_hi[(size_t)r * kxb + h->Kx + o] = 1.0f;
            continue;
        }
        if (p->row_kind[r] == 0) continue;  // deflated rows have no far field
        const int b = row_leaf[r];
        const double c = (b + 0.5) * hleaf, hw = 0.5 * hleaf;
        for (int a = 0; a < kR; ++a) {
            const double v = -p->row_a[r] * cheb_lagrange(a, (ph[r] - c) / hw);
            const float hi = tf32_host((float)v);
            const size_t at = (size_t)r * kxb + (size_t)(b - tile_lmin[t]) * kR + a;
            ext_hi[at] = hi;
            ext_lo[at] = tf32_host((float)(v - (double)hi));
        }
    }
    // segment tables (kGemmTabStride ints per 128-column output tile)
    std::vector<int> tab_out((size_t)ntile * kGemmTabStride, 0);
    h->chunks_out = 0;
    h->acols_out = 0.0;
    for (int t = 0; t < ntile; ++t) {
        int* e = &tab_out[(size_t)t * kGemmTabStride];
        int nseg = 0, nk = 0;
        auto add = [&](int src, int acol, int bcol, int nch) {
            e[2 + 4 * nseg] = src;
            e[3 + 4 * nseg] = acol;
            e[4 + 4 * nseg] = bcol;
            e[5 + 4 * nseg] = nch;
            ++nseg;
            nk += nch;
        };
        // near field: the band of W against s, this tile's own width (the slab is zero
        // beyond it)
        add(0, h->kbeg[t], 0, (tile_lmax[t] - tile_lmin[t] + 3) * kLeaf / 32);
        bool far = false, dense = false;
        for (int r = 128 * t; r < 128 * t + 128; ++r) {
            if (row_leaf[r] >= 0 && p->row_kind[r] == 1) far = true;
            if (row_leaf[r] < 0) dense = true;
        }
        const int xw = (tile_lmax[t] - tile_lmin[t] + 1) * kR;
        if (far) add(1, tile_lmin[t] * kR, 0, (xw + 31) / 32);  // far field: L2P of the leaf window
        if (dense) add(1, h->ncp, h->Kx, 1);                    // dense rows: their values
        e[0] = nseg;
        e[1] = nk;
        h->chunks_out += nk;
        h->acols_out += (tile_lmax[t] - tile_lmin[t] + 3) * kLeaf + (far ? 32.0 * ((xw + 31) / 32) : 0.0) +
                        (dense ? 32.0 : 0.0);
    }
    h->acols_out = std::min(h->acols_out, (double)n + h->ldl);
    std::vector<int> tab_l2l((size_t)(h->ncp / 128) * kGemmTabStride, 0);
    for (int t = 0; t < h->ncp / 128; ++t) {
        int* e = &tab_l2l[(size_t)t * kGemmTabStride];
        e[0] = 1;
        e[1] = (h->nc + 31) / 32;  // columns past nc of K_far are zero
        e[2] = 0;
        e[3] = 0;
        e[4] = 0;
        e[5] = (h->nc + 31) / 32;
    }
    h->chunks_l2l = (int64_t)(h->ncp / 128) * ((h->nc + 31) / 32);
    // leaf-to-leaf kernel 1 / (mu - lambda) = 1 / (2 cos th - 2 cos ph) at the
    // Chebyshev nodes of target leaf I (ph) and source leaf J (th), |I - J| >= 2;
    // rows (I, a), columns (J, b), zero-padded to ncp x ncp
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
    // dense rows for eigenvalues outside [0, 4]: W_oj = g_oj z_j with g_oj = -a_o / (mu_o - lambda_j)
    std::vector<float> outg((size_t)std::max(h->nout, 1) * n, 0.0f);
    for (int o = 0; o < h->nout; ++o) {
        int r = h->out_row[o];
        for (int j = 0; j < n; ++j)
            outg[(size_t)o * n + j] =
                (float)w_entry(n, p->row_pole[r], p->row_tau[r], p->row_a[r], znd[j] != 0.0 ? 1.0 : 0.0, j);
    }

    auto up = [](auto** dst, const auto& v) -> cudaError_t {
        cudaError_t e = cudaMalloc((void**)dst, sizeof(v[0]) * std::max<size_t>(v.size(), 1));
        if (e != cudaSuccess) return e;
        return cudaMemcpy(*dst, v.data(), sizeof(v[0]) * v.size(), cudaMemcpyHostToDevice);
    };
    DCTPLUS_CUDA_TRY(up(&h->zf, zf));
    DCTPLUS_CUDA_TRY(up(&h->tq_hi, tq_hi));
    DCTPLUS_CUDA_TRY(up(&h->tq_lo, tq_lo));
    DCTPLUS_CUDA_TRY(up(&h->ext_hi, ext_hi));
    DCTPLUS_CUDA_TRY(up(&h->ext_lo, ext_lo));
    DCTPLUS_CUDA_TRY(up(&h->tab_out, tab_out));
    DCTPLUS_CUDA_TRY(up(&h->tab_l2l, tab_l2l));
    DCTPLUS_CUDA_TRY(up(&h->row_leaf, row_leaf));
    DCTPLUS_CUDA_TRY(up(&h->kf_hi, kf_hi));
    DCTPLUS_CUDA_TRY(up(&h->kf_lo, kf_lo));
    DCTPLUS_CUDA_TRY(up(&h->out_g, outg));

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

// ------------------------------------------------------------- execute

void* plan_workspace(dctplus_plan_t p, cudaStream_t st, size_t bytes);

// Three launches per batch:
//   1. DCT-II (k_dct_far): s, the leaf moments (P2M) and the dense rows' values,
//      which go to the dense-row slots of the leaf-local array (the slots after
//      them are zeroed);
//   2. leaf-to-leaf product (split-TF32 GEMM): leaf-local coefficients
//      L = M K_far^T, into the leaf-local array;
//   3. output product (split-TF32 GEMM over K segments): per 128-row tile the
//      band of W against its window of s (near field), then the L2P weights
//      against the tile's window of leaf-local coefficients (far field), then
//      the dense rows' slots; y is written once.
// The TF32 remainders of s, M and L are formed on chip by the GEMM.
dctplus_status launch_hier(dctplus_plan_t p, const float* x, int64_t ldx, float* y, int64_t ldy,
                           int64_t batch, cudaStream_t st) {
    HierTables* h = p->hier;
    const int n = p->n;
    if (!h || batch > INT32_MAX || (reinterpret_cast<uintptr_t>(y) & 15) || (ldy & 3))
        return DCTPLUS_ERR_UNSUPPORTED;
    if (batch <= 0) return DCTPLUS_OK;
    const size_t plane = (size_t)batch * n, cplane = (size_t)batch * h->ncp, lplane = (size_t)batch * h->ldl;
    float* ws = static_cast<float*>(plan_workspace(p, st, sizeof(float) * (plane + cplane + lplane)));
    if (!ws) return DCTPLUS_ERR_CUDA;
    float* s_hi = ws;
    float* mc = ws + plane;
    float* lc = mc + cplane;
    DctFar far;
    far.zf = h->zf;
    far.tq_hi = h->tq_hi;
    far.tq_lo = h->tq_lo;
    far.mc = mc;
    far.ldm = h->ncp;
    far.out_g = h->out_g;
    far.nout = h->nout;
    far.dv = lc + h->ncp;
    far.ldd = h->ldl;
    dctplus_status r = launch_dct_far(p, x, ldx, s_hi, n, batch, far, st);
    if (r != DCTPLUS_OK) return r;
    GemmSrc l2l{mc, nullptr, h->ncp, h->nc, h->kf_hi, h->kf_lo, h->ncp, h->ncp};
    r = launch_gemm_tc_segs(&l2l, 1, h->tab_l2l, h->chunks_l2l, (double)h->nc, lc, nullptr, h->ldl,
                            (int)batch, h->ncp, st, p->device, "k_gemm_tc");
    if (r != DCTPLUS_OK) return r;
    GemmSrc out[2] = {{s_hi, nullptr, n, n, h->slab_hi, h->slab_lo, h->Kw, h->Kw},
                      {lc, nullptr, h->ldl, h->ldl, h->ext_hi, h->ext_lo, h->Kx + 32, h->Kx + 32}};
    return launch_gemm_tc_segs(out, 2, h->tab_out, h->chunks_out, h->acols_out, y, nullptr, ldy,
                               (int)batch, n, st, p->device, "k_gemm_tc");
}

}  // namespace dctplus
