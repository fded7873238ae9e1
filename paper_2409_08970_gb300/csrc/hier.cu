// Hierarchical O(n log n) evaluation of the Cauchy product of Theorem 3.1
// (the fast matrix-vector product Theorem 3.2 relies on, in the Gerasoulis /
// fast-multipole family), for a batch of signals.
//
// The product is y_r = sum_j W_rj s_j with W_rj = -a_r z_j / (mu_r - lambda_j)
// (root rows) or e_j (deflated rows), s = U^T x. Write lambda_j = 2 - 2 cos th_j
// with th_j = pi j / n (uniform) and mu_r = 2 - 2 cos ph_r. Then
//   1 / (mu - lambda) = 1 / (2 cos th - 2 cos ph),
// a kernel of (ph, th) that is analytic away from th = +-ph, so Chebyshev
// interpolation in th over a box of width h is accurate for targets at least
// one box away (convergence factor 3 + sqrt(8) per degree). Sources are
// uniform in th, so a binary tree of equal th-boxes with 64 sources per leaf
// is balanced; targets interlace the sources (Lemma 4.1), about 64 per leaf.
//
//   near field  targets of leaf I against sources of leaves I-1, I, I+1: exact
//               entries of W, a band matrix applied on the tensor cores with
//               the split-TF32 GEMM (each 128-row output tile contracts a
//               K window of s against a compact [n x Kw] slab of W entries);
//   far field   every other source, through Chebyshev expansions of degree R:
//               P2M at the leaves (z folded into the weights), M2M up the tree,
//               M2L between well-separated boxes of each level, L2L down, L2P
//               at the target leaves (-a folded into the weights); one CTA per
//               group of up to 16 signals on CUDA cores, added into y.
// Roots outside [0, 4] (at most the largest for rho > 0 or the smallest for
// rho < 0; the paper's pre-processing isolates the same root) have no real
// angle; their rows are dense dot products.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace dctplus {

constexpr int kLeaf = 64;
constexpr int kR = 12;  // Chebyshev degree of the far-field expansions

struct HierTables {
    int nleaf = 0, L = 0, Kw = 0;
    std::vector<int> kbeg;       // per 128-row output tile: first source of the K window
    float* slab_hi = nullptr;    // n x Kw
    float* slab_lo = nullptr;
    float* zf = nullptr;         // n: z_j (0 where deflated)
    float* tq = nullptr;         // 64 x R: S_a at the 64 source positions of any leaf
    float* pu = nullptr;         // n: position of row r in its leaf, in [-1, 1]
    float* pna = nullptr;        // n: -a_r for far-field targets, 0 otherwise
    float* wl = nullptr;         // R x n: L2P weights -a_r S_a(u_r) (0 for other rows)
    float* cheb = nullptr;       // 2 x R: Chebyshev nodes and barycentric weights
    int* row_leaf = nullptr;     // n
    float* tlr = nullptr;        // 2 x R x R: parent basis at left / right child nodes
    float* m2l = nullptr;        // (2^(L+1) - 1) x 3 x R x R
    int* il = nullptr;           // (2^(L+1) - 1) x 3 interaction-list boxes (-1: none)
    int nout = 0;
    int out_row[2] = {-1, -1};
    float* out_w = nullptr;      // nout x n dense rows
};

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
    void* ptrs[] = {h->slab_hi, h->slab_lo, h->zf, h->tq, h->pu, h->pna, h->wl, h->cheb,
                    h->row_leaf, h->tlr, h->m2l, h->il, h->out_w};
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
    h->L = 0;
    while ((1 << h->L) < h->nleaf) ++h->L;
    const int nleaf = h->nleaf, L = h->L;
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
    std::vector<float> zf(n), tq((size_t)kLeaf * kR), pu(n, 0.0f), pna(n, 0.0f), cheb(2 * kR);
    for (int j = 0; j < n; ++j) zf[j] = (float)znd[j];
    for (int jj = 0; jj < kLeaf; ++jj) {
        double u = (jj + 0.0) / kLeaf * 2.0 - 1.0;  // th_j within its leaf, scaled to [-1, 1)
        for (int a = 0; a < kR; ++a) tq[(size_t)jj * kR + a] = (float)cheb_lagrange(a, u);
    }
    for (int r = 0; r < n; ++r) {
        if (row_leaf[r] < 0 || p->row_kind[r] == 0) continue;
        int b = row_leaf[r];
        double c = (b + 0.5) * hleaf, hw = 0.5 * hleaf;
        pu[r] = (float)((ph[r] - c) / hw);
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
    for (int a = 0; a < kR; ++a) {
        cheb[a] = (float)cheb_node(a);
        cheb[kR + a] = (float)(((a & 1) ? -1.0 : 1.0) * std::sin((2 * a + 1) * M_PI / (2.0 * kR)));
    }
    // transfer: parent basis at child nodes, child at (t - 1)/2 (left) or (t + 1)/2 (right)
    std::vector<float> tlr(2 * kR * kR);
    for (int side = 0; side < 2; ++side)
        for (int a = 0; a < kR; ++a)
            for (int a2 = 0; a2 < kR; ++a2)
                tlr[(side * kR + a) * kR + a2] =
                    (float)cheb_lagrange(a, 0.5 * (cheb_node(a2) + (side ? 1.0 : -1.0)));
    // interaction lists and M2L kernels 1 / (2 cos th - 2 cos ph) at the box nodes
    const int nbox = (1 << (L + 1)) - 1;
    std::vector<int> il((size_t)nbox * 3, -1);
    std::vector<float> m2l((size_t)nbox * 3 * kR * kR, 0.0f);
    for (int l = 2; l <= L; ++l) {
        const int nb = 1 << l;
        const double hw = 0.5 * M_PI / nb;
        for (int I = 0; I < nb; ++I) {
            int q = 0;
            int pI = I >> 1;
            for (int pj = pI - 1; pj <= pI + 1; ++pj) {
                if (pj < 0 || pj >= (nb >> 1)) continue;
                for (int J = 2 * pj; J <= 2 * pj + 1; ++J) {
                    if (std::abs(J - I) <= 1) continue;
                    size_t slot = (size_t)((1 << l) - 1 + I) * 3 + q;
                    il[slot] = J;
                    double cI = (I + 0.5) * 2 * hw, cJ = (J + 0.5) * 2 * hw;
                    for (int a = 0; a < kR; ++a)
                        for (int b = 0; b < kR; ++b) {
                            double phi = cI + hw * cheb_node(a), th = cJ + hw * cheb_node(b);
                            double den = 4.0 * std::sin(0.5 * (phi + th)) * std::sin(0.5 * (phi - th));
                            m2l[(slot * kR + a) * kR + b] = (float)(1.0 / den);
                        }
                    ++q;
                }
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
    DCTPLUS_CUDA_TRY(up(&h->pu, pu));
    DCTPLUS_CUDA_TRY(up(&h->pna, pna));
    DCTPLUS_CUDA_TRY(up(&h->wl, wl));
    DCTPLUS_CUDA_TRY(up(&h->cheb, cheb));
    DCTPLUS_CUDA_TRY(up(&h->row_leaf, row_leaf));
    DCTPLUS_CUDA_TRY(up(&h->tlr, tlr));
    DCTPLUS_CUDA_TRY(up(&h->m2l, m2l));
    DCTPLUS_CUDA_TRY(up(&h->il, il));
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

struct FarArgs {
    int n, nleaf, L, nout;
    const float* zf;
    const float* tq;
    const float* pna;
    const float* wl;
    const int* row_leaf;
    const float* tlr;
    const float* m2l;
    const int* il;
    const float* out_w;
    int out_row0, out_row1;
};

constexpr int kFarThreads = 512;

// QS consecutive signals (a quad when NS >= 4) of the NS held in shared memory
template <int QS>
struct Vq {
    float v[QS];
};
template <int QS>
__device__ __forceinline__ Vq<QS> ldq(const float* p) {
    Vq<QS> r;
    if constexpr (QS == 4) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
    } else {
#pragma unroll
        for (int g = 0; g < QS; ++g) r.v[g] = p[g];
    }
    return r;
}

// One CTA per group of NS signals: y[b] += far-field part of W s_b (and the
// dense rows). Every phase splits its work into items of QS signals so that
// all threads stay busy; coefficient arrays are [node][a][signal] so an item
// reads its QS values with one vector load.
template <int NS>
__global__ void __launch_bounds__(kFarThreads) k_far(FarArgs A, const float* __restrict__ s, int64_t lds,
                                                     float* __restrict__ y, int64_t ldy, int64_t batch) {
    constexpr int QS = NS < 4 ? NS : 4;
    constexpr int NQ = NS / QS;
    extern __shared__ __align__(16) float fsm[];
    const int n = A.n, nleaf = A.nleaf, L = A.L;
    const int nbox = (1 << (L + 1)) - 1;
    float* sv = fsm;                      // NS x n
    float* zf = sv + NS * n;              // n
    float* M = zf + n;                    // nbox x R x NS multipole coefficients
    float* Lc = M + nbox * kR * NS;       // nbox x R x NS local coefficients
    float* tq = Lc + nbox * kR * NS;      // 64 x R
    float* tlr = tq + kLeaf * kR;         // 2 x R x R
    float* red = tlr + 2 * kR * kR;       // (threads / 32) x NS
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < kLeaf * kR; e += nt) tq[e] = A.tq[e];
    for (int e = tid; e < 2 * kR * kR; e += nt) tlr[e] = A.tlr[e];
    for (int e = tid; e < n; e += nt) zf[e] = A.zf[e];
    const int n4 = n / 4;  // n is a power of two >= 256 and lds % 4 == 0 (checked by the launcher)
    for (int64_t b0 = (int64_t)blockIdx.x * NS; b0 < batch; b0 += (int64_t)gridDim.x * NS) {
        const int ns = (int)min((int64_t)NS, batch - b0);
        __syncthreads();
        {
            float4* sv4 = reinterpret_cast<float4*>(sv);
#pragma unroll 4
            for (int e = tid; e < NS * n4; e += nt) {
                const int g = e / n4, j4 = e - g * n4;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (g < ns) v = __ldg(reinterpret_cast<const float4*>(s + (b0 + g) * lds) + j4);
                sv4[e] = v;
            }
        }
        __syncthreads();
        // P2M at the leaves: M[leaf][a] = sum_jj z_j S_a(u_jj) s_j
        for (int e = tid; e < nleaf * kR * NQ; e += nt) {
            const int q = e % NQ, la = e / NQ, lf = la / kR, a = la % kR;
            float acc[QS];
#pragma unroll
            for (int g = 0; g < QS; ++g) acc[g] = 0.f;
            const float* sq = sv + (q * QS) * n + lf * kLeaf;
            for (int jj = 0; jj < kLeaf; jj += 4) {
                const int j = lf * kLeaf + jj;
                const float w0 = zf[j] * tq[jj * kR + a], w1 = zf[j + 1] * tq[(jj + 1) * kR + a];
                const float w2 = zf[j + 2] * tq[(jj + 2) * kR + a], w3 = zf[j + 3] * tq[(jj + 3) * kR + a];
#pragma unroll
                for (int g = 0; g < QS; ++g) {
                    const float4 v = *reinterpret_cast<const float4*>(sq + g * n + jj);
                    acc[g] = fmaf(w0, v.x, fmaf(w1, v.y, fmaf(w2, v.z, fmaf(w3, v.w, acc[g]))));
                }
            }
            float* out = M + ((nleaf - 1 + lf) * kR + a) * NS + q * QS;
#pragma unroll
            for (int g = 0; g < QS; ++g) out[g] = acc[g];
        }
        __syncthreads();
        // M2M up to level 2
        for (int l = L - 1; l >= 2; --l) {
            const int nb = 1 << l;
            for (int e = tid; e < nb * kR * NQ; e += nt) {
                const int q = e % NQ, ba = e / NQ, bx = ba / kR, a = ba % kR;
                const float* ml = M + ((2 << l) - 1 + 2 * bx) * kR * NS + q * QS;
                const float* mr = ml + kR * NS;
                float acc[QS];
#pragma unroll
                for (int g = 0; g < QS; ++g) acc[g] = 0.f;
#pragma unroll
                for (int a2 = 0; a2 < kR; ++a2) {
                    const float tl = tlr[a * kR + a2], tr = tlr[(kR + a) * kR + a2];
                    const Vq<QS> vl = ldq<QS>(ml + a2 * NS), vr = ldq<QS>(mr + a2 * NS);
#pragma unroll
                    for (int g = 0; g < QS; ++g) acc[g] = fmaf(tl, vl.v[g], fmaf(tr, vr.v[g], acc[g]));
                }
                float* out = M + ((nb - 1 + bx) * kR + a) * NS + q * QS;
#pragma unroll
                for (int g = 0; g < QS; ++g) out[g] = acc[g];
            }
            __syncthreads();
        }
        // M2L at every level >= 2 (nodes of levels >= 2 start at index 3)
        for (int e = tid; e < (nbox - 3) * kR * NQ; e += nt) {
            const int q = e % NQ, na = e / NQ, node = 3 + na / kR, a = na % kR;
            const int lvl = 31 - __clz(node + 1);
            float acc[QS];
#pragma unroll
            for (int g = 0; g < QS; ++g) acc[g] = 0.f;
            for (int q3 = 0; q3 < 3; ++q3) {
                const int J = A.il[node * 3 + q3];
                if (J < 0) continue;
                const float* mj = M + ((1 << lvl) - 1 + J) * kR * NS + q * QS;
                const float* k = A.m2l + ((size_t)(node * 3 + q3) * kR + a) * kR;
                float kv[kR];
#pragma unroll
                for (int b2 = 0; b2 < kR; ++b2) kv[b2] = __ldg(k + b2);
#pragma unroll
                for (int b2 = 0; b2 < kR; ++b2) {
                    const Vq<QS> v = ldq<QS>(mj + b2 * NS);
#pragma unroll
                    for (int g = 0; g < QS; ++g) acc[g] = fmaf(kv[b2], v.v[g], acc[g]);
                }
            }
            float* out = Lc + (node * kR + a) * NS + q * QS;
#pragma unroll
            for (int g = 0; g < QS; ++g) out[g] = acc[g];
        }
        __syncthreads();
        // L2L down to the leaves
        for (int l = 2; l < L; ++l) {
            const int nb = 1 << l;
            for (int e = tid; e < 2 * nb * kR * NQ; e += nt) {
                const int q = e % NQ, ca = e / NQ, c = ca / kR, a2 = ca % kR;  // child box at level l + 1
                const int side = c & 1;
                const float* lp = Lc + (nb - 1 + (c >> 1)) * kR * NS + q * QS;
                float acc[QS];
#pragma unroll
                for (int g = 0; g < QS; ++g) acc[g] = 0.f;
#pragma unroll
                for (int a = 0; a < kR; ++a) {
                    const float t = tlr[(side * kR + a) * kR + a2];
                    const Vq<QS> v = ldq<QS>(lp + a * NS);
#pragma unroll
                    for (int g = 0; g < QS; ++g) acc[g] = fmaf(t, v.v[g], acc[g]);
                }
                float* out = Lc + ((2 * nb - 1 + c) * kR + a2) * NS + q * QS;
#pragma unroll
                for (int g = 0; g < QS; ++g) out[g] += acc[g];
            }
            __syncthreads();
        }
        // L2P: y_r += sum_a w[a][r] L[leaf(r)][a] with w = -a_r S_a(u_r) from the table
        for (int e = tid; e < n * NQ; e += nt) {
            const int q = e / n, r = e - q * n;
            if (A.pna[r] == 0.f) continue;
            const float* lc = Lc + (nleaf - 1 + A.row_leaf[r]) * kR * NS + q * QS;
            float acc[QS];
#pragma unroll
            for (int g = 0; g < QS; ++g) acc[g] = 0.f;
#pragma unroll
            for (int a = 0; a < kR; ++a) {
                const float w = __ldg(A.wl + (size_t)a * n + r);
                const Vq<QS> v = ldq<QS>(lc + a * NS);
#pragma unroll
                for (int g = 0; g < QS; ++g) acc[g] = fmaf(w, v.v[g], acc[g]);
            }
            float yv[QS];
#pragma unroll
            for (int g = 0; g < QS; ++g) yv[g] = (q * QS + g < ns) ? y[(b0 + q * QS + g) * ldy + r] : 0.f;
#pragma unroll
            for (int g = 0; g < QS; ++g)
                if (q * QS + g < ns) y[(b0 + q * QS + g) * ldy + r] = yv[g] + acc[g];
        }
        // dense rows
        for (int o = 0; o < A.nout; ++o) {
            const float* w = A.out_w + (size_t)o * n;
            float acc[NS];
#pragma unroll
            for (int g = 0; g < NS; ++g) acc[g] = 0.f;
            for (int j = tid; j < n; j += nt) {
                const float wj = w[j];
#pragma unroll
                for (int g = 0; g < NS; ++g) acc[g] = fmaf(wj, sv[g * n + j], acc[g]);
            }
#pragma unroll
            for (int g = 0; g < NS; ++g) {
                float v = acc[g];
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if ((tid & 31) == 0) red[(tid >> 5) * NS + g] = v;
            }
            __syncthreads();
            if (tid < ns) {
                float t = 0.f;
                for (int w2 = 0; w2 < nt / 32; ++w2) t += red[w2 * NS + tid];
                y[(b0 + tid) * ldy + (o == 0 ? A.out_row0 : A.out_row1)] = t;
            }
            __syncthreads();
        }
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
    const size_t plane = (size_t)batch * n;
    float* ws = static_cast<float*>(plan_workspace(p, st, 2 * sizeof(float) * plane));
    if (!ws) return DCTPLUS_ERR_CUDA;
    dctplus_status r = launch_dct_fft(p, x, ldx, ws, ws + plane, n, batch, st);
    if (r != DCTPLUS_OK) return r;
    r = launch_gemm_tc_band(ws, ws + plane, n, n, h->slab_hi, h->slab_lo, h->Kw, y, ldy, (int)batch,
                            n, h->Kw, h->kbeg.data(), st, p->device);
    if (r != DCTPLUS_OK) return r;
    FarArgs A;
    A.n = n;
    A.nleaf = h->nleaf;
    A.L = h->L;
    A.nout = h->nout;
    A.zf = h->zf;
    A.tq = h->tq;
    A.pna = h->pna;
    A.wl = h->wl;
    A.row_leaf = h->row_leaf;
    A.tlr = h->tlr;
    A.m2l = h->m2l;
    A.il = h->il;
    A.out_w = h->out_w;
    A.out_row0 = h->out_row[0];
    A.out_row1 = h->out_row[1];
    const int nbox = (1 << (h->L + 1)) - 1;
    auto smem_for = [&](int ns) {
        return sizeof(float) * ((size_t)ns * n + n + 2 * (size_t)nbox * kR * ns + kLeaf * kR +
                                2 * kR * kR + (kFarThreads / 32) * ns);
    };
    const size_t cap = 100 * 1024;  // several CTAs per SM
    int ns = 16;
    while (ns > 1 && smem_for(ns) > cap) ns >>= 1;
    const size_t smem = smem_for(ns);
    int64_t groups = (batch + ns - 1) / ns;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    const int per_sm = std::max(1, std::min((int)(220 * 1024 / smem), 2048 / kFarThreads));
    int64_t grid = std::min<int64_t>(groups, (int64_t)std::max(sms, 1) * per_sm);
    auto launch = [&](auto kern) -> dctplus_status {
        DCTPLUS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<(unsigned)grid, kFarThreads, smem, st>>>(A, ws, n, y, ldy, batch);
        count_launch();
        DCTPLUS_CUDA_TRY(cudaGetLastError());
        return DCTPLUS_OK;
    };
    switch (ns) {
        case 16: return launch(k_far<16>);
        case 8: return launch(k_far<8>);
        case 4: return launch(k_far<4>);
        case 2: return launch(k_far<2>);
        default: return launch(k_far<1>);
    }
}

}  // namespace dctplus
