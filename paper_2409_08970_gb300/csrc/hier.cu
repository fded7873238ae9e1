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
//   far field   every other source, through a 1-D fast multipole tree over the
//               th-boxes with Chebyshev interpolation of degree R in both
//               variables: P2M (leaf moments, the sources' z-weighted Lagrange
//               weights; in the DCT kernel, a split-TF32 contraction), M2M
//               (the parent's Lagrange basis at its children's nodes, exact
//               for polynomials of the degree; each level composed from its
//               leaves, so the levels are independent), M2L per level (the
//               kernel sampled at the nodes of each box against the boxes of
//               its interaction list: at least one box apart, parents
//               adjacent; at the top level of 4 boxes, every box at least one
//               apart), L2L chains down to the leaves, and L2P (-a folded into
//               the weights) as extra K columns of the output product. Every
//               far leaf pair meets in exactly one list, so the far field is
//               the leaf-level one, evaluated in O(n log n) multiply-adds with
//               O(n) tables. M2M, M2L and L2L are 12 x 12 blocks per signal;
//               they run in FP32 on the CUDA cores, a lane per signal, each
//               block broadcast from shared memory or L1.
// Roots outside [0, 4] (at most the largest for rho > 0 or the smallest for
// rho < 0; the paper's pre-processing isolates the same root) have no real
// angle; their rows are dense dot products, formed by the DCT kernel from the
// same z-weighted coefficients and placed after the leaf-local coefficients.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace dctplus {

constexpr int kLeaf = 64;
constexpr int kR = 12;  // Chebyshev degree of the far-field expansions
// The leaf-to-leaf product's N (12 n / 64, padded to 128) gives few 128-column tiles at
// small n (32 row tiles x 2 at n = 1024, batch 4096). When even twice as many 64-column
// tiles fit in one wave over the SMs it runs 64 wide (measured: 14.3 -> 12.1 us at
// n = 1024); otherwise 128 wide, since narrow tiles cost more per multiply-add (at
// n = 4096, batch 4096: 45 -> 57 us; at n = 16384, batch 512, where 96 wide tiles leave
// SMs idle but each runs K = 3072: 80 -> 139 us). Its table has the same entry for every
// tile, so one table of 64-column tiles serves both widths.
constexpr int kL2lNarrow = 64;

struct HierTables {
    int nleaf = 0, Kw = 0;
    int form = 0;                // far field: 1 = leaf level (one dense leaf-to-leaf product), 2 = tree
    int nc = 0;                  // leaf-local coefficients nleaf R
    int ncp = 0;                 // nc rounded up to 128 (the leaf-to-leaf product's output width)
    int dslot = 0;               // column of the dense-row slots in the leaf-local array
    int dbase = 0;               // this plan's first dense-row slot (even): plans that share a
                                 //   leaf-local array keep their dense rows apart
    int ldl = 0;                 // row pitch of the leaf-local array: dslot + 32
    int ldm = 0;                 // row pitch of the moment (and M2L output) arrays
    int Kx = 0;                  // far-field (L2P) columns per 128-row output tile, multiple of 32
    int nlev = 0, nbox = 0;      // tree levels (leaf level included) and boxes over all levels
    int lev_off[kFarMaxLev] = {}, box_off[kFarMaxLev + 1] = {}, chain_off[kFarMaxLev] = {};
    std::vector<int> kbeg;       // per 128-row output tile: first source of the K window
    float* slab_hi = nullptr;    // n x Kw
    float* slab_lo = nullptr;
    float* zf = nullptr;         // n: z_j (0 where deflated)
    std::vector<float> zf_host;  // the same on the host: plans with equal zf (and form) have the
                                 //   same moments, far field and leaf-local coefficients
    float* tq_hi = nullptr;      // 64 x kFarTqLd: S_a at the 64 source positions of any leaf
    float* tq_lo = nullptr;
    float* tm_hi = nullptr;      // 24 x kFarTqLd: M2M re-expansion of both children (tree)
    float* tm_lo = nullptr;
    float* kf_hi = nullptr;      // ncp x ncp: leaf-to-leaf kernel samples, TF32 hi and lo (leaf
    float* kf_lo = nullptr;      //   level; zero for near pairs and padding)
    int* tab_l2l = nullptr;      // its K-segment table
    int64_t chunks_l2l = 0;
    float* m2l = nullptr;        // nbox x 4 slots x [12][12]: M2L kernel samples (FP32, tree)
    int* slot_box = nullptr;     // nbox x 4: source box (within its level) of each slot, -1 if none
    float* chain = nullptr;      // L2L chains, level l >= 1, leaf position i < 2^l: [12][12] each
    int* row_leaf = nullptr;     // n
    float* ext_hi = nullptr;     // n x (Kx + 32): L2P weights -a_r S_a(u_r) against the leaf-local
    float* ext_lo = nullptr;     //   coefficients of the row's tile window, then the dense-row slots
    int* tab_out = nullptr;      // K-segment table of the output product
    int64_t chunks_out = 0;
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

// Leaf-to-leaf kernel samples of the leaf-level far field: entry (I a, J b) is
// 1 / (mu - lambda) = 1 / (4 sin((ph + th) / 2) sin((ph - th) / 2)) at the Chebyshev node ph of
// target leaf I and th of source leaf J (node[]), for |I - J| >= 2, split into TF32 hi and
// remainder (round to nearest even on the bits, as tf32_host); zero for near pairs and for the
// padding of the nc x nc table to ncp x ncp. FP64, one thread per entry.
__global__ void k_kf_table(int nleaf, int ncp, const double* __restrict__ node, float* __restrict__ hi,
                           float* __restrict__ lo) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)ncp * ncp) return;
    const int ia = (int)(idx / ncp), jb = (int)(idx % ncp);
    const int nc = nleaf * kR;
    float h = 0.f, l = 0.f;
    if (ia < nc && jb < nc && abs(ia / kR - jb / kR) > 1) {
        const double phi = node[ia], th = node[jb];
        const double v = 1.0 / (4.0 * sin(0.5 * (phi + th)) * sin(0.5 * (phi - th)));
        auto rne = [](float f) {
            const uint32_t u = __float_as_uint(f);
            return __uint_as_float((u + 0xFFFu + ((u >> 13) & 1u)) & ~0x1FFFu);
        };
        h = rne((float)v);
        l = rne((float)(v - (double)h));
    }
    hi[idx] = h;
    lo[idx] = l;
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
    void* ptrs[] = {h->slab_hi, h->slab_lo, h->zf,     h->tq_hi,  h->tq_lo,   h->tm_hi, h->tm_lo,
                    h->kf_hi,   h->kf_lo,   h->tab_l2l, h->m2l,   h->slot_box, h->chain, h->row_leaf,
                    h->ext_hi,  h->ext_lo,  h->tab_out, h->out_g};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete h;
}

bool hier_shape(int n) { return n >= 4 * kLeaf && (n & (n - 1)) == 0 && n <= kMaxN; }

dctplus_status setup_hier(dctplus_plan_t p, const double* d_znd) {
    const int n = p->n;
    if (!hier_shape(n)) return DCTPLUS_ERR_UNSUPPORTED;
    const int form = p->far_field;
    if (form != 1 && form != 2) return DCTPLUS_ERR_INVALID_ARG;
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
    // leaf-local array per signal: nleaf R coefficients (leaf I at I R), then 32
    // slots of which the first nout hold the dense rows' values
    h->nc = nleaf * kR;
    h->ncp = (h->nc + 127) / 128 * 128;
    h->form = form;
    h->dslot = form == 1 ? h->ncp : h->nc;  // the leaf-to-leaf product writes all ncp columns
    h->ldl = h->dslot + 32;
    {
        static std::atomic<unsigned> seq{0};  // plans made one after another get distinct slot pairs
        h->dbase = 2 * (int)(seq.fetch_add(1) % 16);
    }
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
                if (h->out_row[o] == r) ext_hi[(size_t)r * kxb + h->Kx + h->dbase + o] = 1.0f;
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
        if (dense) add(1, h->dslot, h->Kx, 1);                  // dense rows: their values
        e[0] = nseg;
        e[1] = nk;
        h->chunks_out += nk;
        h->acols_out += (tile_lmax[t] - tile_lmin[t] + 3) * kLeaf + (far ? 32.0 * ((xw + 31) / 32) : 0.0) +
                        (dense ? 32.0 : 0.0);
    }
    h->acols_out = std::min(h->acols_out, (double)n + h->ldl);

    // the tree (its levels are also counted for the leaf-level form, which uses none of
    // the tables below): level l has nleaf >> l boxes of th-width pi / (nleaf >> l), down to 4 boxes
    h->nlev = 0;
    h->nbox = 0;
    for (int nb = nleaf; nb >= 4; nb >>= 1) {
        if (h->nlev >= kFarMaxLev) return DCTPLUS_ERR_UNSUPPORTED;
        h->box_off[h->nlev] = h->nbox;
        h->lev_off[h->nlev] = h->nbox * kR;
        h->nbox += nb;
        ++h->nlev;
    }
    h->box_off[h->nlev] = h->nbox;
    h->ldm = form == 2 ? h->nbox * kR : h->nc;  // multiples of 4
    // M2M re-expansion: E_k[a][b] = S_a((x_b + 2k - 1) / 2), the parent's basis at child
    // k's nodes (only through the chains below: up the tree the composed re-expansion is
    // the transposed chain)
    double E[2][kR][kR];
    for (int k = 0; k < 2; ++k)
        for (int a = 0; a < kR; ++a)
            for (int b = 0; b < kR; ++b) E[k][a][b] = cheb_lagrange(a, (cheb_node(b) + 2 * k - 1) / 2.0);
    // as the DCT kernel's M2M operand: row k = child * 12 + b, column a, TF32 hi / lo
    std::vector<float> tm_hi((size_t)24 * kFarTqLd, 0.0f), tm_lo((size_t)24 * kFarTqLd, 0.0f);
    for (int k = 0; k < 2; ++k)
        for (int b = 0; b < kR; ++b)
            for (int a = 0; a < kR; ++a) {
                const double v = E[k][a][b];
                const size_t at = (size_t)(k * kR + b) * kFarTqLd + a;
                tm_hi[at] = tf32_host((float)v);
                tm_lo[at] = tf32_host((float)(v - (double)tm_hi[at]));
            }
    // M2L: per box B of level l and slot s (source box B + {-3, -2, 2, 3}[s] if it is in
    // B's interaction list), block [a][b] = 1 / (mu - lambda) at (ph_a of B, th_b of C)
    static const int kSlotOff[4] = {-3, -2, 2, 3};
    std::vector<float> m2l((size_t)h->nbox * 4 * kR * kR, 0.0f);
    std::vector<int> slot_box((size_t)h->nbox * 4, -1);
    for (int l = 0; l < h->nlev; ++l) {
        const int nb = nleaf >> l;
        const bool top = l == h->nlev - 1;
        const double hb = M_PI / nb, hw = 0.5 * hb;
        for (int B = 0; B < nb; ++B) {
            for (int sl = 0; sl < 4; ++sl) {
                const int Cb = B + kSlotOff[sl];
                if (Cb < 0 || Cb >= nb) continue;
                if (!top && std::abs(Cb / 2 - B / 2) > 1) continue;
                const size_t e = (size_t)(h->box_off[l] + B) * 4 + sl;
                slot_box[e] = Cb;
                for (int b = 0; b < kR; ++b) {
                    const double th = (Cb + 0.5) * hb + hw * cheb_node(b);
                    for (int a = 0; a < kR; ++a) {
                        const double phi = (B + 0.5) * hb + hw * cheb_node(a);
                        const double v = 1.0 / (4.0 * std::sin(0.5 * (phi + th)) * std::sin(0.5 * (phi - th)));
                        m2l[(e * kR + a) * kR + b] = (float)v;
                    }
                }
            }
        }
    }
    // L2L chains: level-l local expansion of the ancestor to leaf I, I mod 2^l = i:
    // G = E_{b1}^T E_{b2}^T ... E_{bl}^T with b_m = (i >> (m - 1)) & 1, stored [a][b]
    int nchain = 0;
    for (int l = 1; l < h->nlev; ++l) {
        h->chain_off[l] = nchain;
        nchain += 1 << l;
    }
    std::vector<float> chain((size_t)std::max(nchain, 1) * kR * kR, 0.0f);
    for (int l = 1; l < h->nlev; ++l) {
        for (int i = 0; i < (1 << l); ++i) {
            double G[kR][kR], T[kR][kR];
            for (int a = 0; a < kR; ++a)
                for (int b = 0; b < kR; ++b) G[a][b] = a == b ? 1.0 : 0.0;
            for (int m = 1; m <= l; ++m) {  // G <- G E_{b_m}^T
                const int bm = (i >> (m - 1)) & 1;
                for (int a = 0; a < kR; ++a)
                    for (int b = 0; b < kR; ++b) {
                        double acc = 0.0;
                        for (int c = 0; c < kR; ++c) acc += G[a][c] * E[bm][b][c];
                        T[a][b] = acc;
                    }
                std::memcpy(G, T, sizeof(G));
            }
            const size_t e = (size_t)(h->chain_off[l] + i);
            for (int a = 0; a < kR; ++a)
                for (int b = 0; b < kR; ++b) chain[(e * kR + a) * kR + b] = (float)G[a][b];
        }
    }

    // leaf level: the kernel 1 / (mu - lambda) = 1 / (2 cos th - 2 cos ph) at the
    // Chebyshev nodes of target leaf I (ph) and source leaf J (th), |I - J| >= 2; rows
    // (I, a), columns (J, b), zero-padded to ncp x ncp, and its segment table
    // (filled on the device by k_kf_table from the nodes: ncp^2 FP64 entries)
    std::vector<double> node;
    std::vector<int> tab_l2l;
    if (form == 1) {
        const int nc = h->nc, ncp = h->ncp;
        const double hw = 0.5 * hleaf;
        node.resize(nc);
        for (int I = 0; I < nleaf; ++I)
            for (int a = 0; a < kR; ++a) node[I * kR + a] = (I + 0.5) * hleaf + hw * cheb_node(a);
        tab_l2l.assign((size_t)(ncp / kL2lNarrow) * kGemmTabStride, 0);
        for (int t = 0; t < ncp / kL2lNarrow; ++t) {
            int* e = &tab_l2l[(size_t)t * kGemmTabStride];
            e[0] = 1;
            e[1] = (nc + 31) / 32;  // columns past nc of the kernel samples are zero
            e[5] = (nc + 31) / 32;
        }
        h->chunks_l2l = (int64_t)(ncp / kGemmBN) * ((nc + 31) / 32);  // per 128 columns of N
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
    h->zf_host = zf;
    DCTPLUS_CUDA_TRY(up(&h->tq_hi, tq_hi));
    DCTPLUS_CUDA_TRY(up(&h->tq_lo, tq_lo));
    DCTPLUS_CUDA_TRY(up(&h->ext_hi, ext_hi));
    DCTPLUS_CUDA_TRY(up(&h->ext_lo, ext_lo));
    DCTPLUS_CUDA_TRY(up(&h->tab_out, tab_out));
    if (form == 2) {
        DCTPLUS_CUDA_TRY(up(&h->tm_hi, tm_hi));
        DCTPLUS_CUDA_TRY(up(&h->tm_lo, tm_lo));
        DCTPLUS_CUDA_TRY(up(&h->m2l, m2l));
        DCTPLUS_CUDA_TRY(up(&h->slot_box, slot_box));
        DCTPLUS_CUDA_TRY(up(&h->chain, chain));
    } else {
        const size_t kf = (size_t)h->ncp * h->ncp;
        double* d_node = nullptr;
        DCTPLUS_CUDA_TRY(up(&d_node, node));
        cudaError_t e = cudaMalloc((void**)&h->kf_hi, sizeof(float) * kf);
        if (e == cudaSuccess) e = cudaMalloc((void**)&h->kf_lo, sizeof(float) * kf);
        if (e == cudaSuccess) {
            k_kf_table<<<(unsigned)((kf + 255) / 256), 256>>>(nleaf, h->ncp, d_node, h->kf_hi, h->kf_lo);
            count_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        cudaFree(d_node);
        DCTPLUS_CUDA_TRY(e);
        DCTPLUS_CUDA_TRY(up(&h->tab_l2l, tab_l2l));
    }
    DCTPLUS_CUDA_TRY(up(&h->row_leaf, row_leaf));
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

// ------------------------------------------------------------- far field tree

// Device view of the tree tables (FP32; the tree runs on the CUDA cores with a lane
// per signal, each 12 x 12 block broadcast from shared memory or L1).
struct FarTree {
    const float* m2l;    // nbox x 4 slots x [12 a][12 b]: kernel samples K(ph_a of B, th_b of C)
    const int* slot_box; // nbox x 4: source box of each slot (within its level), -1 if none
    const float* chain;  // L2L chains [a][b], level l >= 1, leaf position i < 2^l at chain_off[l] + i
    int nlev, nbox;
    int lev_off[kFarMaxLev];
    int box_off[kFarMaxLev + 1];
    int chain_off[kFarMaxLev];
};

constexpr int kTreeThreads = 256;  // signals per CTA (a lane each)

__device__ __forceinline__ void load12(float (&m)[kR], const float* p) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float4 v = __ldg(q + i);
        m[4 * i] = v.x;
        m[4 * i + 1] = v.y;
        m[4 * i + 2] = v.z;
        m[4 * i + 3] = v.w;
    }
}

__device__ __forceinline__ void store12(float* p, const float (&m)[kR]) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int i = 0; i < 3; ++i) q[i] = make_float4(m[4 * i], m[4 * i + 1], m[4 * i + 2], m[4 * i + 3]);
}

// acc[a] += sum_b T[a][b] m[b] (trans: T[b][a]) for a 12 x 12 block T read as float4 rows
// at a warp-uniform address (a broadcast)
template <bool kTrans>
__device__ __forceinline__ void block12(float (&acc)[kR], const float* T, const float (&m)[kR]) {
    const float4* t4 = reinterpret_cast<const float4*>(T);
    if (!kTrans) {
#pragma unroll
        for (int a = 0; a < kR; ++a)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float4 t = t4[a * 3 + q];
                acc[a] = fmaf(t.x, m[4 * q], fmaf(t.y, m[4 * q + 1], fmaf(t.z, m[4 * q + 2], fmaf(t.w, m[4 * q + 3], acc[a]))));
            }
    } else {
#pragma unroll
        for (int b = 0; b < kR; ++b)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float4 t = t4[b * 3 + q];  // T[b][4q .. 4q + 3]
                acc[4 * q] = fmaf(t.x, m[b], acc[4 * q]);
                acc[4 * q + 1] = fmaf(t.y, m[b], acc[4 * q + 1]);
                acc[4 * q + 2] = fmaf(t.z, m[b], acc[4 * q + 2]);
                acc[4 * q + 3] = fmaf(t.w, m[b], acc[4 * q + 3]);
            }
    }
}

// M2L: for every box B of every level, the local expansion
// v^l[B] = sum over B's interaction list of K(l, B, C) M^l[C].
// CTA = (box, kTreeThreads signals); the box's slot blocks are staged in shared memory.
// The output is coefficient-major, vv[(lev_off[l] + B R + a) batch + s], so that a warp's
// stores (and k_far_down's loads) are contiguous across its signals.
__global__ void __launch_bounds__(kTreeThreads, 3) k_far_m2l(const FarTree T, const float* __restrict__ mc,
                                                          float* __restrict__ vv, int64_t ldm, int64_t batch) {
    __shared__ __align__(16) float tk[4 * kR * kR];
    __shared__ int cbox[4];
    const int bg = blockIdx.x;
    int l = 0;
    while (l + 1 < T.nlev && bg >= T.box_off[l + 1]) ++l;
    const int B = bg - T.box_off[l];
    if (threadIdx.x < 4) cbox[threadIdx.x] = __ldg(T.slot_box + bg * 4 + threadIdx.x);
    for (int e = threadIdx.x; e < 4 * kR * kR; e += blockDim.x) tk[e] = __ldg(T.m2l + (size_t)bg * 4 * kR * kR + e);
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.y * kTreeThreads + threadIdx.x;
    if (s >= batch) return;
    float acc[kR] = {};
    const float* row = mc + s * ldm + T.lev_off[l];
#pragma unroll
    for (int sl = 0; sl < 4; ++sl) {  // one list entry at a time; three CTAs per SM hide the loads
        const int Cb = cbox[sl];
        if (Cb < 0) continue;  // uniform across the CTA
        float m[kR];
        load12(m, row + (int64_t)Cb * kR);
        block12<false>(acc, tk + sl * kR * kR, m);
    }
    float* out = vv + (size_t)(T.lev_off[l] + B * kR) * batch + s;
#pragma unroll
    for (int a = 0; a < kR; ++a) out[(size_t)a * batch] = acc[a];
}

// L2L down to the leaves: leaf-local coefficients L[I] = v^0[I] + sum over the upper
// levels l of G(l, I mod 2^l) v^l[I >> l], into the leaf-local array the output
// product reads (leaf I at I R). CTA = (leaf, kTreeThreads signals); the leaf's chain
// blocks are staged in shared memory, and each level's coefficients are loaded (contiguous
// across the warp's signals) while the previous level's product runs.
__global__ void __launch_bounds__(kTreeThreads) k_far_down(const FarTree T, const float* __restrict__ vv,
                                                           float* __restrict__ lc, int64_t ldl, int64_t batch) {
    __shared__ __align__(16) float ch[kFarMaxLev][kR * kR];
    const int I = blockIdx.x;
    for (int e = threadIdx.x; e < (T.nlev - 1) * kR * kR; e += blockDim.x) {
        const int l = 1 + e / (kR * kR), q = e % (kR * kR);
        ch[l][q] = __ldg(T.chain + (size_t)(T.chain_off[l] + (I & ((1 << l) - 1))) * kR * kR + q);
    }
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.y * kTreeThreads + threadIdx.x;
    if (s >= batch) return;
    auto load_level = [&](float (&m)[kR], int l) {
        const float* src = vv + (size_t)(T.lev_off[l] + (I >> l) * kR) * batch + s;
#pragma unroll
        for (int a = 0; a < kR; ++a) m[a] = __ldg(src + (size_t)a * batch);
    };
    float acc[kR], m[kR], mn[kR];
    load_level(acc, 0);
    if (T.nlev > 1) load_level(m, 1);
#pragma unroll 1
    for (int l = 1; l < T.nlev; ++l) {
        if (l + 1 < T.nlev) load_level(mn, l + 1);
        block12<false>(acc, ch[l], m);
#pragma unroll
        for (int a = 0; a < kR; ++a) m[a] = mn[a];
    }
    store12(lc + s * ldl + (int64_t)I * kR, acc);
}

// ------------------------------------------------------------- execute

void* plan_workspace(dctplus_plan_t p, cudaStream_t st, size_t bytes);

// Per batch:
//   1. DCT-II (k_dct_far): s, the leaf moments (P2M), for the tree also the upper
//      levels' moments (M2M), and the dense rows' values, which go to the dense-row
//      slots of the leaf-local array (the slots after them are zeroed);
//   2. far field to the leaf-local coefficients: the leaf-level form is one
//      split-TF32 GEMM with the leaf-to-leaf kernel samples; the tree is M2L
//      (k_far_m2l, every box's local expansion from its interaction list), then L2L
//      (k_far_down, summed down the chains to the leaves);
//   3. output product (split-TF32 GEMM over K segments): per 128-row tile the
//      band of W against its window of s (near field), then the L2P weights
//      against the tile's window of leaf-local coefficients (far field), then
//      the dense rows' slots; y is written once.
// The TF32 remainders of every GEMM operand are formed on chip.
namespace {

// A plan's share of the hierarchical product: its workspace (moments, the tree's M2L output,
// leaf-local coefficients with the dense-row slots) and the DCT-kernel inputs that go with it.
struct HierRun {
    float* mc = nullptr;
    float* vv = nullptr;
    float* lc = nullptr;
    DctFar far{};
};

dctplus_status hier_prepare(dctplus_plan_t p, float* ws, int64_t batch, HierRun* R) {
    HierTables* h = p->hier;
    const bool tree = h->form == 2;
    const size_t mplane = (size_t)batch * h->ldm;
    R->mc = ws;
    R->vv = tree ? ws + mplane : nullptr;
    R->lc = ws + (tree ? 2 : 1) * mplane;
    DctFar& far = R->far;
    far.zf = h->zf;
    far.tq_hi = h->tq_hi;
    far.tq_lo = h->tq_lo;
    far.mc = R->mc;
    far.ldm = h->ldm;
    far.tm_hi = h->tm_hi;
    far.tm_lo = h->tm_lo;
    far.nlev = tree ? h->nlev : 1;
    for (int l = 0; l < kFarMaxLev; ++l) far.lev_off[l] = h->lev_off[l];
    far.out_g = h->out_g;
    far.nout = h->nout;
    far.dv = R->lc + h->dslot;
    far.ldd = h->ldl;
    far.dbase = h->dbase;
    far.dzero = 1;
    far.moments = 1;
    return DCTPLUS_OK;
}

// A plan whose far-field sources equal those of a plan prepared before it (lead): lead's
// moments and leaf-local array, into which it writes its dense rows at its own slots.
void hier_prepare_follower(dctplus_plan_t p, const HierRun& lead, HierRun* R) {
    HierTables* h = p->hier;
    *R = lead;
    R->far.out_g = h->out_g;
    R->far.nout = h->nout;
    R->far.dbase = h->dbase;
    R->far.dzero = 0;
    R->far.moments = 0;
}

// Plans whose far field is the same: equal length and form, and equal z with the same entries
// deflated. The moments, the far field and the leaf-local coefficients depend on nothing else:
// the kernel samples at the Chebyshev nodes, the M2L blocks and the L2L chains are fixed by
// the length.
bool same_far_sources(dctplus_plan_t a, dctplus_plan_t b) {
    const HierTables* ha = a->hier;
    const HierTables* hb = b->hier;
    return a->n == b->n && ha->form == hb->form && ha->zf_host.size() == hb->zf_host.size() &&
           std::memcmp(ha->zf_host.data(), hb->zf_host.data(), sizeof(float) * ha->zf_host.size()) == 0;
}

// Far field of one plan into its leaf-local array: the leaf-to-leaf product, or the tree's
// M2L and downward passes.
dctplus_status hier_far(dctplus_plan_t p, const HierRun& R, int64_t batch, cudaStream_t st) {
    HierTables* h = p->hier;
    if (h->form != 2) {
        GemmSrc l2l{R.mc, nullptr, h->ldm, h->nc, h->kf_hi, h->kf_lo, h->ncp, h->ncp};
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
        const int64_t wide_tiles = (batch + 127) / 128 * (h->ncp / kGemmBN);
        const int bn = 2 * wide_tiles <= sms ? kL2lNarrow : kGemmBN;
        return launch_gemm_tc_segs(&l2l, 1, h->tab_l2l, h->chunks_l2l * (kGemmBN / bn), (double)h->nc, R.lc,
                                   nullptr, h->ldl, (int)batch, h->ncp, st, p->device, "k_gemm_tc", bn);
    }
    FarTree T;
    T.m2l = h->m2l;
    T.slot_box = h->slot_box;
    T.chain = h->chain;
    T.nlev = h->nlev;
    T.nbox = h->nbox;
    for (int l = 0; l < kFarMaxLev; ++l) {
        T.lev_off[l] = h->lev_off[l];
        T.chain_off[l] = h->chain_off[l];
    }
    for (int l = 0; l <= kFarMaxLev; ++l) T.box_off[l] = h->box_off[l];
    const int64_t gy = (batch + kTreeThreads - 1) / kTreeThreads;
    if (gy > 65535) return DCTPLUS_ERR_UNSUPPORTED;
    k_far_m2l<<<dim3((unsigned)h->nbox, (unsigned)gy), kTreeThreads, 0, st>>>(T, R.mc, R.vv, h->ldm, batch);
    note_launch(st, "k_far_m2l", 8.0 * (double)batch * h->ldm, 2.0 * kR * kR * 3.5 * h->nbox * (double)batch);
    DCTPLUS_CUDA_TRY(cudaGetLastError());
    k_far_down<<<dim3((unsigned)h->nleaf, (unsigned)gy), kTreeThreads, 0, st>>>(T, R.vv, R.lc, h->ldl, batch);
    note_launch(st, "k_far_down", 4.0 * (double)batch * (h->ldm + h->nc),
                2.0 * kR * kR * (h->nlev - 1) * h->nleaf * (double)batch);
    DCTPLUS_CUDA_TRY(cudaGetLastError());
    return DCTPLUS_OK;
}

// The output product of one plan from s and its leaf-local array: near-field band, L2P of
// the far field and the dense rows.
dctplus_status hier_out(dctplus_plan_t p, const HierRun& R, const float* s_hi, float* y, int64_t ldy,
                        int64_t batch, cudaStream_t st) {
    HierTables* h = p->hier;
    const int n = p->n;
    GemmSrc out[2] = {{s_hi, nullptr, n, n, h->slab_hi, h->slab_lo, h->Kw, h->Kw},
                      {R.lc, nullptr, h->ldl, h->ldl, h->ext_hi, h->ext_lo, h->Kx + 32, h->Kx + 32}};
    return launch_gemm_tc_segs(out, 2, h->tab_out, h->chunks_out, h->acols_out, y, nullptr, ldy,
                               (int)batch, n, st, p->device, "k_gemm_tc");
}

}  // namespace

dctplus_status launch_hier(dctplus_plan_t p, const float* x, int64_t ldx, float* y, int64_t ldy,
                           int64_t batch, cudaStream_t st) {
    return launch_hier_multi(&p, 1, x, ldx, &y, ldy, batch, st);
}

// Several plans of one length over the same signals: one DCT-II (with the moments of every
// distinct far field and every plan's dense rows), then the far fields and each plan's output
// product into ys[k]. s lives in plan 0's workspace. Plans that share v (updates that differ
// in rho only, the progressive case) share z, so their far field is formed once.
dctplus_status launch_hier_multi(const dctplus_plan_t* plans, int K, const float* x, int64_t ldx,
                                 float* const* ys, int64_t ldy, int64_t batch, cudaStream_t st) {
    if (K < 1 || K > kFarMaxPlans || batch > INT32_MAX || (ldy & 3)) return DCTPLUS_ERR_UNSUPPORTED;
    const int n = plans[0]->n;
    for (int k = 0; k < K; ++k)
        if (!plans[k]->hier || plans[k]->n != n || plans[k]->device != plans[0]->device ||
            (reinterpret_cast<uintptr_t>(ys[k]) & 15))
            return DCTPLUS_ERR_UNSUPPORTED;
    if (batch <= 0) return DCTPLUS_OK;
    // plans with the same far-field sources share the first one's moments, far field and
    // leaf-local coefficients (lead[k] = that plan); in the set each lead is followed by the
    // plans that share its sources
    int lead[kFarMaxPlans], order[kFarMaxPlans], nset = 0;
    bool shared = false;
    for (int k = 0; k < K; ++k) {
        lead[k] = k;
        for (int j = 0; j < k && lead[k] == k; ++j) {
            if (lead[j] != j || !same_far_sources(plans[j], plans[k])) continue;
            bool apart = true;  // its dense-row slots differ from those of every plan in j's group
            for (int i = 0; i < k; ++i)
                if (lead[i] == j && plans[i]->hier->dbase == plans[k]->hier->dbase) apart = false;
            if (apart) lead[k] = j;
        }
        shared = shared || lead[k] != k;
    }
    for (int k = 0; k < K; ++k)
        if (lead[k] == k)
            for (int j = k; j < K; ++j)
                if (lead[j] == k) order[nset++] = j;
    HierRun runs[kFarMaxPlans];
    float* s_hi = nullptr;
    for (int k = 0; k < K; ++k) {  // leads: plan 0 is one, and its workspace also holds s
        if (lead[k] != k) continue;
        HierTables* h = plans[k]->hier;
        const size_t plane = k == 0 ? (size_t)batch * n : 0;
        const size_t mplane = (size_t)batch * h->ldm, lplane = (size_t)batch * h->ldl;
        float* ws = static_cast<float*>(
            plan_workspace(plans[k], st, sizeof(float) * (plane + (h->form == 2 ? 2 : 1) * mplane + lplane)));
        if (!ws) return DCTPLUS_ERR_CUDA;
        if (k == 0) s_hi = ws;
        dctplus_status r = hier_prepare(plans[k], ws + plane, batch, &runs[k]);
        if (r != DCTPLUS_OK) return r;
    }
    for (int k = 0; k < K; ++k)
        if (lead[k] != k) hier_prepare_follower(plans[k], runs[lead[k]], &runs[k]);
    DctFarSet set;
    set.K = K;
    for (int i = 0; i < K; ++i) set.f[i] = runs[order[i]].far;
    dctplus_status r = launch_dct_far_multi(plans[0], x, ldx, s_hi, n, batch, set, st);
    if (r != DCTPLUS_OK) return r;
    const int dev = plans[0]->device;
    if (!shared) {
        // The plans' far fields and output products depend on the shared DCT only: the plans
        // after the first run on side streams, so that their products fill the SMs the others
        // leave idle (a leaf-to-leaf product of fewer tiles than SMs, the last wave of an
        // output product).
        return run_forked(dev, st, K, [&](int k, cudaStream_t sk) {
            dctplus_status rk = hier_far(plans[k], runs[k], batch, sk);
            return rk != DCTPLUS_OK ? rk : hier_out(plans[k], runs[k], s_hi, ys[k], ldy, batch, sk);
        });
    }
    // each distinct far field once into its lead's leaf-local array, which the plans sharing it
    // read in place (each with its own dense-row slots), then every plan's output product
    for (int k = 0; k < K; ++k)
        if (lead[k] == k && (r = hier_far(plans[k], runs[k], batch, st)) != DCTPLUS_OK) return r;
    return run_forked(dev, st, K, [&](int k, cudaStream_t sk) {
        return hier_out(plans[k], runs[k], s_hi, ys[k], ldy, batch, sk);
    });
}

}  // namespace dctplus
