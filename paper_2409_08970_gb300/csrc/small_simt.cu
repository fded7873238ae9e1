// CUDA-core kernels for short signals (n <= 64): the whole transform of one
// signal (Algorithm 1: DCT-II, then the Cauchy product with a and z folded
// into W = X^T U) runs in one thread's registers, with U^T and W staged in
// shared memory. Used for FP64 data (n <= 64), for lengths that are not
// powers of two, and for every n <= 64 when the tensor-core kernel is off.
//
// Work is cut into tiles of whole signals (at most kTileElems samples); a
// persistent grid walks a tile list, so one launch serves a mixed batch of
// plans with different n (the grouped execute).
#include <algorithm>

#include "internal.cuh"

namespace dctplus {

struct SmallPlanDev {
    int n;
    int np;            // next power of two >= n
    const void* ct;    // n x n, U^T row-major (T)
    const void* w;     // n x n, W row-major (T)
};

// seg = {plan index, element offset, rows}; tile = {segment, first row, rows}
struct SmallTile {
    int seg;
    int row0;
    int rows;
};

template <typename T>
struct SmallCfg;
template <>
struct SmallCfg<float> { static constexpr int kTileElems = 8192; };
template <>
struct SmallCfg<double> { static constexpr int kTileElems = 4096; };

__host__ __device__ constexpr int next_pow2_small(int n) {
    return n <= 2 ? 2 : n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : n <= 32 ? 32 : 64;
}

template <typename T>
__host__ __device__ constexpr size_t small_smem_bytes() {
    // two 64x64 tables + the largest tile (rows * (np+1)), rows = kTileElems / n
    return sizeof(T) * (2 * 64 * 64 + 2 * SmallCfg<T>::kTileElems + 64);
}

// y = W (U^T x) for one signal held in smem row `row` (stride 1), tables ct/w
// of size NP x NP (zero padded), in place.
template <typename T, int NP>
__device__ __forceinline__ void row_transform(const T* __restrict__ ct, const T* __restrict__ w,
                                              T* row) {
    T r[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) r[j] = row[j];
#pragma unroll 1
    for (int k = 0; k < NP; ++k) {
        T a0 = 0, a1 = 0;
#pragma unroll
        for (int j = 0; j < NP; j += 2) {
            a0 = fma(ct[k * NP + j], r[j], a0);
            a1 = fma(ct[k * NP + j + 1], r[j + 1], a1);
        }
        row[k] = a0 + a1;
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) r[j] = row[j];
#pragma unroll 1
    for (int i = 0; i < NP; ++i) {
        T a0 = 0, a1 = 0;
#pragma unroll
        for (int k = 0; k < NP; k += 2) {
            a0 = fma(w[i * NP + k], r[k], a0);
            a1 = fma(w[i * NP + k + 1], r[k + 1], a1);
        }
        row[i] = a0 + a1;
    }
}

// Launch description. Grouped runs pass device arrays of plans, segments and
// tiles; a one-plan run passes its plan by value and tiles arithmetically.
struct SmallLaunch {
    const SmallPlanDev* plans;  // nullptr: use `single`
    SmallPlanDev single;
    const int64_t* segs;
    const SmallTile* tiles;
    int ntiles;
    int per;        // rows per tile of a one-plan run
    int64_t batch;  // rows of a one-plan run
};

template <typename T>
__global__ void __launch_bounds__(256) k_small_simt(SmallLaunch L, const T* __restrict__ x,
                                                    int64_t ldx, T* __restrict__ y, int64_t ldy,
                                                    unsigned* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* ct = reinterpret_cast<T*>(smem_raw);
    T* w = ct + 64 * 64;
    T* tile = w + 64 * 64;
    int cur_plan = -1;
    for (int t = blockIdx.x; t < L.ntiles; t += gridDim.x) {
        SmallTile tl;
        int pidx;
        int64_t off;
        SmallPlanDev pd;
        if (L.plans) {
            tl = L.tiles[t];
            pidx = (int)L.segs[3 * tl.seg + 0];
            off = L.segs[3 * tl.seg + 1];
            pd = L.plans[pidx];
        } else {
            tl.seg = 0;
            tl.row0 = t * L.per;
            tl.rows = (int)min((int64_t)L.per, L.batch - (int64_t)tl.row0);
            pidx = 0;
            off = 0;
            pd = L.single;
        }
        const int n = pd.n, np = pd.np, stride = np + 1;
        if (tl.rows * stride > 2 * SmallCfg<T>::kTileElems + 64 || n > 64 || n < 2) {
            if (threadIdx.x == 0) atomicOr(err, kErrIndex);
            continue;
        }
        // ldx/ldy < 0 means packed rows of the segment's own n
        const int64_t lx = ldx < 0 ? n : ldx, ly = ldy < 0 ? n : ldy;
        __syncthreads();  // previous tile fully stored before smem is reused
        if (pidx != cur_plan) {
            const T* gct = static_cast<const T*>(pd.ct);
            const T* gw = static_cast<const T*>(pd.w);
            for (int e = threadIdx.x; e < np * np; e += blockDim.x) {
                int r = e / np, c = e % np;
                bool in = r < n && c < n;
                ct[e] = in ? gct[r * n + c] : T(0);
                w[e] = in ? gw[r * n + c] : T(0);
            }
            cur_plan = pidx;
        }
        const T* xs = x + off + (int64_t)tl.row0 * lx;
        for (int e = threadIdx.x; e < tl.rows * np; e += blockDim.x) {
            int r = e / np, c = e % np;
            tile[r * stride + c] = c < n ? xs[(int64_t)r * lx + c] : T(0);
        }
        __syncthreads();
        for (int r = threadIdx.x; r < tl.rows; r += blockDim.x) {
            T* row = tile + r * stride;
            switch (np) {
                case 2: row_transform<T, 2>(ct, w, row); break;
                case 4: row_transform<T, 4>(ct, w, row); break;
                case 8: row_transform<T, 8>(ct, w, row); break;
                case 16: row_transform<T, 16>(ct, w, row); break;
                case 32: row_transform<T, 32>(ct, w, row); break;
                default: row_transform<T, 64>(ct, w, row); break;
            }
        }
        __syncthreads();
        T* ys = y + off + (int64_t)tl.row0 * ly;
        for (int e = threadIdx.x; e < tl.rows * n; e += blockDim.x) {
            int r = e / n, c = e % n;
            ys[(int64_t)r * ly + c] = tile[r * stride + c];
        }
    }
}

// ---------------------------------------------------------------- host side

template <typename T>
static int tile_rows(int n) {
    return std::max(1, SmallCfg<T>::kTileElems / n);
}

// Builds the tile list for segments {plan, offset, rows}.
template <typename T>
static void make_tiles(const std::vector<int64_t>& seg, const std::vector<int>& plan_n,
                       std::vector<SmallTile>& tiles) {
    tiles.clear();
    int nseg = (int)seg.size() / 3;
    for (int s = 0; s < nseg; ++s) {
        int n = plan_n[(int)seg[3 * s]];
        int64_t rows = seg[3 * s + 2];
        int per = tile_rows<T>(n);
        for (int64_t r0 = 0; r0 < rows; r0 += per)
            tiles.push_back({s, (int)r0, (int)std::min<int64_t>(per, rows - r0)});
    }
}

static int sm_count(int dev) {
    static int cached[64] = {0};
    if (dev < 0 || dev >= 64) return 148;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 148;
    }
    return cached[dev];
}

template <typename T>
static dctplus_status launch_small_common(const SmallLaunch& L, const T* x, int64_t ldx, T* y,
                                          int64_t ldy, cudaStream_t s, int dev, double samples,
                                          double flops) {
    if (L.ntiles == 0) return DCTPLUS_OK;
    size_t smem = small_smem_bytes<T>();
    static bool attr_set[2][64] = {};
    bool& done = attr_set[sizeof(T) == 8][dev & 63];
    if (!done) {
        DCTPLUS_CUDA_TRY(cudaFuncSetAttribute(k_small_simt<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        done = true;
    }
    int per_sm = sizeof(T) == 4 ? 2 : 1;
    int grid = std::min(L.ntiles, sm_count(dev) * per_sm);
    k_small_simt<T><<<grid, 256, smem, s>>>(L, x, ldx, y, ldy, device_error_word(dev));
    note_launch(s, sizeof(T) == 4 ? "k_small_simt<float>" : "k_small_simt<double>",
                2.0 * sizeof(T) * samples, flops);
    DCTPLUS_CUDA_TRY(cudaGetLastError());
    return DCTPLUS_OK;
}

template <typename T>
static dctplus_status launch_small_single(dctplus_plan_t p, const T* x, int64_t ldx, T* y,
                                          int64_t ldy, int64_t batch, cudaStream_t s) {
    SmallLaunch L{};
    L.single.n = p->n;
    L.single.np = next_pow2_small(p->n);
    L.single.ct = sizeof(T) == 4 ? (const void*)p->d_ct32 : (const void*)p->d_ct64;
    L.single.w = sizeof(T) == 4 ? (const void*)p->d_w32 : (const void*)p->d_w64;
    if (!L.single.ct || !L.single.w) return DCTPLUS_ERR_UNSUPPORTED;
    L.per = tile_rows<T>(p->n);
    int64_t nt = (batch + L.per - 1) / L.per;
    if (nt > INT32_MAX) return DCTPLUS_ERR_UNSUPPORTED;
    L.ntiles = (int)nt;
    L.batch = batch;
    const double samples = (double)batch * p->n;
    return launch_small_common<T>(L, x, ldx, y, ldy, s, p->device, samples, 4.0 * p->n * samples);
}

dctplus_status launch_small_simt_f32(dctplus_plan_t p, const float* x, int64_t ldx, float* y,
                                     int64_t ldy, int64_t batch, cudaStream_t s) {
    return launch_small_single<float>(p, x, ldx, y, ldy, batch, s);
}


// -------------------------------------------------------------- grouped runs

dctplus_status group_prepare(dctplus_group_t g, const int64_t* seg_host, int nseg,
                             cudaStream_t s) {
    std::vector<int64_t> seg(seg_host, seg_host + 3 * (size_t)nseg);
    if (seg == g->seg_cache && g->d_seg) return DCTPLUS_OK;
    std::vector<int> plan_n;
    for (auto p : g->plans) plan_n.push_back(p->n);
    std::vector<SmallTile> tiles;
    make_tiles<float>(seg, plan_n, tiles);
    if (nseg > g->seg_cap) {
        if (g->d_seg) cudaFree(g->d_seg);
        g->seg_cap = nseg;
        DCTPLUS_CUDA_TRY(cudaMalloc((void**)&g->d_seg, sizeof(int64_t) * 3 * std::max(nseg, 1)));
    }
    if ((int)tiles.size() > g->tile_cap) {
        if (g->d_tiles) cudaFree(g->d_tiles);
        g->tile_cap = (int)tiles.size();
        DCTPLUS_CUDA_TRY(cudaMalloc((void**)&g->d_tiles, sizeof(SmallTile) * std::max<size_t>(tiles.size(), 1)));
    }
    if (nseg)
        DCTPLUS_CUDA_TRY(cudaMemcpyAsync(g->d_seg, seg.data(), sizeof(int64_t) * seg.size(), cudaMemcpyHostToDevice, s));
    if (!tiles.empty())
        DCTPLUS_CUDA_TRY(cudaMemcpyAsync(g->d_tiles, tiles.data(), sizeof(SmallTile) * tiles.size(), cudaMemcpyHostToDevice, s));
    g->ntiles = (int)tiles.size();
    g->seg_cache = seg;
    return DCTPLUS_OK;
}

dctplus_status group_upload_plans(dctplus_group_t g) {
    std::vector<SmallPlanDev> pds;
    for (auto p : g->plans) {
        SmallPlanDev pd;
        pd.n = p->n;
        pd.np = next_pow2_small(p->n);
        pd.ct = p->d_ct32;
        pd.w = p->d_w32;
        pds.push_back(pd);
    }
    DCTPLUS_CUDA_TRY(cudaMalloc(&g->d_plan_tables, sizeof(SmallPlanDev) * std::max<size_t>(pds.size(), 1)));
    DCTPLUS_CUDA_TRY(cudaMemcpy(g->d_plan_tables, pds.data(), sizeof(SmallPlanDev) * pds.size(), cudaMemcpyHostToDevice));
    return DCTPLUS_OK;
}

dctplus_status launch_group_simt(dctplus_group_t g, const float* x, float* y, cudaStream_t s) {
    SmallLaunch L{};
    L.plans = static_cast<const SmallPlanDev*>(g->d_plan_tables);
    L.segs = g->d_seg;
    L.tiles = reinterpret_cast<const SmallTile*>(g->d_tiles);
    L.ntiles = g->ntiles;
    double samples = 0.0, flops = 0.0;
    for (size_t i = 0; i + 2 < g->seg_cache.size(); i += 3) {
        const double rows_n = (double)g->seg_cache[i + 2] * g->plans[g->seg_cache[i]]->n;
        samples += rows_n;
        flops += 4.0 * g->plans[g->seg_cache[i]]->n * rows_n;
    }
    return launch_small_common<float>(L, x, -1, y, -1, s, g->device, samples, flops);
}

}  // namespace dctplus
