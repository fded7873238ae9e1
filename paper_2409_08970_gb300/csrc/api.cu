// C ABI entry points: argument checks, plan lifetime, dispatch to kernels.
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

#include "internal.cuh"

namespace dctplus {

dctplus_status launch_small_tc(dctplus_plan_t p, const float* x, int64_t ldx, float* y,
                               int64_t ldy, int64_t batch, cudaStream_t s);  // small_tc.cu
bool small_tc_available(dctplus_plan_t p);                                   // small_tc.cu
dctplus_status group_prepare(dctplus_group_t g, const int64_t* seg_host, int nseg,
                             cudaStream_t s);                                // small_simt.cu
dctplus_status group_upload_plans(dctplus_group_t g);                        // small_simt.cu
dctplus_status launch_group_simt(dctplus_group_t g, const float* x, float* y, cudaStream_t s);

static std::mutex g_err_mu;
static unsigned* g_err_words[64] = {};

unsigned* device_error_word(int device) {
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_err_mu);
    if (!g_err_words[device]) {
        unsigned* w = nullptr;
        if (cudaMalloc((void**)&w, sizeof(unsigned)) != cudaSuccess) return nullptr;
        cudaMemset(w, 0, sizeof(unsigned));
        g_err_words[device] = w;
    }
    return g_err_words[device];
}

// Per-(plan, stream) scratch, grown on demand. The first call on a stream
// allocates, so it must precede any stream capture.
struct Workspace {
    cudaStream_t stream;
    void* ptr;
    size_t bytes;
};
static std::mutex g_ws_mu;

struct PlanWs {
    dctplus_plan_t plan;
    std::vector<Workspace> ws;
};
static std::vector<PlanWs> g_ws;

void* plan_workspace(dctplus_plan_t p, cudaStream_t st, size_t bytes) {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    PlanWs* pw = nullptr;
    for (auto& e : g_ws)
        if (e.plan == p) pw = &e;
    if (!pw) { g_ws.push_back({p, {}}); pw = &g_ws.back(); }
    for (auto& w : pw->ws) {
        if (w.stream != st) continue;
        if (w.bytes >= bytes) return w.ptr;
        cudaStreamSynchronize(st);
        cudaFree(w.ptr);
        w.ptr = nullptr;
        if (cudaMalloc(&w.ptr, bytes) != cudaSuccess) { w.bytes = 0; return nullptr; }
        w.bytes = bytes;
        return w.ptr;
    }
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(bytes, 256)) != cudaSuccess) return nullptr;
    pw->ws.push_back({st, q, std::max<size_t>(bytes, 256)});
    return q;
}

static void release_workspaces(dctplus_plan_t p) {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    for (size_t i = 0; i < g_ws.size(); ++i) {
        if (g_ws[i].plan != p) continue;
        for (auto& w : g_ws[i].ws) cudaFree(w.ptr);
        g_ws.erase(g_ws.begin() + i);
        return;
    }
}

static bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

static dctplus_status check_device(int want) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return DCTPLUS_ERR_NO_DEVICE;
    return cur == want ? DCTPLUS_OK : DCTPLUS_ERR_INVALID_ARG;
}

// Host-buffer execution in chunks so that the host-to-device copy of chunk c + 1,
// the kernel of chunk c and the device-to-host copy of chunk c - 1 overlap (three
// streams: the caller's for uploads, two of the group's for kernels and downloads).
// Segments are cut at whole 128-row tiles of packed rows (8192 samples), so every
// piece is a valid tensor-core segment; each chunk copies the address range its
// pieces cover, merged where pieces touch.
constexpr int64_t kPipeMinElems = int64_t(1) << 22;  // below this one pass is as fast
constexpr int kPipeChunks = 8;
constexpr int64_t kPipeCut = 128 * 64;                // samples per tensor-core tile

static dctplus_status group_host_pipelined(dctplus_group_t g, const float* x_host, float* y_host,
                                           float* dx, float* dy, const int64_t* seg, int nseg,
                                           cudaStream_t up) {
    if (!g->pipe_compute) {
        DCTPLUS_CUDA_TRY(cudaStreamCreateWithFlags(&g->pipe_compute, cudaStreamNonBlocking));
        DCTPLUS_CUDA_TRY(cudaStreamCreateWithFlags(&g->pipe_d2h, cudaStreamNonBlocking));
        for (int i = 0; i < 2 * kPipeChunks + 1; ++i) {
            cudaEvent_t e;
            DCTPLUS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            g->pipe_events.push_back(e);
        }
    }
    // pieces: (plan, offset, rows), in the callers' segment order
    struct Piece { dctplus_plan_t p; int64_t off, rows, elems; };
    std::vector<Piece> pieces;
    int64_t total = 0;
    for (int i = 0; i < nseg; ++i) {
        const int64_t rows = seg[3 * i + 2];
        if (rows > 0) total += rows * g->plans[seg[3 * i]]->n;
    }
    const int64_t target = (total + kPipeChunks - 1) / kPipeChunks;
    std::vector<std::vector<Piece>> chunks(1);
    int64_t in_chunk = 0;
    for (int i = 0; i < nseg; ++i) {
        dctplus_plan_t p = g->plans[seg[3 * i]];
        const int n = p->n;
        int64_t off = seg[3 * i + 1], rows = seg[3 * i + 2];
        while (rows > 0) {
            if (in_chunk >= target && (int)chunks.size() < kPipeChunks) {
                chunks.emplace_back();
                in_chunk = 0;
            }
            int64_t take = rows;
            const int64_t room = target - in_chunk;
            if ((int)chunks.size() < kPipeChunks && rows * n > room) {
                // cut at a whole tile of packed rows, at least one tile
                const int64_t tiles = std::max<int64_t>(1, room / kPipeCut);
                take = std::min<int64_t>(rows, tiles * kPipeCut / n);
            }
            chunks.back().push_back({p, off, take, take * n});
            in_chunk += take * n;
            off += take * n;
            rows -= take;
        }
    }
    cudaEvent_t done_up = g->pipe_events[2 * kPipeChunks];
    for (size_t c = 0; c < chunks.size(); ++c) {
        // address ranges of this chunk, merged where pieces touch
        std::vector<std::pair<int64_t, int64_t>> ranges;
        for (const Piece& q : chunks[c]) {
            if (!ranges.empty() && ranges.back().second == q.off) ranges.back().second = q.off + q.elems;
            else ranges.push_back({q.off, q.off + q.elems});
        }
        for (auto& r : ranges)
            DCTPLUS_CUDA_TRY(cudaMemcpyAsync(dx + r.first, x_host + r.first,
                                             sizeof(float) * (r.second - r.first),
                                             cudaMemcpyHostToDevice, up));
        cudaEvent_t ev_up = g->pipe_events[2 * c], ev_k = g->pipe_events[2 * c + 1];
        DCTPLUS_CUDA_TRY(cudaEventRecord(ev_up, up));
        DCTPLUS_CUDA_TRY(cudaStreamWaitEvent(g->pipe_compute, ev_up, 0));
        std::vector<TcSegHost> tc;
        for (const Piece& q : chunks[c]) tc.push_back({q.p, dx + q.off, dy + q.off, q.rows});
        dctplus_status st = launch_tc_segments(tc, g->pipe_compute, g->device);
        if (st != DCTPLUS_OK) return st;
        DCTPLUS_CUDA_TRY(cudaEventRecord(ev_k, g->pipe_compute));
        DCTPLUS_CUDA_TRY(cudaStreamWaitEvent(g->pipe_d2h, ev_k, 0));
        for (auto& r : ranges)
            DCTPLUS_CUDA_TRY(cudaMemcpyAsync(y_host + r.first, dy + r.first,
                                             sizeof(float) * (r.second - r.first),
                                             cudaMemcpyDeviceToHost, g->pipe_d2h));
    }
    DCTPLUS_CUDA_TRY(cudaEventRecord(done_up, g->pipe_d2h));
    DCTPLUS_CUDA_TRY(cudaStreamWaitEvent(up, done_up, 0));  // the caller's stream sees the result
    DCTPLUS_CUDA_TRY(cudaStreamSynchronize(g->pipe_d2h));
    DCTPLUS_CUDA_TRY(cudaStreamSynchronize(up));
    return DCTPLUS_OK;
}

}  // namespace dctplus

// ------------------------------------------------------------ kernel trace

namespace dctplus {

struct TraceRec {
    const char* name;
    double bytes, flops;
    cudaEvent_t ev;
};

static std::mutex g_trace_mu;
static cudaStream_t g_trace_stream = nullptr;
static bool g_trace_on = false;
static cudaEvent_t g_trace_start = nullptr;
static std::vector<TraceRec> g_trace;
static std::vector<cudaEvent_t> g_trace_pool;

static cudaEvent_t trace_event() {
    if (!g_trace_pool.empty()) {
        cudaEvent_t e = g_trace_pool.back();
        g_trace_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void note_launch(cudaStream_t s, const char* name, double bytes, double flops) {
    count_launch();
    std::lock_guard<std::mutex> lk(g_trace_mu);
    if (!g_trace_on || s != g_trace_stream) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    cudaEvent_t e = trace_event();
    if (!e) return;
    cudaEventRecord(e, s);
    g_trace.push_back({name, bytes, flops, e});
}

struct SideSet {
    int dev;
    cudaStream_t caller;
    SideStreams s;
};
static std::mutex g_side_mu;
static std::vector<SideSet*> g_side;  // kept until exit: a graph captured on the caller's stream may hold them

const SideStreams* side_streams(int dev, cudaStream_t caller) {
    {
        // the kernel trace times the launches one after another on the traced stream
        std::lock_guard<std::mutex> lk(g_trace_mu);
        if (g_trace_on && caller == g_trace_stream) return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_side_mu);
    for (SideSet* e : g_side)
        if (e->dev == dev && e->caller == caller) return &e->s;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(caller, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    SideSet* e = new (std::nothrow) SideSet{dev, caller, {}};
    if (!e) return nullptr;
    bool ok = cudaEventCreateWithFlags(&e->s.fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < kFarMaxPlans - 1 && ok; ++k)
        ok = cudaStreamCreateWithFlags(&e->s.side[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&e->s.join[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        if (e->s.fork) cudaEventDestroy(e->s.fork);
        for (int k = 0; k < kFarMaxPlans - 1; ++k) {
            if (e->s.side[k]) cudaStreamDestroy(e->s.side[k]);
            if (e->s.join[k]) cudaEventDestroy(e->s.join[k]);
        }
        delete e;
        return nullptr;
    }
    g_side.push_back(e);
    return &e->s;
}

}  // namespace dctplus

using namespace dctplus;

extern "C" {

const char* dctplus_status_string(dctplus_status s) {
    switch (s) {
        case DCTPLUS_OK: return "ok";
        case DCTPLUS_ERR_INVALID_ARG: return "invalid argument";
        case DCTPLUS_ERR_UNSUPPORTED: return "unsupported configuration";
        case DCTPLUS_ERR_NOT_CONVERGED: return "secular root iteration did not converge";
        case DCTPLUS_ERR_CUDA: return "CUDA runtime error";
        case DCTPLUS_ERR_TIMEOUT: return "bounded device wait timed out";
        case DCTPLUS_ERR_DEVICE_CHECK: return "device-side check failed";
        case DCTPLUS_ERR_NO_DEVICE: return "no CUDA device";
        case DCTPLUS_ERR_SCRATCH_LIMIT:
            return "batch * n exceeds the fixed scratch of dctplus_execute_noalloc (2^22 samples)";
    }
    return "unknown status";
}

int64_t dctplus_launch_count(void) { return g_launches.load(); }


dctplus_status dctplus_trace_begin(dctplus_stream_t stream) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(g_trace_mu);
    if (g_trace_on) return DCTPLUS_ERR_INVALID_ARG;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    DCTPLUS_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return DCTPLUS_ERR_INVALID_ARG;
    if (!g_trace_start) DCTPLUS_CUDA_TRY(cudaEventCreate(&g_trace_start));
    DCTPLUS_CUDA_TRY(cudaEventRecord(g_trace_start, s));
    g_trace_stream = s;
    g_trace_on = true;
    return DCTPLUS_OK;
}

int dctplus_trace_end(dctplus_stream_t stream, const char** names, float* ms, double* bytes,
                      double* flops, int cap) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(g_trace_mu);
    if (!g_trace_on || s != g_trace_stream) return -1;
    g_trace_on = false;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    const int cnt = (int)g_trace.size();
    cudaEvent_t prev = g_trace_start;
    for (int i = 0; i < cnt; ++i) {
        if (i < cap) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, prev, g_trace[i].ev) != cudaSuccess) t = -1.f;
            if (names) names[i] = g_trace[i].name;
            if (ms) ms[i] = t;
            if (bytes) bytes[i] = g_trace[i].bytes;
            if (flops) flops[i] = g_trace[i].flops;
        }
        prev = g_trace[i].ev;
    }
    for (auto& r : g_trace) g_trace_pool.push_back(r.ev);
    g_trace.clear();
    return cnt;
}

dctplus_status dctplus_plan(dctplus_plan_t* out, int n, const double* v_host, double rho,
                            const dctplus_opts* opts) {
    if (!out) return DCTPLUS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!v_host || n < 2 || n > kMaxN || !std::isfinite(rho)) return DCTPLUS_ERR_INVALID_ARG;
    for (int j = 0; j < n; ++j)
        if (!std::isfinite(v_host[j])) return DCTPLUS_ERR_INVALID_ARG;
    dctplus_opts o{};
    o.device = -1;
    if (opts) o = *opts;
    if (o.cauchy_mode < 0 || o.cauchy_mode > DCTPLUS_CAUCHY_NFST || o.max_secular_iter < 0 ||
        o.far_field < 0 || o.far_field > 2)
        return DCTPLUS_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return DCTPLUS_ERR_NO_DEVICE;
    int dev = o.device;
    if (dev < 0) {
        if (cudaGetDevice(&dev) != cudaSuccess) return DCTPLUS_ERR_NO_DEVICE;
    } else {
        if (dev >= ndev) return DCTPLUS_ERR_INVALID_ARG;
        if (cudaSetDevice(dev) != cudaSuccess) return DCTPLUS_ERR_CUDA;
    }
    dctplus_plan_s* p = new (std::nothrow) dctplus_plan_s();
    if (!p) return DCTPLUS_ERR_CUDA;
    p->n = n;
    p->rho = rho;
    p->device = dev;
    p->v.assign(v_host, v_host + n);
    p->cauchy_mode = o.cauchy_mode;
    p->far_field = o.far_field;
    dctplus_status st = build_plan(p, o);
    if (st != DCTPLUS_OK) {
        free_plan_tables(p);
        delete p;
        return st;
    }
    *out = p;
    return DCTPLUS_OK;
}

void dctplus_destroy(dctplus_plan_t p) {
    if (!p) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    release_workspaces(p);
    pruned_forget(p);
    free_plan_tables(p);
    if (cur >= 0 && cur != p->device) cudaSetDevice(cur);
    delete p;
}

int dctplus_plan_size(dctplus_plan_t p) { return p ? p->n : -1; }

int dctplus_plan_cauchy_mode(dctplus_plan_t p) { return p ? p->cauchy_mode : -1; }

int dctplus_plan_far_field(dctplus_plan_t p) {
    return p && p->cauchy_mode == DCTPLUS_CAUCHY_HIER ? p->far_field : 0;
}

dctplus_status dctplus_plan_inspect(dctplus_plan_t p, double* eigenvalues, double* z,
                                    int* row_kind, int* row_pole, double* row_tau,
                                    double* row_a) {
    if (!p) return DCTPLUS_ERR_INVALID_ARG;
    size_t n = (size_t)p->n;
    if (eigenvalues) memcpy(eigenvalues, p->eig.data(), sizeof(double) * n);
    if (z) memcpy(z, p->z.data(), sizeof(double) * n);
    if (row_kind) memcpy(row_kind, p->row_kind.data(), sizeof(int) * n);
    if (row_pole) memcpy(row_pole, p->row_pole.data(), sizeof(int) * n);
    if (row_tau) memcpy(row_tau, p->row_tau.data(), sizeof(double) * n);
    if (row_a) memcpy(row_a, p->row_a.data(), sizeof(double) * n);
    return DCTPLUS_OK;
}

static dctplus_status check_exec_args(dctplus_plan_t p, dctplus_dtype dtype, const void* x,
                                      int64_t ldx, const void* y, int64_t ldy, int64_t batch) {
    if (!p || batch < 0) return DCTPLUS_ERR_INVALID_ARG;
    if (dtype != DCTPLUS_F32 && dtype != DCTPLUS_F64) return DCTPLUS_ERR_INVALID_ARG;
    if (batch == 0) return DCTPLUS_OK;
    if (!x || !y || x == y) return DCTPLUS_ERR_INVALID_ARG;
    if (ldx < p->n || ldy < p->n) return DCTPLUS_ERR_INVALID_ARG;
    size_t es = dtype == DCTPLUS_F32 ? 4 : 8;
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & (es - 1))
        return DCTPLUS_ERR_INVALID_ARG;
    // reject overlapping x / y ranges
    uintptr_t xa = (uintptr_t)x, ya = (uintptr_t)y;
    uintptr_t xe = xa + es * (size_t)((batch - 1) * ldx + p->n);
    uintptr_t ye = ya + es * (size_t)((batch - 1) * ldy + p->n);
    if (xa < ye && ya < xe) return DCTPLUS_ERR_INVALID_ARG;
    return DCTPLUS_OK;
}

dctplus_status dctplus_execute(dctplus_plan_t p, dctplus_dtype dtype, const void* x_dev,
                               int64_t ldx, void* y_dev, int64_t ldy, int64_t batch,
                               dctplus_stream_t stream) {
    dctplus_status st = check_exec_args(p, dtype, x_dev, ldx, y_dev, ldy, batch);
    if (st != DCTPLUS_OK || batch == 0) return st;
    if ((st = check_device(p->device)) != DCTPLUS_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int n = p->n;
    if (p->cauchy_mode == DCTPLUS_CAUCHY_NFST) {  // the paper's trigonometric route, FP64 inside
        if (dtype == DCTPLUS_F64)
            return launch_nfst<double>(p, static_cast<const double*>(x_dev), ldx,
                                       static_cast<double*>(y_dev), ldy, batch, s);
        return launch_nfst<float>(p, static_cast<const float*>(x_dev), ldx, static_cast<float*>(y_dev),
                                  ldy, batch, s);
    }
    if (dtype == DCTPLUS_F64) {
        if (n > kF64Max) return DCTPLUS_ERR_UNSUPPORTED;
        if (n > kSmallMax)
            return launch_dense_f64(p, static_cast<const double*>(x_dev), ldx,
                                    static_cast<double*>(y_dev), ldy, batch, s);
        return launch_small_f64(p, static_cast<const double*>(x_dev), ldx, static_cast<double*>(y_dev),
                                ldy, batch, s);
    }
    const float* x = static_cast<const float*>(x_dev);
    float* y = static_cast<float*>(y_dev);
    if (n <= kSmallMax) {
        if (p->cauchy_mode != DCTPLUS_CAUCHY_SIMT && small_tc_available(p))
            return launch_small_tc(p, x, ldx, y, ldy, batch, s);
        return launch_small_simt_f32(p, x, ldx, y, ldy, batch, s);
    }
    return launch_large_f32(p, x, ldx, y, ldy, batch, s);
}

dctplus_status dctplus_execute_multi(const dctplus_plan_t* plans, int count, const float* x_dev, int64_t ldx,
                                     float* y_dev, int64_t ldy, int64_t batch, dctplus_stream_t stream) {
    if (!plans || count < 1 || batch < 0) return DCTPLUS_ERR_INVALID_ARG;
    for (int k = 0; k < count; ++k)
        if (!plans[k] || plans[k]->n != plans[0]->n || plans[k]->device != plans[0]->device)
            return DCTPLUS_ERR_INVALID_ARG;
    const int n = plans[0]->n;
    if (batch == 0) return DCTPLUS_OK;
    if (!x_dev || !y_dev || ldx < n || ldy < (int64_t)count * n) return DCTPLUS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(x_dev) | reinterpret_cast<uintptr_t>(y_dev)) & 3) return DCTPLUS_ERR_INVALID_ARG;
    {  // reject overlapping x / y ranges
        const uintptr_t xa = (uintptr_t)x_dev, ya = (uintptr_t)y_dev;
        const uintptr_t xe = xa + 4 * (size_t)((batch - 1) * ldx + n);
        const uintptr_t ye = ya + 4 * (size_t)((batch - 1) * ldy + (int64_t)count * n);
        if (xa < ye && ya < xe) return DCTPLUS_ERR_INVALID_ARG;
    }
    dctplus_status st = check_device(plans[0]->device);
    if (st != DCTPLUS_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    bool all_hier = n > kSmallMax && (n & (n - 1)) == 0, all_dense = all_hier;
    for (int k = 0; k < count; ++k) {
        all_hier = all_hier && plans[k]->cauchy_mode == DCTPLUS_CAUCHY_HIER && plans[k]->hier;
        all_dense = all_dense && plans[k]->cauchy_mode == DCTPLUS_CAUCHY_DENSE && plans[k]->d_whi;
        // a handle given twice would share its workspace between two of the group's slots
        for (int j = 0; j < k; ++j) all_hier = all_hier && plans[j] != plans[k];
    }
    const bool y_ok = (reinterpret_cast<uintptr_t>(y_dev) & 15) == 0 && (ldy & 3) == 0 && batch <= INT32_MAX;
    if (all_hier && y_ok) {
        // one DCT-II per group of up to kFarMaxPlans plans, every plan's far field and output after it
        for (int k0 = 0; k0 < count; k0 += kFarMaxPlans) {
            const int K = std::min(kFarMaxPlans, count - k0);
            float* ys[kFarMaxPlans];
            for (int k = 0; k < K; ++k) ys[k] = y_dev + (int64_t)(k0 + k) * n;
            if ((st = launch_hier_multi(plans + k0, K, x_dev, ldx, ys, ldy, batch, s)) != DCTPLUS_OK) return st;
        }
        return DCTPLUS_OK;
    }
    const int dev = plans[0]->device;
    if (all_dense && y_ok) {
        // one DCT-II, then each plan's dense product from the same s (up to four at a time)
        float* ws = static_cast<float*>(plan_workspace(plans[0], s, sizeof(float) * (size_t)batch * n));
        if (!ws) return DCTPLUS_ERR_CUDA;
        if ((st = launch_dct_fft(plans[0], x_dev, ldx, ws, n, batch, s)) != DCTPLUS_OK) return st;
        for (int k0 = 0; k0 < count && st == DCTPLUS_OK; k0 += kFarMaxPlans)
            st = run_forked(dev, s, std::min(kFarMaxPlans, count - k0), [&](int k, cudaStream_t sk) {
                const dctplus_plan_t p = plans[k0 + k];
                return launch_gemm_tc(ws, nullptr, n, p->d_whi, p->d_wlo, n, y_dev + (int64_t)(k0 + k) * n, ldy,
                                      (int)batch, n, n, sk, dev);
            });
        return st;
    }
    // plan by plan, up to four at a time (each on its own stream's workspace)
    for (int k0 = 0; k0 < count && st == DCTPLUS_OK; k0 += kFarMaxPlans)
        st = run_forked(dev, s, std::min(kFarMaxPlans, count - k0), [&](int k, cudaStream_t sk) {
            return dctplus_execute(plans[k0 + k], DCTPLUS_F32, x_dev, ldx, y_dev + (int64_t)(k0 + k) * n, ldy,
                                   batch, reinterpret_cast<dctplus_stream_t>(sk));
        });
    return st;
}

dctplus_status dctplus_execute_host(dctplus_plan_t p, dctplus_dtype dtype, const void* x_host,
                                    void* y_host, int64_t batch, dctplus_stream_t stream) {
    if (!p || batch < 0 || (batch > 0 && (!x_host || !y_host))) return DCTPLUS_ERR_INVALID_ARG;
    if (dtype != DCTPLUS_F32 && dtype != DCTPLUS_F64) return DCTPLUS_ERR_INVALID_ARG;
    if (batch == 0) return DCTPLUS_OK;
    dctplus_status st = check_device(p->device);
    if (st != DCTPLUS_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    size_t es = dtype == DCTPLUS_F32 ? 4 : 8;
    size_t bytes = es * (size_t)batch * p->n;
    size_t half = (bytes + 255) & ~size_t(255);
    if (p->stage_bytes < 2 * half) {
        if (p->d_stage) { cudaStreamSynchronize(s); cudaFree(p->d_stage); p->d_stage = nullptr; }
        DCTPLUS_CUDA_TRY(cudaMalloc(&p->d_stage, 2 * half));
        p->stage_bytes = 2 * half;
    }
    char* dx = static_cast<char*>(p->d_stage);
    char* dy = dx + half;
    DCTPLUS_CUDA_TRY(cudaMemcpyAsync(dx, x_host, bytes, cudaMemcpyHostToDevice, s));
    st = dctplus_execute(p, dtype, dx, p->n, dy, p->n, batch, stream);
    if (st != DCTPLUS_OK) return st;
    DCTPLUS_CUDA_TRY(cudaMemcpyAsync(y_host, dy, bytes, cudaMemcpyDeviceToHost, s));
    DCTPLUS_CUDA_TRY(cudaStreamSynchronize(s));
    return DCTPLUS_OK;
}

dctplus_status dctplus_group_create(dctplus_group_t* out, int count, const dctplus_plan_t* plans) {
    if (!out) return DCTPLUS_ERR_INVALID_ARG;
    *out = nullptr;
    if (count <= 0 || !plans) return DCTPLUS_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        if (!plans[i]) return DCTPLUS_ERR_INVALID_ARG;
        if (plans[i]->n > kSmallMax) return DCTPLUS_ERR_UNSUPPORTED;
        if (plans[i]->device != plans[0]->device) return DCTPLUS_ERR_INVALID_ARG;
    }
    dctplus_status st = check_device(plans[0]->device);
    if (st != DCTPLUS_OK) return st;
    dctplus_group_s* g = new (std::nothrow) dctplus_group_s();
    if (!g) return DCTPLUS_ERR_CUDA;
    g->device = plans[0]->device;
    g->plans.assign(plans, plans + count);
    st = group_upload_plans(g);
    if (st != DCTPLUS_OK) { dctplus_group_destroy(g); return st; }
    *out = g;
    return DCTPLUS_OK;
}

void dctplus_group_destroy(dctplus_group_t g) {
    if (!g) return;
    cudaDeviceSynchronize();
    if (g->d_plan_tables) cudaFree(g->d_plan_tables);
    if (g->d_seg) cudaFree(g->d_seg);
    if (g->d_tiles) cudaFree(g->d_tiles);
    if (g->d_stage) cudaFree(g->d_stage);
    for (cudaEvent_t e : g->pipe_events) cudaEventDestroy(e);
    if (g->pipe_compute) cudaStreamDestroy(g->pipe_compute);
    if (g->pipe_d2h) cudaStreamDestroy(g->pipe_d2h);
    delete g;
}

static dctplus_status check_segments(dctplus_group_t g, const int64_t* seg, int nseg,
                                     int64_t total_elems) {
    if (nseg < 0 || (nseg > 0 && !seg)) return DCTPLUS_ERR_INVALID_ARG;
    for (int s = 0; s < nseg; ++s) {
        int64_t pi = seg[3 * s], off = seg[3 * s + 1], rows = seg[3 * s + 2];
        if (pi < 0 || pi >= (int64_t)g->plans.size() || off < 0 || rows < 0 || (off & 3))
            return DCTPLUS_ERR_INVALID_ARG;
        if (rows > INT32_MAX / 2) return DCTPLUS_ERR_UNSUPPORTED;
        if (total_elems >= 0 && off + rows * g->plans[pi]->n > total_elems)
            return DCTPLUS_ERR_INVALID_ARG;
    }
    return DCTPLUS_OK;
}

dctplus_status dctplus_execute_group(dctplus_group_t g, const float* x_dev, float* y_dev,
                                     const int64_t* seg_host, int nseg, dctplus_stream_t stream) {
    if (!g) return DCTPLUS_ERR_INVALID_ARG;
    dctplus_status st = check_segments(g, seg_host, nseg, -1);
    if (st != DCTPLUS_OK) return st;
    if (nseg == 0) return DCTPLUS_OK;
    if (!x_dev || !y_dev || x_dev == y_dev) return DCTPLUS_ERR_INVALID_ARG;
    if ((st = check_device(g->device)) != DCTPLUS_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // segments of tensor-core-capable plans go to the tensor-core kernel (one
    // launch for all of them), the others to the CUDA-core kernel
    const bool tc_ok = aligned16(x_dev) && aligned16(y_dev);
    std::vector<TcSegHost> tc;
    std::vector<int64_t> simt;
    for (int i = 0; i < nseg; ++i) {
        int64_t pi = seg_host[3 * i], off = seg_host[3 * i + 1], rows = seg_host[3 * i + 2];
        dctplus_plan_t p = g->plans[pi];
        if (rows == 0) continue;
        if (tc_ok && small_tc_capable(p)) {
            tc.push_back({p, x_dev + off, y_dev + off, rows});
        } else {
            simt.push_back(pi);
            simt.push_back(off);
            simt.push_back(rows);
        }
    }
    if (!tc.empty() && (st = launch_tc_segments(tc, s, g->device)) != DCTPLUS_OK) return st;
    if (!simt.empty()) {
        if ((st = group_prepare(g, simt.data(), (int)simt.size() / 3, s)) != DCTPLUS_OK) return st;
        return launch_group_simt(g, x_dev, y_dev, s);
    }
    return DCTPLUS_OK;
}

dctplus_status dctplus_execute_group_host(dctplus_group_t g, const float* x_host, float* y_host,
                                          int64_t total_elems, const int64_t* seg_host, int nseg,
                                          dctplus_stream_t stream) {
    if (!g || total_elems < 0 || (total_elems > 0 && (!x_host || !y_host)))
        return DCTPLUS_ERR_INVALID_ARG;
    dctplus_status st = check_segments(g, seg_host, nseg, total_elems);
    if (st != DCTPLUS_OK) return st;
    if (total_elems == 0 || nseg == 0) return DCTPLUS_OK;
    if ((st = check_device(g->device)) != DCTPLUS_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    size_t bytes = sizeof(float) * (size_t)total_elems;
    size_t half = (bytes + 255) & ~size_t(255);
    if (g->stage_bytes < 2 * half) {
        if (g->d_stage) { cudaStreamSynchronize(s); cudaFree(g->d_stage); g->d_stage = nullptr; }
        DCTPLUS_CUDA_TRY(cudaMalloc(&g->d_stage, 2 * half));
        g->stage_bytes = 2 * half;
    }
    float* dx = static_cast<float*>(g->d_stage);
    float* dy = reinterpret_cast<float*>(static_cast<char*>(g->d_stage) + half);
    bool all_tc = true;
    for (int i = 0; i < nseg; ++i)
        if (seg_host[3 * i + 2] > 0 && !small_tc_capable(g->plans[seg_host[3 * i]])) all_tc = false;
    if (all_tc && total_elems >= kPipeMinElems)
        return group_host_pipelined(g, x_host, y_host, dx, dy, seg_host, nseg, s);
    DCTPLUS_CUDA_TRY(cudaMemcpyAsync(dx, x_host, bytes, cudaMemcpyHostToDevice, s));
    st = dctplus_execute_group(g, dx, dy, seg_host, nseg, stream);
    if (st != DCTPLUS_OK) return st;
    DCTPLUS_CUDA_TRY(cudaMemcpyAsync(y_host, dy, bytes, cudaMemcpyDeviceToHost, s));
    DCTPLUS_CUDA_TRY(cudaStreamSynchronize(s));
    return DCTPLUS_OK;
}

dctplus_status dctplus_sync_check(dctplus_stream_t stream) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DCTPLUS_CUDA_TRY(cudaStreamSynchronize(s));
    int dev = 0;
    DCTPLUS_CUDA_TRY(cudaGetDevice(&dev));
    unsigned* w = device_error_word(dev);
    if (!w) return DCTPLUS_ERR_CUDA;
    unsigned h = 0;
    DCTPLUS_CUDA_TRY(cudaMemcpy(&h, w, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (h) DCTPLUS_CUDA_TRY(cudaMemset(w, 0, sizeof(unsigned)));
    if (h & kErrTimeout) return DCTPLUS_ERR_TIMEOUT;
    if (h) return DCTPLUS_ERR_DEVICE_CHECK;
    return DCTPLUS_OK;
}

}  // extern "C"
