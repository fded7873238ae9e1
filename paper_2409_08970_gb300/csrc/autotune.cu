// Autotuner for the FP32 evaluation of the Cauchy product at large n (a
// measurement aid; the paper has no counterpart): which of the dense
// tensor-core product, the hierarchical product with the leaf-level or the
// tree far field, and the CUDA-core product is fastest for a length n and a
// batch size on this device. The choices go to a JSON cache file keyed by
// device name, n and batch bucket (the batch rounded up to a power of two);
// dctplus_plan with DCTPLUS_CAUCHY_AUTO reads it (plan.cu) and falls back to
// its fixed rule when no entry matches.
//
// Cache file: one entry per line inside "entries", flat objects of string and
// number values, e.g.
//   {"device": "NVIDIA GB300", "n": 1024, "batch_bucket": 4096, "cauchy_mode": 2,
//    "far_field": 1, "ms": 0.0612, "ms_dense": 0.0655, ...}
// Lines that do not parse are skipped (and dropped when the file is rewritten).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

namespace dctplus {

namespace {

constexpr int kCand = 4;  // dense, hierarchical leaf level, hierarchical tree, CUDA cores
const char* const kCandKey[kCand] = {"ms_dense", "ms_hier_leaf", "ms_hier_tree", "ms_simt"};
const int kCandMode[kCand] = {DCTPLUS_CAUCHY_DENSE, DCTPLUS_CAUCHY_HIER, DCTPLUS_CAUCHY_HIER, DCTPLUS_CAUCHY_SIMT};
const int kCandFar[kCand] = {0, 1, 2, 0};

struct TuneEntry {
    std::string device;
    int n = 0;
    int64_t bucket = 0;
    int mode = 0, far = 0;
    double ms = -1.0;
    double cand[kCand] = {-1.0, -1.0, -1.0, -1.0};
};

std::mutex g_tune_mu;

// value of "key": in a flat object line; false if absent
bool find_value(const std::string& line, const char* key, std::string* out) {
    const std::string k = std::string("\"") + key + "\"";
    size_t p = line.find(k);
    if (p == std::string::npos) return false;
    p = line.find(':', p + k.size());
    if (p == std::string::npos) return false;
    ++p;
    while (p < line.size() && (line[p] == ' ' || line[p] == '\t')) ++p;
    if (p >= line.size()) return false;
    if (line[p] == '"') {
        const size_t e = line.find('"', p + 1);
        if (e == std::string::npos) return false;
        *out = line.substr(p + 1, e - p - 1);
        return true;
    }
    size_t e = p;
    while (e < line.size() && line[e] != ',' && line[e] != '}') ++e;
    *out = line.substr(p, e - p);
    return !out->empty();
}

bool find_number(const std::string& line, const char* key, double* out) {
    std::string v;
    if (!find_value(line, key, &v)) return false;
    char* end = nullptr;
    const double d = std::strtod(v.c_str(), &end);
    if (end == v.c_str() || !std::isfinite(d)) return false;
    *out = d;
    return true;
}

bool parse_entry(const std::string& line, TuneEntry* e) {
    double n, b, m, f, ms;
    std::string dev;
    if (!find_value(line, "device", &dev) || !find_number(line, "n", &n) ||
        !find_number(line, "batch_bucket", &b) || !find_number(line, "cauchy_mode", &m) ||
        !find_number(line, "far_field", &f) || !find_number(line, "ms", &ms))
        return false;
    e->device = dev;
    e->n = (int)n;
    e->bucket = (int64_t)b;
    e->mode = (int)m;
    e->far = (int)f;
    e->ms = ms;
    for (int c = 0; c < kCand; ++c) {
        double v;
        e->cand[c] = find_number(line, kCandKey[c], &v) ? v : -1.0;
    }
    return e->n > 0 && e->bucket > 0 && e->mode >= 0 && e->mode <= DCTPLUS_CAUCHY_NFST && e->far >= 0 &&
           e->far <= 2;
}

std::vector<TuneEntry> read_cache(const char* path) {
    std::vector<TuneEntry> out;
    FILE* f = std::fopen(path, "r");
    if (!f) return out;
    std::string line;
    char buf[4096];
    while (std::fgets(buf, sizeof(buf), f)) {
        line = buf;
        if (line.find("\"device\"") == std::string::npos) continue;
        TuneEntry e;
        if (parse_entry(line, &e)) out.push_back(e);
    }
    std::fclose(f);
    return out;
}

bool write_cache(const char* path, const std::vector<TuneEntry>& entries) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return false;
    std::fprintf(f, "{\n  \"format\": \"dctplus autotune cache 1\",\n  \"entries\": [\n");
    for (size_t i = 0; i < entries.size(); ++i) {
        const TuneEntry& e = entries[i];
        std::string dev;  // device names carry no quotes or backslashes; drop any anyway
        for (char c : e.device)
            if (c != '"' && c != '\\' && c != '\n') dev += c;
        std::fprintf(f,
                     "    {\"device\": \"%s\", \"n\": %d, \"batch_bucket\": %lld, \"cauchy_mode\": %d, "
                     "\"far_field\": %d, \"ms\": %.6g",
                     dev.c_str(), e.n, (long long)e.bucket, e.mode, e.far, e.ms);
        for (int c = 0; c < kCand; ++c) std::fprintf(f, ", \"%s\": %.6g", kCandKey[c], e.cand[c]);
        std::fprintf(f, "}%s\n", i + 1 < entries.size() ? "," : "");
    }
    std::fprintf(f, "  ]\n}\n");
    const bool ok = std::fclose(f) == 0;
    return ok && std::rename(tmp.c_str(), path) == 0;
}

// deterministic pseudo-random signals in [-1, 1) (a 32-bit integer hash per element)
__global__ void k_tune_fill(float* x, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 2654435761u + 0x9E3779B9u;
        h ^= h >> 16;
        h *= 0x85EBCA6Bu;
        h ^= h >> 13;
        h *= 0xC2B2AE35u;
        h ^= h >> 16;
        x[i] = (float)(h >> 8) * (1.0f / 8388608.0f) - 1.0f;
    }
}

}  // namespace

int64_t tune_bucket(int64_t batch) {
    int64_t b = 1;
    while (b < batch && b < (int64_t(1) << 40)) b <<= 1;
    return b;
}

bool tune_lookup(const char* path, const char* device, int n, int64_t batch, int* mode, int* far) {
    if (!path || !*path || !device) return false;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int64_t b = tune_bucket(batch);
    for (const TuneEntry& e : read_cache(path)) {
        if (e.device == device && e.n == n && e.bucket == b) {
            *mode = e.mode;
            *far = e.far;
            return true;
        }
    }
    return false;
}

static dctplus_status tune_record(const char* path, const TuneEntry& ne) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::vector<TuneEntry> entries = read_cache(path);
    bool replaced = false;
    for (TuneEntry& e : entries) {
        if (e.device == ne.device && e.n == ne.n && e.bucket == ne.bucket) {
            e = ne;
            replaced = true;
        }
    }
    if (!replaced) entries.push_back(ne);
    return write_cache(path, entries) ? DCTPLUS_OK : DCTPLUS_ERR_INVALID_ARG;
}

}  // namespace dctplus

using namespace dctplus;

extern "C" {

dctplus_status dctplus_tune_lookup(const char* cache_path, const char* device_name, int n, int64_t batch,
                                   int* cauchy_mode, int* far_field) {
    if (!cache_path || !device_name || !cauchy_mode || !far_field || n < 2 || batch < 1)
        return DCTPLUS_ERR_INVALID_ARG;
    return tune_lookup(cache_path, device_name, n, batch, cauchy_mode, far_field) ? DCTPLUS_OK
                                                                                   : DCTPLUS_ERR_UNSUPPORTED;
}

dctplus_status dctplus_tune_record(const char* cache_path, const char* device_name, int n, int64_t batch,
                                   int cauchy_mode, int far_field, double ms, const double* candidate_ms) {
    if (!cache_path || !device_name || n < 2 || batch < 1 || cauchy_mode < 0 ||
        cauchy_mode > DCTPLUS_CAUCHY_NFST || far_field < 0 || far_field > 2 || !std::isfinite(ms))
        return DCTPLUS_ERR_INVALID_ARG;
    TuneEntry e;
    e.device = device_name;
    e.n = n;
    e.bucket = tune_bucket(batch);
    e.mode = cauchy_mode;
    e.far = far_field;
    e.ms = ms;
    for (int c = 0; c < kCand; ++c) e.cand[c] = candidate_ms ? candidate_ms[c] : -1.0;
    return tune_record(cache_path, e);
}

dctplus_status dctplus_autotune(int n, const double* v_host, double rho, int64_t batch, const char* cache_path,
                                dctplus_stream_t stream, int* cauchy_mode, int* far_field, double* candidate_ms) {
    if (!v_host || !cauchy_mode || !far_field || n <= kSmallMax || n > kMaxN || batch < 1 ||
        batch * n > (int64_t(1) << 28) || !std::isfinite(rho))
        return DCTPLUS_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DCTPLUS_ERR_NO_DEVICE;
    cudaDeviceProp prop;
    DCTPLUS_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t count = (size_t)batch * n;
    float *x = nullptr, *y = nullptr, *yref = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (x) cudaFree(x);
        if (y) cudaFree(y);
        if (yref) cudaFree(yref);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc(&x, count * 4) != cudaSuccess || cudaMalloc(&y, count * 4) != cudaSuccess ||
        cudaMalloc(&yref, count * 4) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        return DCTPLUS_ERR_CUDA;
    }
    k_tune_fill<<<1024, 256, 0, st>>>(x, (int64_t)count);
    count_launch();
    // the rows compared between candidates (the first, the last and some between)
    const int64_t nsample = std::min<int64_t>(batch, 16);
    std::vector<float> ref_rows((size_t)nsample * n), rows((size_t)nsample * n);
    auto sample = [&](const float* d, std::vector<float>& h) -> bool {
        for (int64_t i = 0; i < nsample; ++i) {
            const int64_t r = nsample > 1 ? i * (batch - 1) / (nsample - 1) : 0;
            if (cudaMemcpyAsync(h.data() + i * n, d + r * n, 4 * (size_t)n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
                return false;
        }
        return cudaStreamSynchronize(st) == cudaSuccess;
    };
    // the CUDA-core product first: the reference the others must agree with
    const int order[kCand] = {3, 0, 1, 2};
    double ms[kCand] = {-1.0, -1.0, -1.0, -1.0};
    int best = -1;
    bool have_ref = false;
    for (int oi = 0; oi < kCand; ++oi) {
        const int c = order[oi];
        dctplus_opts o{};
        o.cauchy_mode = kCandMode[c];
        o.far_field = kCandFar[c];
        o.device = -1;
        dctplus_plan_t p = nullptr;
        if (dctplus_plan(&p, n, v_host, rho, &o) != DCTPLUS_OK) continue;  // not applicable at this n
        dctplus_status s = DCTPLUS_OK;
        float* out = have_ref ? y : yref;
        for (int w = 0; w < 3 && s == DCTPLUS_OK; ++w) s = dctplus_execute(p, DCTPLUS_F32, x, n, out, n, batch, stream);
        if (s == DCTPLUS_OK && cudaStreamSynchronize(st) != cudaSuccess) s = DCTPLUS_ERR_CUDA;
        const int kReps = 5;
        if (s == DCTPLUS_OK) {
            cudaEventRecord(e0, st);
            for (int r = 0; r < kReps && s == DCTPLUS_OK; ++r)
                s = dctplus_execute(p, DCTPLUS_F32, x, n, out, n, batch, stream);
            cudaEventRecord(e1, st);
        }
        float t = 0.f;
        if (s == DCTPLUS_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) {
            bool correct = true;
            if (!have_ref) {
                correct = sample(out, ref_rows);
                have_ref = correct;
            } else if (!sample(out, rows)) {
                correct = false;
            } else {
                for (int64_t i = 0; i < nsample && correct; ++i) {
                    double num = 0.0, den = 0.0;
                    for (int j = 0; j < n; ++j) {
                        const double d = (double)rows[i * n + j] - ref_rows[i * n + j];
                        num += d * d;
                        den += (double)ref_rows[i * n + j] * ref_rows[i * n + j];
                    }
                    correct = num <= 16e-12 * den;  // normwise relative difference below 4e-6
                }
            }
            if (correct) {
                ms[c] = t / kReps;
                if (best < 0 || ms[c] < ms[best]) best = c;
            }
        }
        dctplus_destroy(p);
    }
    cleanup();
    if (candidate_ms)
        for (int c = 0; c < kCand; ++c) candidate_ms[c] = ms[c];
    if (best < 0) return DCTPLUS_ERR_UNSUPPORTED;
    *cauchy_mode = kCandMode[best];
    *far_field = kCandFar[best];
    if (cache_path && *cache_path)
        return dctplus_tune_record(cache_path, prop.name, n, batch, kCandMode[best], kCandFar[best], ms[best], ms);
    return DCTPLUS_OK;
}

}  // extern "C"
