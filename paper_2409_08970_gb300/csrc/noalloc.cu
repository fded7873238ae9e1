// dctplus_execute_noalloc: the large-n FP32 forward transform (the DCT-II
// kernel, then the CUDA-core Cauchy product) with its intermediate DCT-II
// coefficients held in a fixed scratch array compiled into this translation
// unit instead of a workspace allocated on demand. The paper has no
// counterpart; this is an execution variant of dctplus_execute.
//
// Who needs it: a caller that cannot let the library allocate device memory
// while it executes. cudaMalloc and cudaFree may synchronise the whole device,
// which stalls every other stream of a latency-bound serving loop, and some
// hosts hand all device memory to their own pool up front, so an allocation
// behind their back either fails or breaks their accounting. The ordinary
// dctplus_execute grows a per-(plan, stream) workspace on first use, which
// such callers cannot accept.
//
// Set-up: the first call on a device (in a given CUDA context), with that
// device current, looks up the device address of the scratch array
// (cudaGetSymbolAddress) and caches it with the context it belongs to. With
// lazy module loading (the CUDA default) that first lookup is also what loads
// this file's module, and the driver reserves the 16 MiB array at that moment;
// so the first call belongs in the caller's set-up, before any stream capture
// begins. A later call in another context (after cudaDeviceReset, say) looks
// the address up again instead of reusing one from a destroyed context.
//
// Nothing in the scratch has to start at zero: the DCT kernel writes every
// coefficient the Cauchy kernel then reads, within the same call.
//
// All calls on one device share the one scratch array. Two calls whose work
// overlaps in time (different streams, or different host threads, without an
// ordering between them) overwrite each other's coefficients; callers must
// order them, e.g. by issuing them on one stream.
#include <cuda.h>

#include <mutex>

#include "internal.cuh"

namespace dctplus {

constexpr int64_t kNoAllocMaxSamples = int64_t(1) << 22;  // batch * n limit (16 MiB of FP32)
constexpr int kNoAllocMaxN = kMaxN;
// the Cauchy product's grid.y (batch / 64 signal tiles) can never exceed its limit here
static_assert(kNoAllocMaxSamples / 128 / kCauchySimtSigTile <= 65535, "Cauchy grid limit");

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocMaxSamples];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

static CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &f, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(f);
    });
    return fn;
}

static std::mutex g_noalloc_mu;
static float* g_noalloc_ptr[64] = {};
static CUcontext g_noalloc_ctx[64] = {};

// Device address of the scratch array on `device` (which must be current), for
// the current context.
static dctplus_status noalloc_scratch(int device, float** out) {
    CtxGetCurrentFn get_ctx = ctx_get_current();
    CUcontext ctx = nullptr;
    if (!get_ctx || get_ctx(&ctx) != CUDA_SUCCESS || !ctx) return DCTPLUS_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[device] || g_noalloc_ctx[device] != ctx) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return DCTPLUS_ERR_CUDA;
        g_noalloc_ptr[device] = static_cast<float*>(ptr);
        g_noalloc_ctx[device] = ctx;
    }
    *out = g_noalloc_ptr[device];
    return DCTPLUS_OK;
}

}  // namespace dctplus

using namespace dctplus;

extern "C" dctplus_status dctplus_execute_noalloc(dctplus_plan_t p, const float* x_dev,
                                                  int64_t ldx, float* y_dev, int64_t ldy,
                                                  int64_t batch, dctplus_stream_t stream) {
    if (!p || batch < 0) return DCTPLUS_ERR_INVALID_ARG;
    if (batch == 0) return DCTPLUS_OK;
    const int n = p->n;
    if (!x_dev || !y_dev || ldx < n || ldy < n) return DCTPLUS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(x_dev) | reinterpret_cast<uintptr_t>(y_dev)) & 3)
        return DCTPLUS_ERR_INVALID_ARG;
    const uintptr_t xa = (uintptr_t)x_dev, ya = (uintptr_t)y_dev;
    const uintptr_t xe = xa + 4 * (size_t)((batch - 1) * ldx + n);
    const uintptr_t ye = ya + 4 * (size_t)((batch - 1) * ldy + n);
    if (xa < ye && ya < xe) return DCTPLUS_ERR_INVALID_ARG;
    // every precondition of both launches is checked here, before the DCT kernel is
    // queued to write the shared scratch: n a power of two in [128, 16384] (also a
    // multiple of the Cauchy product's K step) and, through the sample limit, at most
    // 2^22 / 128 / 64 signal tiles in the Cauchy grid (static_assert above)
    if (n <= kSmallMax || n > kNoAllocMaxN || (n & (n - 1)) || !p->d_twiddle)
        return DCTPLUS_ERR_UNSUPPORTED;
    if (batch > kNoAllocMaxSamples / n) return DCTPLUS_ERR_SCRATCH_LIMIT;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return DCTPLUS_ERR_NO_DEVICE;
    if (cur != p->device || cur < 0 || cur >= 64) return DCTPLUS_ERR_INVALID_ARG;
    float* s = nullptr;
    dctplus_status st = noalloc_scratch(cur, &s);
    if (st != DCTPLUS_OK) return st;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    st = launch_dct_fft(p, x_dev, ldx, s, n, batch, cs);
    if (st != DCTPLUS_OK) return st;
    return launch_cauchy_simt(p, s, n, y_dev, ldy, batch, cs);
}
