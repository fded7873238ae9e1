/*
 * dctplus.h — C ABI of the GB300 Fast DCT+ library.
 *
 * The transform: for the path graph Laplacian L~ = U diag(lambda) U^T and a
 * rank-one update L = L~ + rho v v^T (Def. 2.3) with eigenbasis X, a signal
 * x in R^n maps to its GFT coefficients y = X^T x. Theorem 3.1 (eq. fwd_map)
 * factors this as
 *     y = -diag(a) C(mu, lambda) diag(z) U^T x,
 * with U^T x the orthonormal DCT-II, z = U^T v, C_ij = 1 / (mu_i - lambda_j)
 * (Def. 2.1), mu the roots of the secular equation
 * 1 + rho sum_j z_j^2 / (lambda_j - mu) = 0 (Remark on the setup stage), and
 * a the column normalisation. Algorithm 1 gives the forward steps: DCT-II,
 * scale by z, Cauchy product, scale by a.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Sizes are in elements. Signals are rows: signal b occupies
 *   x[b * ldx + 0 .. b * ldx + n - 1]; outputs likewise with ldy.
 * - Output row order: coefficient i of a signal belongs to the i-th smallest
 *   eigenvalue of L. Eigenvector signs follow the rule <u_pi(i), x_i> > 0
 *   (pi pairs the i-th non-deflated root with the i-th non-deflated pole in
 *   ascending order; a deflated eigenvector u_j keeps its DCT sign). With
 *   rho = 0 the transform is exactly the orthonormal DCT-II.
 * - Ownership: the caller owns every buffer passed in. A plan owns its own
 *   device tables (a few n-vectors, plus at most O(n^2) floats for n <= 4096)
 *   and frees them in dctplus_destroy.
 * - Streams: execute calls are asynchronous on the given stream (0 = legacy
 *   default stream), never synchronise, and only read the plan, so one plan may
 *   be executed concurrently on several streams. Plans are immutable after
 *   creation.
 * - Errors: every call returns a dctplus_status and never throws. Argument
 *   errors are detected on the host before any launch. Device-side checks
 *   (index guards) write a device error word, read by dctplus_sync_check.
 * - Device: a plan lives on the device that was current at dctplus_plan
 *   (or opts->device); execute calls must be issued with that device current.
 */
#ifndef DCTPLUS_H
#define DCTPLUS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dctplus_plan_s* dctplus_plan_t;
typedef struct dctplus_group_s* dctplus_group_t;
typedef struct CUstream_st* dctplus_stream_t; /* same handle as cudaStream_t */

typedef enum {
    DCTPLUS_OK = 0,
    DCTPLUS_ERR_INVALID_ARG = 1,   /* bad size, pointer, stride or non-finite input */
    DCTPLUS_ERR_UNSUPPORTED = 2,   /* valid request the library does not implement */
    DCTPLUS_ERR_NOT_CONVERGED = 3, /* secular root iteration hit its cap */
    DCTPLUS_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    DCTPLUS_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    DCTPLUS_ERR_DEVICE_CHECK = 6,  /* a device-side guard recorded a violation */
    DCTPLUS_ERR_NO_DEVICE = 7,     /* no CUDA device is visible */
    DCTPLUS_ERR_SCRATCH_LIMIT = 8  /* batch * n above the fixed scratch of dctplus_execute_noalloc */
} dctplus_status;

typedef enum { DCTPLUS_F32 = 0, DCTPLUS_F64 = 1 } dctplus_dtype;

/* How the Cauchy product of Theorem 3.1 is evaluated for FP32 data with
 * n > 64 (n <= 64 always runs the fused small-n kernels). */
typedef enum {
    DCTPLUS_CAUCHY_AUTO = 0,  /* pick by n */
    DCTPLUS_CAUCHY_DENSE = 1, /* dense split-TF32 tensor-core product with the plan's
                                 W = diag(a) C(mu, lambda) diag(z) table; n % 128 == 0, n <= 4096 */
    DCTPLUS_CAUCHY_HIER = 2,  /* near-field band + Chebyshev far field, leaf level or a multipole
                                 tree (Theorem 3.2's fast-product family); n a power of two,
                                 256 <= n <= 16384 */
    DCTPLUS_CAUCHY_SIMT = 3,  /* CUDA-core product, W from a stored table (n <= 4096) or
                                 generated tile by tile in shared memory */
    DCTPLUS_CAUCHY_DENSE_GFT = 4, /* comparison baseline, not the factored method: one dense
                                    tensor-core product with the full X^T (n % 128 == 0,
                                    n <= 4096; X^T built in FP64 up to n = 1024, beyond that
                                    as W U^T on the tensor cores) */
    DCTPLUS_CAUCHY_NFST = 5       /* the paper's own route (Algorithm 1 steps 3-7): the zero
                                    pole's column kept explicit, a DST-I to the Chebyshev
                                    coefficients, and the sine series over sin(n theta) at the
                                    roots. FP64 inside for both dtypes. n a power of two with
                                    16 <= n <= 8192: O(n log n) per signal (FFT-based DCT-II
                                    and DST-I, the series by a nonuniform sine transform with
                                    a 16-point Kaiser-Bessel window on a twice-oversampled
                                    grid); other n <= 1024: direct sums, O(n^2). Loses
                                    accuracy like eps / |sin(n theta)| when a root sits next
                                    to a pole. Used by dctplus_execute only; groups, pruned
                                    and backward calls use their own kernels. */
} dctplus_cauchy_mode;

typedef struct {
    int cauchy_mode;      /* dctplus_cauchy_mode; 0 = auto */
    int max_secular_iter; /* cap on root iterations per root; 0 = 200 */
    int far_field;        /* hierarchical mode's far field: 0 = default (the tree from n = 8192),
                             1 = leaf level (one dense product with the leaf-to-leaf kernel
                             samples: (12 n / 64)^2 tensor-core multiply-adds per signal,
                             2 (12 n / 64)^2 floats of tables), 2 = multipole tree (M2M, M2L,
                             L2L over the angle boxes: O(n log n) work, O(n) tables) */
    int device;           /* CUDA device ordinal; -1 = current device */
    int64_t batch_hint;   /* expected batch, for the autotune cache lookup (0 = 4096) */
    const char* tune_cache; /* autotune cache file read when cauchy_mode is AUTO (see
                             dctplus_autotune); NULL = the DCTPLUS_TUNE_CACHE environment
                             variable, if set. With no matching entry AUTO takes its fixed
                             rule: dense for 128 <= n < 1024 (n % 128 == 0), hierarchical from
                             1024 (powers of two), the CUDA-core product otherwise. */
} dctplus_opts;

/* ------------------------------------------------------------------ plans */

/* Setup stage (Remark in Sec. 3): computes lambda (closed form), z = U^T v,
 * deflation of z_j ~ 0 (Sec. 4), the secular roots mu inside the Lemma 4.1
 * brackets (FP64, on the GPU) stored as nearest pole + offset, and the
 * normalisation a, then uploads the tables the execute kernels read.
 *   out   : receives the plan handle (owned by the library).
 *   n     : signal length, 2 <= n <= 16384.
 *   v_host: n doubles in host memory (copied; need not outlive the call).
 *   rho   : update weight; 0 gives the plain DCT-II. Must be finite.
 *   opts  : NULL for defaults.
 * Synchronous. Errors: INVALID_ARG (n out of range, NULL pointers, non-finite
 * v or rho), NOT_CONVERGED, CUDA, NO_DEVICE. On error *out is NULL. */
dctplus_status dctplus_plan(dctplus_plan_t* out, int n, const double* v_host, double rho,
                            const dctplus_opts* opts);

void dctplus_destroy(dctplus_plan_t plan);

/* Plan inspection (host copies of the FP64 setup quantities), for checking
 * the setup stage against Lemma 4.1 and the secular equation.
 *   eigenvalues: n doubles, ascending eigenvalues of L (output row order).
 *   z          : n doubles, z = U^T v.
 *   row_kind   : n ints, 1 = secular-root row, 0 = deflated row.
 *   row_pole   : n ints, the origin pole index of the row (deflated: its own j).
 *   row_tau    : n doubles, eigenvalue - lambda[row_pole].
 *   row_a      : n doubles, a_i of Theorem 3.1 (0 for deflated rows).
 * Any output pointer may be NULL. */
dctplus_status dctplus_plan_inspect(dctplus_plan_t plan, double* eigenvalues, double* z,
                                    int* row_kind, int* row_pole, double* row_tau,
                                    double* row_a);

/* Returns n, or -1 for a NULL plan. */
int dctplus_plan_size(dctplus_plan_t plan);

/* The Cauchy evaluation the plan uses for FP32 execute (a dctplus_cauchy_mode). */
int dctplus_plan_cauchy_mode(dctplus_plan_t plan);

/* The far-field form of a hierarchical plan (1 = leaf level, 2 = tree), 0 otherwise. */
int dctplus_plan_far_field(dctplus_plan_t plan);

/* --------------------------------------------------------------- forward */

/* Forward transform of a batch (Algorithm 1; Theorem 3.1 eq. fwd_map):
 * y_b = X^T x_b for b = 0..batch-1.
 *   dtype : DCTPLUS_F32 (split-TF32 tensor-core contractions, FP32 in/out) or
 *           DCTPLUS_F64 (FP64 CUDA-core path, n <= 1024). FP32 takes every
 *           n <= 4096 (lengths above 64 that are not powers of two run the
 *           DCT-II and the Cauchy product as CUDA-core products with the plan's
 *           tables) and powers of two up to 16384.
 *   x_dev, y_dev: device pointers aligned to the element size, rows of n
 *           elements with leading dimensions ldx, ldy >= n. The tensor-core
 *           kernels run when both bases are 16-byte aligned and ldx, ldy are
 *           multiples of 4; other layouts take the CUDA-core kernels.
 *           x and y must not overlap.
 *   batch : number of signals, >= 0 (0 is a no-op).
 * Scratch: for n >= 128 the plan keeps a device workspace per stream, grown
 * on the first call that needs more: batch n floats (the DCT coefficients);
 * the hierarchical mode adds batch (2 c + 32) floats (c = 12 n / 64 rounded up
 * to 128: the leaf moments and the leaf-local coefficients). A call that grows
 * it allocates, so make the first call at the largest batch before capturing
 * the stream into a CUDA graph.
 * Asynchronous on `stream`. Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
dctplus_status dctplus_execute(dctplus_plan_t plan, dctplus_dtype dtype, const void* x_dev,
                               int64_t ldx, void* y_dev, int64_t ldy, int64_t batch,
                               dctplus_stream_t stream);

/* Several updates of one graph over the same signals: y_k = X_k^T x for the
 * `count` plans (same n and device), FP32. Algorithm 1 step 1, the DCT-II
 * s = U^T x, does not depend on the update (v, rho), so plans in the
 * hierarchical mode share it (one DCT per group of up to 4 plans, each plan's
 * far-field inputs formed from the same s), and plans in the dense mode share
 * it before their own products; other sets (and a set listing one plan twice)
 * run plan by plan. Hierarchical plans that also share v (updates that differ
 * in rho only, with the same entries of z deflated) share the source side of
 * the far field too (Theorem 3.2's expansions depend on z and s alone): its
 * moments and far-field product are formed once per group and read by every
 * plan of it. Each plan keeps its dense rows (the rows whose eigenvalue lies
 * outside [0, 4]) in one of 16 slot pairs taken in turn at plan creation;
 * plans created 16 apart take the same pair and form their far fields apart.
 *   x_dev : batch rows of n floats, row stride ldx >= n.
 *   y_dev : batch rows, row stride ldy >= count * n; plan k's coefficients at
 *           columns k n .. k n + n - 1 (ascending eigenvalue). Must not
 *           overlap x.
 * Results equal those of dctplus_execute per plan. Asynchronous on `stream`:
 * the plans' own products are independent, so within each group of four the
 * plans after the first run on side streams that the library forks from
 * `stream` (an event after the work it holds) and joins back into it (the
 * call returns with `stream` waiting on all of them). The side streams (three
 * per device and caller stream, kept until the process exits, so a caller
 * should reuse its streams rather than make one per call) are created by the
 * first call on `stream`;
 * make that call before capturing `stream` into a CUDA graph (a call captured
 * before it runs the plans one after another on `stream`). Scratch: the
 * hierarchical and dense sets use the plans' workspaces of `stream` (plan 0's
 * holds the shared s); plan by plan, each plan uses its workspace of the
 * stream it runs on. Calls that share a plan and a stream must not overlap.
 * Errors: INVALID_ARG (null or mixed plans, count < 1, strides too small,
 * misaligned or overlapping buffers), the errors of dctplus_execute. */
dctplus_status dctplus_execute_multi(const dctplus_plan_t* plans, int count, const float* x_dev, int64_t ldx,
                                     float* y_dev, int64_t ldy, int64_t batch, dctplus_stream_t stream);

/* Same transform with HOST buffers: copies x to the device, transforms, copies
 * y back, all on `stream`, and returns after the stream has finished. Pinned
 * host memory gives full copy bandwidth. Uses a device staging buffer owned by
 * the plan (grown on demand), so calls on one plan must not overlap. */
dctplus_status dctplus_execute_host(dctplus_plan_t plan, dctplus_dtype dtype, const void* x_host,
                                    void* y_host, int64_t batch, dctplus_stream_t stream);

/* Same FP32 forward transform as dctplus_execute, for callers that cannot let
 * the library allocate device memory while it executes (an allocation may
 * synchronise the whole device and stall a latency-bound serving loop, and
 * some hosts hand all device memory to their own pool up front). The paper has
 * no counterpart: this is an execution variant only, with the same results as
 * dctplus_execute up to FP32 rounding.
 *   - Allocates nothing at execute time. The DCT-II coefficients go to a
 *     scratch array of 2^22 floats (16 MiB) compiled into the library's
 *     device image, which every GPU that loads it holds until exit.
 *   - Supports plans with n a power of two, 128 <= n <= 16384 (else
 *     UNSUPPORTED), and batch * n <= 2^22 (else SCRATCH_LIMIT); both are
 *     checked before any launch.
 *   - x_dev, y_dev: FP32 device rows as in dctplus_execute, 4-byte aligned,
 *     ldx, ldy >= n, not overlapping.
 *   - The first call on a device (with the plan's device current) looks up the
 *     scratch address. With lazy module loading (the CUDA default) that first
 *     call also loads the module holding the array, and the driver reserves
 *     the 16 MiB then: make the first call during set-up, before any stream
 *     capture begins. The address is cached per device and context; a call in
 *     a new context (e.g. after cudaDeviceReset) looks it up again.
 *   - The scratch need not start at zero; each call writes all it reads.
 *   - All calls on one device share the scratch: calls that may run at the
 *     same time (other streams or threads, unordered) race on it and must be
 *     ordered by the caller.
 * Asynchronous on `stream`. Errors: INVALID_ARG, UNSUPPORTED, SCRATCH_LIMIT,
 * NO_DEVICE, CUDA. */
dctplus_status dctplus_execute_noalloc(dctplus_plan_t plan, const float* x_dev, int64_t ldx,
                                       float* y_dev, int64_t ldy, int64_t batch,
                                       dctplus_stream_t stream);

/* ---------------------------------------------------- backward (FP32) */

/* Reverse-mode derivatives of the FP32 forward transform y_b = X^T x_b, given
 * upstream gradients g_b = dLoss/dy_b:
 *   gx_b     = X g_b = U W^T g_b: the inverse transform, undone step by step
 *              (Sec. 3: the transposed Cauchy product, then DCT-III);
 *   grad_rho = sum_b sum_i g_bi w_i (K (y_b * w))_i;
 *   grad_v   = rho X sum_b (y_b * (K^T (g_b * w)) + g_b * (K (y_b * w))),
 * with w = X^T v, K_ik = 1 / (mu_i - mu_k) (K_ii = 0): first-order
 * perturbation of the eigenvectors of L~ + rho v v^T (Def. 2.3). The
 * eigenvalues do not enter y, so no derivative of them is needed.
 *   gy_dev   : batch FP32 rows of n (ldg >= n).
 *   y_dev    : the forward output for the same signals (ldy >= n); needed only
 *              when grad_rho or grad_v is requested, else may be NULL.
 *   gx_dev   : NULL, or batch FP32 rows of n (ldgx >= n) receiving X g_b;
 *              must not overlap gy or y.
 *   grad_rho : NULL, or one device double (overwritten).
 *   grad_v   : NULL, or n device doubles (overwritten).
 * 2 <= n <= 16384 (every plan length); device pointers 4-byte aligned. The
 * first call for a plan builds its backward tables (W^T and K, 3 x 4 n^2 bytes
 * each, plus U for lengths without an FFT: 1.1 GB each at n = 16384;
 * allocates and synchronises, so make it before any stream capture); later
 * calls use the plan's per-stream workspace (4 batch n floats). Asynchronous
 * on `stream` otherwise. Errors: INVALID_ARG, NO_DEVICE, CUDA (also when the
 * tables do not fit). */
dctplus_status dctplus_backward(dctplus_plan_t plan, const float* gy_dev, int64_t ldg,
                                const float* y_dev, int64_t ldy, float* gx_dev, int64_t ldgx,
                                double* grad_rho, double* grad_v, int64_t batch,
                                dctplus_stream_t stream);

/* ------------------------------------------- progressive + pruned (FP32) */

/* Progressive multi-transform with output pruning (Theorem 3.4, Fig. 2): K
 * updates (v_k, rho_k) of the same path graph share one DCT-II per signal, and
 * each keeps only its first m_out coefficients, computed from the first c_p
 * DCT coefficients:
 *     y_k = W_k[0:m_out, 0:c_p] s[0:c_p],  s = DCT-II(x),
 *     W_k = -diag(a) C(mu, lambda) diag(z) of plan k (Theorem 3.1).
 * c_p = n gives the exact first m_out coefficients of every transform;
 * c_p < n is the truncation C^ of Theorem 3.4, whose error over all n
 * outputs is at most ||s_{c_p+1:n}|| + ||W_hl s_{1:c_p}||.
 *   plans  : nplans (1..64) plans, all with the same n and device (borrowed).
 *   x_dev  : batch FP32 rows of n, leading dimension ldx >= n.
 *   y_dev  : batch FP32 rows of nplans * m_out, leading dimension
 *            ldy >= nplans * m_out; row b holds y_0 | y_1 | ... (plan order).
 *   1 <= m_out <= c_p <= n. x and y must not overlap; 4-byte aligned.
 * n > 64 that is not a power of two (n <= 4096) uses CUDA-core products
 * throughout. The tensor-core contraction runs when n > 64 is a power of two,
 * nplans * m_out is a multiple of 128, c_p a multiple of 32, y 16-byte aligned
 * and ldy a multiple of 4; otherwise the CUDA-core one.
 * The first call for a given (plans, m_out, c_p) builds and caches the stacked
 * rows of the W_k on the device (allocates and copies synchronously, so make
 * it before any stream capture); dctplus_destroy of any of the plans drops
 * the cache entry. Scratch: the per-stream workspace of plans[0].
 * Asynchronous on `stream` otherwise. Errors: INVALID_ARG, UNSUPPORTED,
 * NO_DEVICE, CUDA. */
dctplus_status dctplus_execute_pruned(const dctplus_plan_t* plans, int nplans, const float* x_dev,
                                      int64_t ldx, float* y_dev, int64_t ldy, int64_t batch,
                                      int m_out, int c_p, dctplus_stream_t stream);

/* ------------------------------------------------- mixed-size batches (FP32) */

/* A group of plans with n <= 64 executed together in one persistent launch:
 * each segment of the input names one plan. `plans` are borrowed (must outlive
 * the group). All plans must live on the same device. */
dctplus_status dctplus_group_create(dctplus_group_t* out, int count, const dctplus_plan_t* plans);
void dctplus_group_destroy(dctplus_group_t group);

/* Segment descriptor: three int64 per segment, {plan index in the group,
 * element offset of the segment's first sample in x and y, number of rows}.
 * A segment's rows are contiguous (stride = n of its plan); offsets must be
 * multiples of 4 elements. */
#define DCTPLUS_SEG_WORDS 3

/* Forward transform of every segment in one launch (CUDA-graph capturable).
 *   x_dev, y_dev : FP32 device buffers holding all segments.
 *   seg_host     : nseg * 3 int64 in host memory (validated, then uploaded
 *                  into a group-owned device table; the upload is a
 *                  host-to-device copy on `stream` when the table changes).
 * Errors: INVALID_ARG, UNSUPPORTED (a plan with n > 64), CUDA. */
dctplus_status dctplus_execute_group(dctplus_group_t group, const float* x_dev, float* y_dev,
                                     const int64_t* seg_host, int nseg, dctplus_stream_t stream);

/* Host-buffer variant of dctplus_execute_group (copies inside, synchronous).
 * total_elems = size of x_host and y_host in floats. For large batches of
 * tensor-core segments (>= 2^22 samples) the work runs in chunks so that the
 * upload of one chunk, the kernel of the previous and the download of the one
 * before overlap (the group's own streams plus `stream`); only the address
 * ranges of the segments are copied back. Pinned host memory is needed for
 * the copies to overlap. */
dctplus_status dctplus_execute_group_host(dctplus_group_t group, const float* x_host,
                                          float* y_host, int64_t total_elems,
                                          const int64_t* seg_host, int nseg,
                                          dctplus_stream_t stream);

/* ------------------------------------------------------------ diagnostics */

/* Synchronises `stream`, then reads and clears the device error word.
 * Returns DCTPLUS_OK, DCTPLUS_ERR_DEVICE_CHECK or DCTPLUS_ERR_TIMEOUT. */
dctplus_status dctplus_sync_check(dctplus_stream_t stream);

/* ------------------------------------------------------------ autotuning */

/* Measures the FP32 Cauchy evaluations that apply at length n (dense tensor-core
 * product, hierarchical with the leaf-level far field, hierarchical with the
 * tree, CUDA-core product) for the update (v_host, rho) and `batch` signals
 * (generated on the device, a hash of the element index in [-1, 1)) on this
 * device: three warm-up calls, then five timed calls each (CUDA events on
 * `stream`). Every candidate's output on 16 sampled signals must agree with the
 * CUDA-core product's to 4e-6 normwise, else it is not chosen. Writes the
 * fastest correct choice to *cauchy_mode and *far_field, the per-call ms of each
 * candidate to candidate_ms[4] (dense, hierarchical leaf level, hierarchical
 * tree, CUDA cores; -1 where not applicable or not correct; may be NULL), and,
 * with cache_path non-NULL, records the choice there under (this device's name,
 * n, batch rounded up to a power of two), replacing an entry with that key.
 * A tuning call: it allocates (3 batch n floats) and synchronises; 64 < n <= 16384,
 * batch n <= 2^28. The paper has no counterpart. Errors: INVALID_ARG,
 * UNSUPPORTED (no candidate ran), NO_DEVICE, CUDA. */
dctplus_status dctplus_autotune(int n, const double* v_host, double rho, int64_t batch,
                                const char* cache_path, dctplus_stream_t stream, int* cauchy_mode,
                                int* far_field, double* candidate_ms);

/* Host-only access to an autotune cache file (no GPU needed). Lookup writes the
 * entry for (device_name, n, batch rounded up to a power of two) and returns OK,
 * or returns UNSUPPORTED when there is none (or the file is missing). Record
 * adds or replaces that entry (candidate_ms[4] may be NULL); the file is
 * rewritten through a temporary file and renamed. */
dctplus_status dctplus_tune_lookup(const char* cache_path, const char* device_name, int n,
                                   int64_t batch, int* cauchy_mode, int* far_field);
dctplus_status dctplus_tune_record(const char* cache_path, const char* device_name, int n,
                                   int64_t batch, int cauchy_mode, int far_field, double ms,
                                   const double* candidate_ms);

/* Number of kernels this library has launched in this process (all devices). */
int64_t dctplus_launch_count(void);

/* Kernel timing trace, a measurement aid with no counterpart in the paper.
 * dctplus_trace_begin records a start event on `stream`; until
 * dctplus_trace_end, every kernel an execute, pruned or backward call launches
 * on that stream is followed by an event. dctplus_trace_end synchronises the
 * stream and reports, for the first `cap` launches in order, the kernel's name
 * (a static string), its device time in ms (from the previous event, so a
 * launch's time includes any gap before it), and its algorithmic work: bytes
 * of global memory it must move (inputs read once, outputs written once) and
 * flops (tensor-core products counted as executed, the three products of a
 * split operand included). Any output array may be NULL. Returns the number of
 * launches traced, or -1 (no trace open on `stream`, or a CUDA error). One
 * trace at a time per process; begin fails with INVALID_ARG while one is open
 * or while `stream` is capturing, and launches issued during a capture are not
 * traced. Meant for profiling runs, not for the timed region of a benchmark. */
dctplus_status dctplus_trace_begin(dctplus_stream_t stream);
int dctplus_trace_end(dctplus_stream_t stream, const char** names, float* ms, double* bytes,
                      double* flops, int cap);

const char* dctplus_status_string(dctplus_status status);

#ifdef __cplusplus
}
#endif

#endif /* DCTPLUS_H */
