/*
 * fbcorr.h -- C ABI of the GB300 (sm_103a) filter-bank correlation library.
 *
 * The operation is the 3D filter-bank correlation that the paper's vision
 * case study (Sec. 6.2, "Computational Visual Neuroscience") identifies as the
 * bottleneck of its models and auto-tunes with run-time code generation
 * (Table "Performance of RTCG auto-tuning on 3D filter-bank convolutions"):
 * an H x W x D input stack correlated 'valid' against a bank of N filters of
 * fh x fw x D, giving an H' x W' x N output (H' = H-fh+1, W' = W-fw+1):
 *
 *     y[p][q][n] = epi( sum_{i<fh} sum_{j<fw} sum_{d<D} x[p+i][q+j][d] * w[n][i][j][d] )
 *
 * with an optional fused elementwise epilogue epi (a static non-linearity,
 * Sec. 6.2).  The backward pass gives the gradients of a scalar loss L with
 * respect to x and w from g = dL/dy.
 *
 * Conventions (all calls):
 *  - Tensors are FP32, row-major with the last index fastest, contiguous and
 *    16-byte aligned, in DEVICE memory owned by the caller:
 *      x [H][W][D], w [N][fh][fw][D], y / g [H'][W'][N], dx [H][W][D], dw like w.
 *  - Every call returns a status and never aborts or exits.  Argument and
 *    shape errors are detected before any work is enqueued.  A CUDA error is
 *    reported as FBCORR_ERR_CUDA; fbcorr_last_error() gives the detail
 *    (a thread-local message, valid until the next call on that thread).
 *  - forward / backward / forward_batched are stream-ordered, never
 *    synchronise the host, and allocate no memory: scratch space is the
 *    caller's workspace (size from the *_workspace_size queries).
 *  - The generated FP32 kernels (forward and dL/dx) are launched as
 *    programmatic dependents: each waits (griddepcontrol.wait) for the
 *    previous kernel of the stream to complete before touching memory, then
 *    lets the next kernel begin launching.  A kernel the caller launches after
 *    them with programmatic stream serialization must likewise wait
 *    (cudaGridDependencySynchronize) before it reads their outputs; kernels
 *    launched without that attribute see ordinary stream order.
 *  - Kernels are specialised per (fh, fw, D, tile) at plan time by run-time
 *    code generation (NVRTC, cached on disk) -- the paper's RTCG approach
 *    (Sec. 4, Sec. 6.2) -- with a prebuilt generic "default" kernel when
 *    code generation is unavailable.  There is no CPU fallback.
 */
#ifndef FBCORR_H
#define FBCORR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* fbcorr_stream_t;

typedef struct fbcorr_plan* fbcorr_plan_t;
typedef struct fbcorr_batch_plan* fbcorr_batch_plan_t;
typedef struct fbcorr_nn_plan* fbcorr_nn_plan_t;

typedef enum {
    FBCORR_OK = 0,
    FBCORR_ERR_INVALID_ARG = 1,  /* null pointer, bad enum, bad count          */
    FBCORR_ERR_SHAPE = 2,        /* non-positive dim, fh > H, depth mismatch,  */
                                 /* index arithmetic that would overflow int32 */
    FBCORR_ERR_UNSUPPORTED = 3,  /* valid request the library cannot run       */
    FBCORR_ERR_ALIGNMENT = 4,    /* a tensor pointer is not 16-byte aligned    */
    FBCORR_ERR_WORKSPACE = 5,    /* workspace missing or smaller than required */
    FBCORR_ERR_CUDA = 6,         /* a CUDA runtime call or a launch failed     */
    FBCORR_ERR_NVRTC = 7,        /* run-time compilation of a variant failed   */
    FBCORR_ERR_OOM = 8,          /* host or plan-time device allocation failed */
    FBCORR_ERR_TIMEOUT = 9,      /* a kernel gave up a bounded wait            */
    FBCORR_ERR_INTERNAL = 10
} fbcorr_status_t;

/* Arithmetic of the forward pass; tensors are FP32 in every mode.
 *  F32    : FP32 products, FP32 accumulation (CUDA cores).
 *  BF16   : x and w rounded to BF16 (round-to-nearest-even), BF16 x BF16
 *           products with FP32 accumulation on the tcgen05 tensor cores.
 *  BF16X3 : "split BF16": v = hi + lo with hi = bf16(v), lo = bf16(v - hi);
 *           y accumulates hi*hi + hi*lo + lo*hi in FP32 on the tensor cores,
 *           recovering close to FP32 accuracy.
 * The backward pass always runs in F32. */
typedef enum { FBCORR_F32 = 0, FBCORR_BF16 = 1, FBCORR_BF16X3 = 2 } fbcorr_dtype_t;

typedef enum { FBCORR_EPI_NONE = 0, FBCORR_EPI_CLAMP = 1, FBCORR_EPI_SNIPPET = 2 } fbcorr_epilogue_kind_t;

/* Fused epilogue applied to the FP32 accumulator before the store.
 * CLAMP: y = fminf(fmaxf(acc, lo), hi), lo <= hi.  Its gradient passes g only
 * where lo < y < hi strictly.
 * SNIPPET: a user expression compiled into the kernels (fbcorr_plan_create_snippet);
 * lo and hi are then two free parameters of the expression. */
typedef struct {
    int kind;   /* fbcorr_epilogue_kind_t */
    float lo, hi;
} fbcorr_epilogue_t;

/* ---- single-image plans ------------------------------------------------- */

/* Validate the shapes, pick (and on first use compile) the kernel variants for
 * the current CUDA device, and return a plan.  in_shape = {H, W, D},
 * filt_shape = {N, fh, fw, D}.  The chosen variant comes from, in order:
 * FBCORR_VARIANT, the on-disk tuning cache, a measurement run when
 * FBCORR_AUTOTUNE=1 (or force), and otherwise a built-in heuristic.
 * The plan owns its compiled modules and device bookkeeping, released by
 * fbcorr_plan_destroy. */
fbcorr_status_t fbcorr_plan_create(fbcorr_plan_t* out, const int64_t in_shape[3],
                                   const int64_t filt_shape[4], fbcorr_dtype_t dtype,
                                   fbcorr_epilogue_t epilogue);
/* Release what the plan owns (modules, streams, events, pinned status word,
 * tensor-core descriptors).  NULL is accepted and does nothing.  The caller
 * makes sure no work the plan enqueued is still running (synchronise its
 * streams first); caller-owned tensors and workspaces are not touched. */
fbcorr_status_t fbcorr_plan_destroy(fbcorr_plan_t plan);

/* A plan whose epilogue is a user C expression compiled into the forward
 * kernels at plan time: the run-time generated element-wise operation of the
 * paper (Sec. 5.2, the ElementwiseKernel of Fig. 4) fused into the store of the
 * correlation.  `expr` is an expression of float y (the FP32 accumulator of
 * one output), int n (its filter index) and float lo, hi (epilogue.lo / .hi),
 * evaluating to the float that is stored, e.g. "y > 0.f ? y : lo * y" or
 * "tanhf(y)".  CUDA device math functions may be used; ';', braces, '#',
 * quotes and backslashes may not (FBCORR_ERR_INVALID_ARG), and at most 1024
 * characters.  epilogue.kind must be FBCORR_EPI_SNIPPET.  A snippet that does
 * not compile gives FBCORR_ERR_NVRTC with the compiler log in
 * fbcorr_last_error().  Forward only: fbcorr_backward on such a plan returns
 * FBCORR_ERR_UNSUPPORTED (the expression has no known derivative).  Every
 * forward variant is generated (there is no prebuilt fallback for it). */
fbcorr_status_t fbcorr_plan_create_snippet(fbcorr_plan_t* out, const int64_t in_shape[3],
                                           const int64_t filt_shape[4], fbcorr_dtype_t dtype,
                                           fbcorr_epilogue_t epilogue, const char* expr);

/* out = {H', W', N}. */
fbcorr_status_t fbcorr_plan_out_shape(fbcorr_plan_t plan, int64_t out[3]);

/* Bytes of device workspace that forward and backward need (either pointer
 * may be NULL).  Zero means the call accepts ws = NULL. */
fbcorr_status_t fbcorr_plan_workspace_size(fbcorr_plan_t plan, size_t* fwd_bytes,
                                           size_t* bwd_bytes);

/* y = epi(corr(x, w)).  x, w, y: device pointers as above; ws: device
 * workspace of at least the forward size (NULL allowed when it is zero).
 * y must not alias x, w or ws. */
fbcorr_status_t fbcorr_forward(fbcorr_plan_t plan, const float* x, const float* w, float* y,
                               void* ws, size_t ws_bytes, fbcorr_stream_t stream);

/* The forward from HOST buffers, with the host<->device transfers overlapped
 * (end-to-end use: inputs and result in host memory).  x_host [H][W][D],
 * w_host [N][fh][fw][D] and y_host [H'][W'][N] are host pointers; page-locked
 * memory (cudaHostAlloc / cudaHostRegister) lets the copies run asynchronously,
 * pageable memory works but serialises them.  The output rows are split into
 * `bands` bands of a multiple of 4 rows (0: automatic, 8): band b's new input
 * rows are copied in on an internal stream, the band is correlated on `stream`
 * by a plan of the band's shape (tuned when this plan is tuned), and its output
 * rows are copied back on a second internal stream while the next band runs.
 * Stream-ordered: returns once everything is enqueued; y_host is complete when
 * `stream` reaches the point of the call.  The first call (and a call with a
 * different band count) allocates the plan-owned device copies of x, w and y,
 * the band plans and their workspace; later calls allocate nothing.  Not
 * capturable (internal streams).  Errors as fbcorr_forward; a bounded-wait
 * timeout of a band kernel is reported by fbcorr_plan_device_status. */
fbcorr_status_t fbcorr_forward_host(fbcorr_plan_t plan, const float* x_host, const float* w_host,
                                    float* y_host, int bands, fbcorr_stream_t stream);

/* Gradients of L from g = dL/dy (shape of y):
 *   dx[p][q][d]    = sum_{n,i,j} g~[p-i][q-j][n] * w[n][i][j][d]   (zero outside the output)
 *   dw[n][i][j][d] = sum_{p,q}   g~[p][q][n]     * x[p+i][q+j][d]
 * with g~ = g, or g masked to lo < y < hi when the plan's epilogue is CLAMP
 * (then y_or_null must be the forward output; otherwise it is ignored).
 * Either dx_or_null or dw_or_null may be NULL to skip that gradient.  Both
 * are deterministic run to run: the dw reduction sums fixed chunks in a fixed
 * order (no atomics), and a dL/dx tile that splits the gradient channels over
 * lanes combines their partial sums by a fixed shuffle tree.  Always F32. */
fbcorr_status_t fbcorr_backward(fbcorr_plan_t plan, const float* x, const float* w,
                                const float* g, const float* y_or_null, float* dx_or_null,
                                float* dw_or_null, void* ws, size_t ws_bytes,
                                fbcorr_stream_t stream);

/* Measure the candidate variants for this plan's shape on `stream` (CUDA
 * events, the paper's coarse grid search of Sec. 6.2), keep the fastest, and
 * record it in the tuning cache.  Synchronises the stream; not capturable. */
fbcorr_status_t fbcorr_autotune(fbcorr_plan_t plan, fbcorr_stream_t stream);

/* Force the forward variant: "default" (the prebuilt generic kernel),
 * "heuristic", "tuned", or an explicit spec as printed by fbcorr_plan_info. */
fbcorr_status_t fbcorr_plan_set_variant(fbcorr_plan_t plan, const char* spec);

/* The forward variants fbcorr_autotune would time for this plan, one spec per
 * line (each accepted by fbcorr_plan_set_variant), NUL-terminated into buf;
 * FBCORR_ERR_INVALID_ARG when cap is too small.  No GPU work. */
fbcorr_status_t fbcorr_plan_candidates(fbcorr_plan_t plan, char* buf, size_t cap);

/* A one-line JSON description of the plan and its chosen variants, written
 * into buf (NUL-terminated, truncated to cap bytes). */
fbcorr_status_t fbcorr_plan_info(fbcorr_plan_t plan, char* buf, size_t cap);

/* FBCORR_OK, or FBCORR_ERR_TIMEOUT once a kernel of this plan has given up a
 * bounded wait (read from host-mapped memory; no synchronisation).  Clears
 * the flag when `clear` is non-zero. */
fbcorr_status_t fbcorr_plan_device_status(fbcorr_plan_t plan, int clear);

/* Timing service (the paper's auto-tuning relies on the runtime's timers,
 * Sec. 4.1 and 5): when capacity > 0, every later forward call of this plan records a
 * pair of CUDA events on its stream around its main kernel (the correlation
 * kernel itself, not the BF16 split pre-pass), for up to `capacity` calls.
 * capacity = 0 switches recording off. */
fbcorr_status_t fbcorr_plan_profile(fbcorr_plan_t plan, int capacity);

/* Milliseconds of each recorded main-kernel launch, oldest first, into ms
 * (up to cap values); *n receives the count.  Waits for the recorded events,
 * then clears the record. */
fbcorr_status_t fbcorr_plan_profile_read(fbcorr_plan_t plan, float* ms, int cap, int* n);

/* Forward without any device allocation.  The paper has no counterpart: this
 * is for callers that cannot allocate device memory when they run the
 * correlation (no cudaMalloc after start-up in a real-time loop, a plugin host
 * whose allocator belongs to another runtime, a process that budgets all
 * device memory at initialisation).  It runs the same kernels as
 * fbcorr_forward, but the scratch that tensor-core plans need (the BF16 copies
 * of x and w) lives in one 48 MiB array built into the library, which every
 * GPU that loads the library keeps until the process exits.  Plans whose
 * forward workspace (fbcorr_plan_workspace_size) exceeds 48 MiB are rejected
 * with FBCORR_ERR_WORKSPACE; FP32 plans need no scratch.  The first call on a
 * device looks up the array's device address, so make that first call before
 * any stream capture; the address is kept for the life of the process, so do
 * not call this entry point after cudaDeviceReset.  The plan's device must be
 * the current device (else FBCORR_ERR_INVALID_ARG).  All calls on a device share the one array: calls whose
 * GPU work may overlap (different streams, or different threads without
 * ordering) race on it; order them on one stream.  The array keeps the last
 * call's contents; every call rewrites all the scratch it reads first.
 * Calls no cudaMalloc, cudaFree or other allocating routine. */
fbcorr_status_t fbcorr_forward_noalloc(fbcorr_plan_t plan, const float* x, const float* w,
                                       float* y, fbcorr_stream_t stream);

/* ---- batches of uneven images ------------------------------------------- */

/* A plan for n independent problems, image k with in_shapes[k] = {H, W, D}
 * and its own bank filt_shapes[k] = {N, fh, fw, D}, all run by ONE persistent
 * kernel launch (replayed from a CUDA graph) over a largest-first tile list. */
fbcorr_status_t fbcorr_batch_plan_create(fbcorr_batch_plan_t* out, int n,
                                         const int64_t (*in_shapes)[3],
                                         const int64_t (*filt_shapes)[4], fbcorr_dtype_t dtype,
                                         fbcorr_epilogue_t epilogue);
/* Release the batch plan's graph, work list and counters (NULL: no-op); its
 * launches must have finished. */
fbcorr_status_t fbcorr_batch_plan_destroy(fbcorr_batch_plan_t plan);
/* Device workspace fbcorr_forward_batched needs: currently always 0 (the plan
 * owns its work list and counter). */
fbcorr_status_t fbcorr_batch_plan_workspace_size(fbcorr_batch_plan_t plan, size_t* bytes);
/* A JSON description of the plan (images, work items, grid, residency,
 * variants and their tiles) into buf (NUL-terminated, cap bytes). */
fbcorr_status_t fbcorr_batch_plan_info(fbcorr_batch_plan_t plan, char* buf, size_t cap);

/* x[k], w[k], y[k]: HOST arrays of n DEVICE pointers (image k's tensors). */
fbcorr_status_t fbcorr_forward_batched(fbcorr_batch_plan_t plan, const float* const* x,
                                       const float* const* w, float* const* y, void* ws,
                                       size_t ws_bytes, fbcorr_stream_t stream);

/* ---- exact nearest-neighbour search -------------------------------------- */

/* The paper's second case study (Sec. 6.4, Table "NN-speedup"): for each of
 * n_targets vectors, its nearest neighbour in Euclidean distance among
 * n_neighbors vectors of the same dimension, by exhaustive comparison.
 * targets [n_targets][dim], neighbors [n_neighbors][dim]: FP32, row-major, DEVICE
 * memory, 16-byte aligned.  Results: idx_out[i] (int64, device) = the index of
 * the nearest neighbour, dist_out[i] (FP32, device) = its squared distance
 * sum_k (t_k - n_k)^2 computed exactly in FP32.
 * Method: every (target, neighbour) pair is screened on the tensor cores by
 * d' = |n|^2 - 2 t.n (dtype BF16X3: split-BF16 products, error about 2^-16
 * sum_k |t_k||n_k|; BF16: plain, about 2^-8), and the two best candidates of
 * every part of the screening are kept.  A bound E on the screening error of the
 * target's keys (from |t|, the largest |n| and the arithmetic of each step)
 * gives the window of keys within 2E of the smallest one, which holds the true
 * nearest neighbour; every candidate in it is re-ranked by its exact FP32
 * distance.  Where a part may hold more candidates in the window than it kept,
 * the target's exact FP32 distance to every neighbour of that part is taken too
 * (to every neighbour when more than 8 of its parts are incomplete).  With 32
 * or more neighbour tiles of 256, the first 1/16 of them are screened first
 * (FBCORR_NN_PRESCREEN=k: 1/k, 0: none) and the window at a target's best key
 * there bounds the window of the full screening from above, so keys at or
 * above it are not kept; this changes no result.  So the
 * result is always the argmin of the exact FP32 distance over all neighbours
 * (ties: the lowest index): the exact nearest neighbour up to FP32 rounding of
 * the distances.  dim <= 64, n_targets and n_neighbors < 2^31.  The plan
 * compiles its kernel (NVRTC) at creation; the search allocates nothing, performs
 * no host synchronisation and is stream-ordered. */
fbcorr_status_t fbcorr_nn_plan_create(fbcorr_nn_plan_t* out, int64_t n_targets, int64_t n_neighbors,
                                      int64_t dim, fbcorr_dtype_t dtype);
/* Release the plan (NULL: no-op); its searches must have finished. */
fbcorr_status_t fbcorr_nn_plan_destroy(fbcorr_nn_plan_t plan);
/* Device workspace the search needs (BF16 copies of both sets, norms, candidates). */
fbcorr_status_t fbcorr_nn_workspace_size(fbcorr_nn_plan_t plan, size_t* bytes);
/* Run the search on `stream`: targets, neighbors, idx_out, dist_out and ws are
 * DEVICE pointers (NULL: FBCORR_ERR_INVALID_ARG), 16-byte aligned
 * (FBCORR_ERR_ALIGNMENT otherwise); ws must hold fbcorr_nn_workspace_size bytes
 * (FBCORR_ERR_WORKSPACE otherwise).  All checks happen before any launch. */
fbcorr_status_t fbcorr_nn_search(fbcorr_nn_plan_t plan, const float* targets, const float* neighbors,
                                 int64_t* idx_out, float* dist_out, void* ws, size_t ws_bytes,
                                 fbcorr_stream_t stream);
/* As fbcorr_plan_device_status, for the nearest-neighbour kernel. */
fbcorr_status_t fbcorr_nn_plan_device_status(fbcorr_nn_plan_t plan, int clear);
/* How many targets of the plan's last search were re-scanned exactly (their
 * window could not be certified from the kept candidates alone) into *count;
 * 0 before the first search.  Waits for the last search's stream and reads its
 * workspace, which must still hold that search's counters (diagnostics, not for
 * a hot loop). */
fbcorr_status_t fbcorr_nn_last_fallbacks(fbcorr_nn_plan_t plan, int64_t* count);
/* Offline check (no GPU): generate and compile the screening kernel for dim. */
fbcorr_status_t fbcorr_nn_rtcg_check(int64_t dim, fbcorr_dtype_t dtype, char* log, size_t cap);

/* ---- diagnostics -------------------------------------------------------- */

/* The enumerator's name, e.g. "FBCORR_ERR_SHAPE" (a static string). */
const char* fbcorr_status_string(fbcorr_status_t status);
/* Detail of the last failing call on this thread (thread-local; every other
 * entry point clears it when it starts, so read it before the next call). */
const char* fbcorr_last_error(void);
/* Library version string, e.g. "fbcorr 0.1 sm_103a". */
const char* fbcorr_version(void);

/* The FP32 multiply-add rate the current device sustains, the measured
 * counterpart of the nominal FP32 peak (SMs x 128 lanes x 2 FLOP x clock) that
 * the FP32 kernels are rated against; the paper has no counterpart.  Runs 8
 * independent multiply-add chains per thread in registers on 2048 threads per
 * SM, `iters` x 128 multiply-adds per thread per launch, packed = 0 with scalar
 * FMAs or 1 with packed pairs (fma.rn.f32x2); one warm-up and three timed
 * launches on an internal stream.  *tflops = 2 x multiply-adds / best launch
 * time; *best_ms (may be NULL) = that time.  Allocates and frees one small
 * device buffer and synchronises with its own stream: a diagnostic, not for
 * use inside a capture.  iters in [1, 2^24], else FBCORR_ERR_INVALID_ARG. */
fbcorr_status_t fbcorr_fp32_fma_probe(int packed, int iters, double* tflops, double* best_ms);

/* Generate and compile (NVRTC, sm_103a) -- without loading or running -- the
 * forward, dL/dx and dL/dw kernels that an FP32 plan of this shape would use,
 * with the forward tile `spec` ("heuristic" or a "direct:..." spec; a chunked
 * K-split spec -- ks with cc > 0 -- is a dL/dx tile and replaces the dL/dx
 * heuristic instead, FBCORR_ERR_UNSUPPORTED where the shape's dL/dx cannot take
 * it: a clamp epilogue, or a depth or filter count not a multiple of 4); or, for a
 * "tcgen05:na=..,nb=..,nt=..,bt=..,ew=..,fz=.." spec, the tensor-core kernel
 * that spec generates for this depth and filter width, in both BF16 and split
 * BF16 form.  Needs no GPU.  On failure the NVRTC log (or the reason the spec
 * does not fit) is written into log (NUL-terminated, cap bytes). */
fbcorr_status_t fbcorr_rtcg_check(const int64_t in_shape[3], const int64_t filt_shape[4],
                                  fbcorr_epilogue_t epilogue, const char* spec, char* log,
                                  size_t cap);

/* Offline check of a snippet epilogue (no GPU): generate and compile the
 * forward kernel that fbcorr_plan_create_snippet would build for this shape and
 * dtype (the heuristic FP32 tile, or the default tcgen05 configuration).
 * Status and log as fbcorr_rtcg_check. */
fbcorr_status_t fbcorr_snippet_check(const int64_t in_shape[3], const int64_t filt_shape[4],
                                     fbcorr_dtype_t dtype, const char* expr, char* log, size_t cap);

/* The same offline check for a batch plan: generate and compile (without
 * loading) the single persistent kernel that fbcorr_batch_plan_create would
 * build for these n images.  Needs no GPU. */
fbcorr_status_t fbcorr_batch_rtcg_check(int n, const int64_t (*in_shapes)[3],
                                        const int64_t (*filt_shapes)[4], fbcorr_epilogue_t epilogue,
                                        char* log, size_t cap);

#ifdef __cplusplus
}
#endif

#endif /* FBCORR_H */
