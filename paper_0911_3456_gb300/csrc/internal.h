// internal.h -- shared declarations of the libfbcorr host code (not installed).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <string>
#include <vector>

#include "fbcorr.h"

namespace fbc {

// ---- errors -----------------------------------------------------------------
fbcorr_status_t set_error(fbcorr_status_t s, const char* fmt, ...);
void clear_error();

#define FBC_CUDA(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return ::fbc::set_error(FBCORR_ERR_CUDA, "%s failed: %s (%s:%d)", #call,         \
                                    cudaGetErrorString(e_), __FILE__, __LINE__);            \
    } while (0)

#define FBC_TRY(expr)                                                                       \
    do {                                                                                    \
        fbcorr_status_t s_ = (expr);                                                        \
        if (s_ != FBCORR_OK) return s_;                                                     \
    } while (0)

// ---- environment knobs -------------------------------------------------------
std::string env_str(const char* name, const char* dflt = "");
bool log_enabled();
void logf(const char* fmt, ...);
bool fault_injected(const char* what);   // FBCORR_FAULT contains `what`
std::string cache_dir();                  // FBCORR_CACHE_DIR or ~/.cache/fbcorr

// ---- device facts ------------------------------------------------------------
struct DeviceInfo {
    int device = -1;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    size_t smem_optin = 0;
    int driver_version = 0;
    char name[256] = {0};
};
fbcorr_status_t device_info(DeviceInfo* out);

// ---- run-time code generation (NVRTC -> cubin -> driver module) --------------
struct Kernel {
    CUfunction fn = nullptr;
    int threads = 0;
    size_t smem = 0;
    std::string name;
    unsigned long long src_hash = 0;   // of the generated source and compile options (the cubin cache key)
};
std::string hex64(unsigned long long v);

// Compile `src` (with `name` as the extern "C" kernel) for sm_103a, using the
// on-disk cubin cache, load it into the current context and return a handle.
fbcorr_status_t rtcg_kernel(const std::string& src, const std::string& name, size_t smem,
                            int threads, Kernel* out);
// Compile many sources on host threads into the on-disk cubin cache.
fbcorr_status_t rtcg_precompile(const std::vector<std::string>& sources);
// Compile only (no GPU needed); returns the NVRTC log on failure.
fbcorr_status_t rtcg_compile_only(const std::string& src, std::string* log);
fbcorr_status_t launch(const Kernel& k, dim3 grid, void** args, cudaStream_t stream);
// Launch allowed to begin before the previous kernel in the stream has finished
// (programmatic dependent launch): the kernel must execute griddepcontrol.wait
// before it reads anything that kernel writes.  Falls back to launch() on a
// driver without cuLaunchKernelEx.
fbcorr_status_t launch_dependent(const Kernel& k, dim3 grid, void** args, cudaStream_t stream);
// A 3D FP32 tensor map for tiled bulk stores (128-byte swizzle, dims innermost
// first, strides in bytes of dims 1 and 2) written into the 128-byte `map`;
// false when the driver offers no tensor maps or rejects the arguments.
bool encode_f32_store_map(void* map, const float* base, const unsigned long long dims[3],
                          const unsigned long long strides[2], const unsigned box[3]);
// CUDA-graph kernel nodes for NVRTC kernels (driver API under the hood).
fbcorr_status_t graph_add_kernel(cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                                 const Kernel& k, dim3 grid, void** args, cudaGraphNode_t* out);
fbcorr_status_t graph_set_kernel(cudaGraphExec_t e, cudaGraphNode_t n, const Kernel& k, dim3 grid,
                                 void** args);
fbcorr_status_t kernel_occupancy(const Kernel& k, int* blocks_per_sm);
// registers per thread and local (spill and stack) bytes per thread of a loaded kernel
fbcorr_status_t kernel_resources(const Kernel& k, int* regs, int* local_bytes);
const char* rtcg_header_source();     // contents of rtcg_direct.cuh
const char* rtcg_tc_params_source();  // contents of tc_params.h
const char* rtcg_ptx_source();        // contents of rtcg_ptx.cuh
const char* rtcg_tc_source();         // contents of rtcg_tc.cuh
const char* rtcg_nn_params_source();  // contents of nn_params.h
const char* rtcg_nn_source();         // contents of rtcg_nn.cuh

// ---- variants ------------------------------------------------------------------
enum class VarKind { Default = 0, Direct = 1, Tensor = 2 };

struct DirectTile {
    int tr = 8, tf = 8, wr = 1, wf = 2;
    int cc = 0;   // input channels staged per chunk; 0 = the whole depth
    int pk = 0;   // 1: multiply-adds issued as packed pairs (fma.rn.f32x2), same bits
    int pf = 0;   // 1: the next channel chunk is loaded into registers while one is summed
    // K split (forward only): ks > 1 lanes share each output and split the depth,
    // combined by warp shuffles; a warp then covers 32 / ks columns and the CTA
    // wq warps side by side; sh = 1 takes the depth share from the high lane
    // bits (the lanes of a quarter warp then read the same filter values).
    // ks = 1: one column per lane (wq = 1, sh = 0).
    int ks = 1, wq = 1, sh = 0;
    // ks > 1 with cc > 0 (dL/dx without a clamp mask only): the chunked K-split
    // tile, cc channels per chunk through a cp.async ring of 2 stages, 3 with pf = 1
    // mb > 0: compiled with __launch_bounds__(threads, mb), so that mb CTAs fit in
    // an SM's registers (one stages while the others compute); 0: no bound
    int mb = 0;
    bool ks_chunked() const { return ks > 1 && cc > 0; }
    int chunk(int c) const { return (ks > 1 && cc == 0) ? c : ((cc > 0 && cc < c) ? cc : c); }
    int bh() const { return tr * wr; }
    int bn() const { return tf * wf; }
    int bw() const { return (32 / ks) * wq; }
    int threads() const { return 32 * wr * wf * wq; }
};
size_t direct_smem_bytes(const DirectTile& t, int fh, int fw, int c);
std::string direct_tile_spec(const DirectTile& t);
bool parse_direct_spec(const std::string& s, DirectTile* t);

// A direct-correlation problem in kernel terms (forward or dL/dx).
struct DirectProblem {
    int in_h, in_w, c;        // input extents and channels
    int out_h, out_w, nf;     // output extents and channels
    int fh, fw;
    int pad_y, pad_x;
    int flip, epi, mask;      // epi: 0 none, 1 clamp, 2 user snippet
    std::string snippet;      // the expression of epi = 2
};
// The generated definition of the snippet epilogue function (empty for no snippet).
std::string snippet_definition(const std::string& expr);
// 8 hex digits of a hash of the expression, for kernel names.
std::string snippet_tag(const std::string& expr);
std::string direct_kernel_source(const DirectProblem& pr, const DirectTile& t,
                                 const std::string& kname);
// threads > 0 restricts the candidates to one CTA size (the batched kernel).
// max_block bounds the per-thread accumulator block TR*TF (register pressure).
// dL/dx without a clamp mask, c % 4 == 0 and nf % 4 == 0: the chunked K-split tile applies.
bool ks_chunked_fits(const DirectProblem& pr);
std::vector<DirectTile> direct_candidates(const DirectProblem& pr, size_t smem_limit,
                                          int threads = 0, int max_block = 64);
// The specs the tuner times: the first topk tiles of a ranked list, each as
// written and with packed-pair FMAs (pk=1; FBCORR_TUNE_PK=0 keeps only the
// former), and, given the problem's depth, tiles of several channel chunks also
// with the register prefetch (pf=1; FBCORR_TUNE_PF=0 leaves it out).
std::vector<std::string> direct_tuning_specs(const std::vector<DirectTile>& ranked, int topk, int depth = 0);
DirectTile direct_heuristic(const DirectProblem& pr, size_t smem_limit, int sm_count,
                            int threads = 0, int max_block = 64);
// candidates ordered by the analytic model, best first
std::vector<DirectTile> direct_ranked(const DirectProblem& pr, size_t smem_limit, int sm_count,
                                      int threads = 0, int max_block = 64);

// Build / launch generated direct kernels and measure candidates (variants.cu).
std::string kname_for(const char* base, const DirectProblem& pr, const DirectTile& t);
size_t smem_limit(const DeviceInfo& dev);
fbcorr_status_t build_direct(const DirectProblem& pr, const DirectTile& t, Kernel* k);
dim3 direct_grid(const DirectProblem& pr, const DirectTile& t);
fbcorr_status_t run_direct(const Kernel& k, const DirectProblem& pr, const DirectTile& t,
                           const float* x, const float* m, const float* w, float* y, float lo,
                           float hi, cudaStream_t s);
fbcorr_status_t run_default(const DirectProblem& pr, const float* x, const float* m,
                            const float* w, float* y, float lo, float hi, cudaStream_t s);
fbcorr_status_t tune_direct_problem(const DeviceInfo& dev, const DirectProblem& pr, cudaStream_t s,
                                    int threads, int max_block, size_t smem_cap, int topk,
                                    bool include_default, const char* what, std::string* best_spec,
                                    float* best_ms_out);

// dL/dw partial-sum kernel: TN filters x fw taps per thread, NG filter groups of
// C threads per CTA, rows walked in blocks of QB columns staged in shared memory.
size_t dw_smem_bytes(int fw, int c, int tn, int ng, int qb, int pk);
// pk = 1: packed-pair FMAs in the double-buffered path (bit-identical); pk = 2:
// the same with each thread's chunk totals in shared memory (fewer registers).
// min_blocks > 0: CTAs per SM asked of the register allocator (launch bounds).
std::string dw_kernel_source(int fh, int fw, int c, int tn, int ng, int qb, int mask, int pk,
                             const std::string& kname, int min_blocks = 0);

// prebuilt (nvcc) kernels, launchers defined in default_kernels.cu
struct DirectArgsRT {
    const float* x;
    const float* m;
    const float* w;
    float* y;
    int in_h, in_w, c, out_h, out_w, nf, fh, fw, pad_y, pad_x, flip, epi, mask;
    float lo, hi;
};
cudaError_t launch_default_direct(const DirectArgsRT& a, cudaStream_t s);
cudaError_t launch_default_dw(const float* x, const float* g, const float* m, float* part,
                              int H, int W, int C, int Ho, int Wo, int N, int fh, int fw,
                              int chunks, int rows_per_chunk, int mask, float lo, float hi,
                              cudaStream_t s);
cudaError_t launch_dw_reduce(const float* part, float* dw, int S, long long E, cudaStream_t s);

// Fill p[0..n) with values in [-scale, scale) from an integer hash (timing runs only).
cudaError_t launch_fill_pattern(float* p, size_t n, float scale, unsigned seed, cudaStream_t s);

// ---- forward from host buffers (host_pipeline.cu) ----------------------------------
struct HostPipe;
void hostpipe_destroy(HostPipe* hp);
fbcorr_status_t hostpipe_device_status(HostPipe* hp, int clear);   // of the band plans

// ---- tensor-core path (tc_kernel.cu) -----------------------------------------------
struct TcPlan;   // opaque
fbcorr_status_t tc_plan_create(TcPlan** out, int H, int W, int D, int N, int fh, int fw,
                               int split, int epi, float lo, float hi, const std::string& snippet,
                               const DeviceInfo& dev);
void tc_plan_destroy(TcPlan* p);
size_t tc_workspace_bytes(const TcPlan* p);
// ev_start / ev_stop (may be null): recorded around the main GEMM kernel.
fbcorr_status_t tc_forward(TcPlan* p, const float* x, const float* w, float* y, void* ws,
                           int* err_word, cudaStream_t s, cudaEvent_t ev_start, cudaEvent_t ev_stop);
int tc_launches(const TcPlan* p);
std::string tc_describe(const TcPlan* p);           // JSON object
std::string tc_spec(const TcPlan* p);               // "tcgen05:na=..,nb=..,nt=.."
std::vector<std::string> tc_candidates(TcPlan* p);  // feasible specs, default first
fbcorr_status_t tc_set_spec(TcPlan* p, const std::string& spec);
// Compile the generated kernels of `specs` on host threads into the cubin cache.
fbcorr_status_t tc_precompile(TcPlan* p, const std::vector<std::string>& specs);
// Compile-only check of the generated kernel of `spec` (BF16 and split) for depth D, width fw.
fbcorr_status_t tc_rtcg_check(int D, int fw, const std::string& spec, std::string* log);
// Compile-only check of the generated kernel with a snippet epilogue (default configuration).
fbcorr_status_t tc_snippet_check(int D, int fw, int split, const std::string& snippet, std::string* log);

// ---- argument validation (api.cu) -------------------------------------------------------
fbcorr_status_t validate_shapes(const int64_t* in, const int64_t* fs, fbcorr_dtype_t dtype,
                                const fbcorr_epilogue_t& epi);

// ---- tune cache ----------------------------------------------------------------------
std::string tune_key(const DeviceInfo& dev, const std::string& what);
bool tune_lookup(const std::string& key, std::string* value);
void tune_store(const std::string& key, const std::string& value);

}  // namespace fbc

// ---- the plan object ------------------------------------------------------------------
struct fbcorr_plan {
    int64_t H = 0, W = 0, D = 0, N = 0, fh = 0, fw = 0, Ho = 0, Wo = 0;
    fbcorr_dtype_t dtype = FBCORR_F32;
    fbcorr_epilogue_t epi{0, 0.f, 0.f};
    fbc::DeviceInfo dev;

    // forward
    fbc::VarKind fwd_kind = fbc::VarKind::Direct;
    fbc::DirectTile fwd_tile;
    fbc::Kernel fwd_kernel;
    std::string fwd_source;        // "heuristic", "tuned", "cache", "env", "forced"
    fbc::TcPlan* tc = nullptr;
    std::string snippet;           // user epilogue expression (epi.kind == FBCORR_EPI_SNIPPET)

    // backward (F32 always)
    bool bwd_ready = false;
    fbc::VarKind dx_kind = fbc::VarKind::Direct;
    fbc::DirectTile dx_tile;
    fbc::Kernel dx_kernel;
    fbc::VarKind dw_kind = fbc::VarKind::Direct;
    fbc::Kernel dw_kernel;
    int dw_tn = 4, dw_ng = 1, dw_qb = 64, dw_nblocks = 1;
    int dw_pk = 2;                 // dL/dw FMA form: 0 scalar, 1 packed pairs, 2 packed pairs + shared totals
    int dw_mb = 0;                 // CTAs per SM in the dL/dw kernel's launch bounds (0: none)
    int dw_regs = 0;               // registers per thread of the built dL/dw kernel
    int dw_chunks = 1, dw_rows_per_chunk = 1;

    size_t ws_fwd = 0, ws_bwd = 0;

    // backward with both gradients: dL/dw on a side stream forked from and joined
    // back to the caller's stream (created with the backward kernels)
    cudaStream_t bwd_side = nullptr;
    cudaEvent_t bwd_fork = nullptr, bwd_join = nullptr;

    // bounded-wait failure flag in host-mapped memory
    int* err_host = nullptr;
    int* err_dev = nullptr;

    // timing service: events around the main forward kernel
    std::vector<cudaEvent_t> prof_start, prof_stop;
    int prof_count = 0;

    // fbcorr_forward_host: device buffers, band plans and streams (first call)
    fbc::HostPipe* hostpipe = nullptr;
};
