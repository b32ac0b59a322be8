// nn.cu -- exact brute-force nearest-neighbour search (Sec. 6.4 of the paper):
// plans, the split / norm pre-pass, the run-time generated tensor-core screening
// kernel (rtcg_nn.cuh) and the exact re-ranking.
//
// Per call: (1) fbc_nn_split writes targets and neighbours as BF16 hi (and lo)
// chunk planes in tile-major order (one bulk copy brings a whole tile) and
// fbc_nn_norms the neighbour norms |n|^2 in FP32; (2) the generated kernel
// screens every (target, neighbour) pair on the tensor cores and keeps, per work
// item and target, the two smallest keys of d' = |n|^2 - 2 t.n; (3)
// fbc_nn_finalize takes the kRerank best distinct candidates of each target and
// re-ranks them by their exact FP32 squared distance sum_k (t_k - n_k)^2 (ties:
// lowest index).  The answer is the true nearest neighbour (up to FP32 distance
// rounding) whenever fewer than kRerank neighbours lie within the screening
// error of it; the distance reported is the exact FP32 one.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <new>
#include <sstream>

#include "internal.h"
#include "nn_params.h"

namespace fbc {
namespace {

constexpr int kRerank = 4;       // candidates re-ranked exactly per target
constexpr int kEW = 8;           // epilogue warps
constexpr size_t kSmemMax = 227 * 1024 - 1024;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// rows x dim FP32 -> tile-major BF16 planes [tiles][nc][tile_rows][8 values]; one
// thread per (row, plane); rows >= `rows` and dimensions >= dim are zero.
__global__ void fbc_nn_split(const float* __restrict__ src, long long rows, int dim, int tile_rows, int nc,
                             long long padded_rows, uint8_t* __restrict__ hi, uint8_t* __restrict__ lo, int split) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= padded_rows * nc) return;
    const long long row = i / nc;
    const int c = (int)(i - row * nc);
    __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int d = c * 8 + k;
        const float v = (row < rows && d < dim) ? __ldg(src + row * dim + d) : 0.f;
        h[k] = __float2bfloat16_rn(v);
        l[k] = __float2bfloat16_rn(v - __bfloat162float(h[k]));
    }
    const long long tile = row / tile_rows, rr = row - tile * tile_rows;
    const long long off = ((tile * nc + c) * tile_rows + rr) * 16;
    *reinterpret_cast<uint4*>(hi + off) = *reinterpret_cast<const uint4*>(h);
    if (split) *reinterpret_cast<uint4*>(lo + off) = *reinterpret_cast<const uint4*>(l);
}

// n2[j] = sum_k n[j][k]^2 (FP32, sequential); +inf for the padding rows.
__global__ void fbc_nn_norms(const float* __restrict__ n, long long rows, int dim, long long padded_rows,
                             float* __restrict__ n2) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= padded_rows) return;
    if (j >= rows) {
        n2[j] = __int_as_float(0x7f800000);
        return;
    }
    float s = 0.f;
    for (int k = 0; k < dim; ++k) {
        const float v = __ldg(n + j * dim + k);
        s = fmaf(v, v, s);
    }
    n2[j] = s;
}

// One thread per target: the kRerank smallest distinct candidate keys, then the
// exact FP32 distance of each; the smallest wins (lowest index on ties).
__global__ void fbc_nn_finalize(const unsigned long long* __restrict__ part, int cands, long long rows_total,
                                const float* __restrict__ t, const float* __restrict__ n, long long nt, int dim,
                                long long* __restrict__ idx_out, float* __restrict__ dist_out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    unsigned long long best[kRerank];
#pragma unroll
    for (int r = 0; r < kRerank; ++r) best[r] = ~0ull;
    for (int q = 0; q < cands; ++q) {
        // candidate q of target i: slot q % 2 of item-part q / 2
        const unsigned long long key = __ldg(part + ((long long)(q >> 1) * rows_total + i) * 2 + (q & 1));
        if (key >= best[kRerank - 1]) continue;
        bool dup = false;
#pragma unroll
        for (int r = 0; r < kRerank; ++r) dup |= (best[r] == key);
        if (dup) continue;
        unsigned long long v = key;
#pragma unroll
        for (int r = 0; r < kRerank; ++r)
            if (v < best[r]) {
                const unsigned long long tmp = best[r];
                best[r] = v;
                v = tmp;
            }
    }
    long long bj = -1;
    float bd = __int_as_float(0x7f800000);
    const float* ti = t + i * dim;
    for (int r = 0; r < kRerank; ++r) {
        if (best[r] == ~0ull) break;
        const long long j = (long long)(best[r] & 0xffffffffull);
        const float* nj = n + j * dim;
        float d = 0.f;
        for (int k = 0; k < dim; ++k) {
            const float e = __ldg(ti + k) - __ldg(nj + k);
            d = fmaf(e, e, d);
        }
        if (d < bd || (d == bd && j < bj)) {
            bd = d;
            bj = j;
        }
    }
    idx_out[i] = bj;
    dist_out[i] = bd;
}

std::string nn_kernel_name(int nc, int split) {
    char b[64];
    snprintf(b, sizeof b, "fbc_nn_c%d_s%d_e%d", nc, split, kEW);
    return b;
}

std::string nn_kernel_source(int nc, int split) {
    std::ostringstream o;
    o << rtcg_nn_params_source() << "\n" << rtcg_ptx_source() << "\n" << rtcg_nn_source() << "\n";
    o << "static_assert(sizeof(FbcNnParams) == " << sizeof(FbcNnParams)
      << ", \"host and device disagree on the parameter block\");\n";
    o << "extern \"C\" __global__ void __launch_bounds__(" << 64 + 32 * kEW << ", 1) " << nn_kernel_name(nc, split)
      << "(const __grid_constant__ FbcNnParams P) {\n  fbc_nn_body<" << nc << "," << split << "," << kEW
      << ">(P);\n}\n";
    return o.str();
}

}  // namespace
}  // namespace fbc

using namespace fbc;

struct fbcorr_nn_plan {
    int64_t nt = 0, nn = 0, dim = 0;
    int nc = 0, split = 1;
    FbcNnParams kp{};
    int grid = 0;
    size_t smem = 0, ws = 0;
    size_t off_thi = 0, off_tlo = 0, off_nhi = 0, off_nlo = 0, off_n2 = 0, off_part = 0;
    Kernel k;
    int* err_host = nullptr;
    int* err_dev = nullptr;
};

extern "C" {

fbcorr_status_t fbcorr_nn_plan_create(fbcorr_nn_plan_t* out, int64_t n_targets, int64_t n_neighbors, int64_t dim,
                                      fbcorr_dtype_t dtype) {
    clear_error();
    if (!out) return set_error(FBCORR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (dtype != FBCORR_BF16X3 && dtype != FBCORR_BF16)
        return set_error(FBCORR_ERR_UNSUPPORTED, "nearest-neighbour search runs in BF16X3 or BF16");
    if (n_targets <= 0 || n_neighbors <= 0 || dim <= 0)
        return set_error(FBCORR_ERR_SHAPE, "n_targets, n_neighbors and dim must be positive");
    if (dim > 64) return set_error(FBCORR_ERR_UNSUPPORTED, "dimension %lld > 64", (long long)dim);
    if (n_neighbors > (1LL << 31) || n_targets > (1LL << 31))
        return set_error(FBCORR_ERR_SHAPE, "more than 2^31 targets or neighbours");
    DeviceInfo dev;
    FBC_TRY(device_info(&dev));
    if (dev.cc_major != 10 || dev.cc_minor != 3)
        return set_error(FBCORR_ERR_UNSUPPORTED, "libfbcorr is built for sm_103a (GB300)");
    fbcorr_nn_plan* p = new (std::nothrow) fbcorr_nn_plan();
    if (!p) return set_error(FBCORR_ERR_OOM, "host allocation failed");
    p->nt = n_targets;
    p->nn = n_neighbors;
    p->dim = dim;
    p->nc = (int)((dim + 15) / 16 * 2);
    p->split = dtype == FBCORR_BF16X3 ? 1 : 0;
    FbcNnParams& k = p->kp;
    k.t_tiles = (int)((n_targets + FBC_NN_TILE_T - 1) / FBC_NN_TILE_T);
    k.n_tiles = (int)((n_neighbors + FBC_NN_TILE_N - 1) / FBC_NN_TILE_N);
    k.a_bytes = (unsigned)(p->nc * FBC_NN_TILE_T * 16);
    k.b_bytes = (unsigned)(p->nc * FBC_NN_TILE_N * 16);
    const size_t halves = p->split ? 2 : 1;
    // as many B stages as fit next to two A slots (at least two)
    // (barriers: 512 bytes; two 1 KB slots of |n|^2).  The target tile changes once
    // per work item, so one A slot costs a short wait per item; it is used when it
    // makes room for one more neighbour stage (the refill latency of a stage is
    // what the screening MMAs wait on)
    const size_t room = kSmemMax - 512 - 2048;
    auto stages = [&](int na) {
        return std::min<size_t>(6, (room - (size_t)na * halves * k.a_bytes) / (halves * k.b_bytes));
    };
    k.na = stages(1) > stages(2) ? 1 : 2;
    k.nb = (int)stages(k.na);
    if (k.nb < 2) {
        delete p;
        return set_error(FBCORR_ERR_UNSUPPORTED, "tiles do not fit in shared memory");
    }
    k.a_off = 0;
    k.b_off = (unsigned)(k.na * halves * k.a_bytes);
    k.bar_off = (unsigned)(k.b_off + k.nb * halves * k.b_bytes);
    k.nrm_off = k.bar_off + 512;
    p->smem = k.nrm_off + 2 * FBC_NN_TILE_N * 4;
    // work items: one target tile against a chunk of neighbour tiles, about four
    // waves of items over the SMs, at most 64 tiles per chunk
    const long long want = 4LL * std::max(1, dev.sm_count);
    long long chunk = ((long long)k.n_tiles * k.t_tiles + want - 1) / want;
    chunk = std::max(1LL, std::min(64LL, chunk));
    k.chunk_tiles = (int)chunk;
    k.chunks = (int)((k.n_tiles + chunk - 1) / chunk);
    p->grid = (int)std::min<long long>((long long)k.chunks * k.t_tiles, dev.sm_count);
    const long long rows_total = (long long)k.t_tiles * FBC_NN_TILE_T;
    size_t off = 0;
    p->off_thi = off; off = align_up(off + (size_t)k.t_tiles * k.a_bytes, 256);
    p->off_tlo = off; if (p->split) off = align_up(off + (size_t)k.t_tiles * k.a_bytes, 256);
    p->off_nhi = off; off = align_up(off + (size_t)k.n_tiles * k.b_bytes, 256);
    p->off_nlo = off; if (p->split) off = align_up(off + (size_t)k.n_tiles * k.b_bytes, 256);
    p->off_n2 = off; off = align_up(off + (size_t)k.n_tiles * FBC_NN_TILE_N * 4, 256);
    p->off_part = off; off = align_up(off + (size_t)k.chunks * (kEW / 4) * rows_total * 2 * 8, 256);
    p->ws = off;
    const long long wait_ms = atoll(env_str("FBCORR_WAIT_MS", "4000").c_str());
    k.wait_ns = (unsigned long long)std::max(1LL, wait_ms) * 1000000ull;
    fbcorr_status_t s = FBCORR_OK;
    if (cudaHostAlloc((void**)&p->err_host, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&p->err_dev, p->err_host, 0) != cudaSuccess) {
        cudaGetLastError();
        s = set_error(FBCORR_ERR_OOM, "mapped host allocation for the error word failed");
    } else {
        *p->err_host = 0;
        s = rtcg_kernel(nn_kernel_source(p->nc, p->split), nn_kernel_name(p->nc, p->split), kSmemMax,
                        64 + 32 * kEW, &p->k);
    }
    if (s != FBCORR_OK) {
        fbcorr_nn_plan_destroy(p);
        return s;
    }
    p->k.smem = p->smem;
    logf("nn plan: %lld targets x %lld neighbours x %lld: %d x %d tiles, chunk %d, %d items, grid %d, nb %d, ws %zu",
         (long long)n_targets, (long long)n_neighbors, (long long)dim, k.t_tiles, k.n_tiles, k.chunk_tiles,
         k.chunks * k.t_tiles, p->grid, k.nb, p->ws);
    *out = p;
    return FBCORR_OK;
}

fbcorr_status_t fbcorr_nn_plan_destroy(fbcorr_nn_plan_t p) {
    clear_error();
    if (!p) return FBCORR_OK;
    if (p->err_host) cudaFreeHost(p->err_host);
    delete p;
    return FBCORR_OK;
}

fbcorr_status_t fbcorr_nn_workspace_size(fbcorr_nn_plan_t p, size_t* bytes) {
    clear_error();
    if (!p || !bytes) return set_error(FBCORR_ERR_INVALID_ARG, "NULL argument");
    *bytes = p->ws;
    return FBCORR_OK;
}

fbcorr_status_t fbcorr_nn_plan_device_status(fbcorr_nn_plan_t p, int clear) {
    clear_error();
    if (!p) return set_error(FBCORR_ERR_INVALID_ARG, "NULL plan");
    const int v = p->err_host ? *(volatile int*)p->err_host : 0;
    if (clear && p->err_host) *(volatile int*)p->err_host = 0;
    if (v != 0) return set_error(FBCORR_ERR_TIMEOUT, "the nearest-neighbour kernel gave up a bounded wait (code %d)", v);
    return FBCORR_OK;
}

fbcorr_status_t fbcorr_nn_search(fbcorr_nn_plan_t p, const float* targets, const float* neighbors,
                                 int64_t* idx_out, float* dist_out, void* ws, size_t ws_bytes,
                                 fbcorr_stream_t stream) {
    clear_error();
    if (!p || !targets || !neighbors || !idx_out || !dist_out)
        return set_error(FBCORR_ERR_INVALID_ARG, "NULL argument");
    const void* ptrs[] = {targets, neighbors, idx_out, dist_out, ws};
    for (const void* q : ptrs)
        if (((uintptr_t)q & 15u) != 0) return set_error(FBCORR_ERR_ALIGNMENT, "pointers must be 16-byte aligned");
    if (!ws || ws_bytes < p->ws)
        return set_error(FBCORR_ERR_WORKSPACE, "search needs %zu bytes of workspace (got %zu)", p->ws, ws_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t* base = static_cast<uint8_t*>(ws);
    FbcNnParams kp = p->kp;
    kp.thi = base + p->off_thi;
    kp.tlo = base + p->off_tlo;
    kp.nhi = base + p->off_nhi;
    kp.nlo = base + p->off_nlo;
    kp.n2 = reinterpret_cast<const float*>(base + p->off_n2);
    kp.part = reinterpret_cast<unsigned long long*>(base + p->off_part);
    kp.err = p->err_dev;
    const long long t_rows = (long long)kp.t_tiles * FBC_NN_TILE_T, n_rows = (long long)kp.n_tiles * FBC_NN_TILE_N;
    const long long tw = t_rows * p->nc, nw = n_rows * p->nc;
    fbc_nn_split<<<(unsigned)((tw + 255) / 256), 256, 0, s>>>(targets, p->nt, (int)p->dim, FBC_NN_TILE_T, p->nc,
                                                              t_rows, base + p->off_thi, base + p->off_tlo, p->split);
    fbc_nn_split<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(neighbors, p->nn, (int)p->dim, FBC_NN_TILE_N, p->nc,
                                                              n_rows, base + p->off_nhi, base + p->off_nlo, p->split);
    fbc_nn_norms<<<(unsigned)((n_rows + 255) / 256), 256, 0, s>>>(neighbors, p->nn, (int)p->dim, n_rows,
                                                                  reinterpret_cast<float*>(base + p->off_n2));
    FBC_CUDA(cudaGetLastError());
    void* args[] = {&kp};
    FBC_TRY(launch(p->k, dim3(p->grid), args, s));
    const int cands = kp.chunks * (kEW / 4) * 2;
    fbc_nn_finalize<<<(unsigned)((p->nt + 127) / 128), 128, 0, s>>>(
        reinterpret_cast<const unsigned long long*>(base + p->off_part), cands, t_rows, targets, neighbors, p->nt,
        (int)p->dim, reinterpret_cast<long long*>(idx_out), dist_out);
    FBC_CUDA(cudaGetLastError());
    return FBCORR_OK;
}

fbcorr_status_t fbcorr_nn_rtcg_check(int64_t dim, fbcorr_dtype_t dtype, char* log, size_t cap) {
    clear_error();
    if (log && cap) log[0] = '\0';
    if (dtype != FBCORR_BF16X3 && dtype != FBCORR_BF16)
        return set_error(FBCORR_ERR_UNSUPPORTED, "nearest-neighbour search runs in BF16X3 or BF16");
    if (dim <= 0 || dim > 64) return set_error(FBCORR_ERR_UNSUPPORTED, "dimension must be 1..64");
    std::string lg;
    const fbcorr_status_t st = rtcg_compile_only(nn_kernel_source((int)((dim + 15) / 16 * 2), dtype == FBCORR_BF16X3), &lg);
    if (st != FBCORR_OK && log && cap) snprintf(log, cap, "%s", lg.c_str());
    return st;
}

}  // extern "C"
