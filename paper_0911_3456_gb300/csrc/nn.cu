// nn.cu -- exact brute-force nearest-neighbour search (Sec. 6.4 of the paper):
// plans, the split / norm pre-pass, the run-time generated tensor-core screening
// kernel (rtcg_nn.cuh) and the exact re-ranking.
//
// Per call: (1) fbc_nn_split writes targets and neighbours as BF16 hi (and lo)
// chunk planes in tile-major order (one bulk copy brings a whole tile) and, in
// the same pass (or fbc_nn_norms for 48-dimension planes), the neighbour norms
// |n|^2 in FP32 and their maximum; (2) the
// generated kernel screens every (target, neighbour) pair on the tensor cores
// and keeps, per work item part and target, the FBC_NN_KEEP smallest keys of
// d' = |n|^2 - 2 t.n; (3) fbc_nn_finalize certifies the screening per target:
// with E the bound on the screening error of any d' of that target (below), the
// true nearest neighbour j* satisfies d'(j*) <= m + 2E, m the smallest screened
// key, so every neighbour screened at most m + 2E (the window) is re-ranked by
// its exact FP32 squared distance sum_k (t_k - n_k)^2 (ties: lowest index).  The
// window is known to be complete when no part's last kept key lies inside it (a
// part keeps FBC_NN_KEEP keys, so a last key inside the window may hide another);
// otherwise (4) fbc_nn_part_scan takes the target's exact FP32 distance to every
// neighbour of each such part (up to kPartCap parts per target; beyond that
// fbc_nn_exact_scan takes all neighbours), and fbc_nn_exact_write stores the
// result.  So every target gets the argmin of the exact FP32 distance over all
// neighbours.
//
// The screening error bound, per target t with |n_j| <= Nmax for every j:
//   |d'_screened - d'| <= 2 (c_prod + c_acc) |t| Nmax     (the dot product)
//                       + gamma_dim Nmax^2                (the FP32 norm |n|^2)
//                       + u (Nmax^2 + 2 |t| Nmax)         (rounding of the key)
// c_prod: operand rounding per product, 3.05 * 2^-16 for split BF16 (the hi*lo,
// lo*hi, lo*lo and residual terms) and 2 * 2^-8 + 2^-16 for plain BF16; c_acc =
// (MMAs accumulated + 2) * 2^-22 for the FP32 accumulation in the tensor core;
// u = 2^-24, gamma_dim = dim * u / (1 - dim * u); sum_k |t_k n_k| <= |t| |n| by
// Cauchy-Schwarz.  The bound is taken 1.25-fold, and the window is widened by
// the FP32 rounding of the exact distances, so that the FP32 argmin over all
// neighbours lies in it.  Nmax can be lowered per target: the screened best j_m
// and the true nearest j* both lie within sqrt(|t|^2 + m + E(Nmax)) of t, so
// |n_j| <= |t| + sqrt(|t|^2 + m + E(Nmax)) for both, and E is taken with the
// smaller of that and Nmax.
//
// Key threshold (FBCORR_NN_PRESCREEN, default 16): the same screening kernel
// first runs over the first 1/16 of the neighbour tiles (at least two); U, the
// smallest key it finds for a target, is a screened key of some neighbour, and
// the full screening computes that neighbour's key bit for bit the same, so
// m <= U.  The window m + 2E(+ rounding) grows with m (every step of its FP32
// formula is monotone), so it lies below T = the window formula at U, moved up
// by one ulp.  The full screening keeps, per part, only keys below T: a part
// with fewer than FBC_NN_KEEP of them stores the empty key (complete, its other
// neighbours are at or above T, outside the window), the smallest key m is
// unchanged (it is at most U < T), and every neighbour inside the window is
// still kept or its part listed.  With T known from the first tile on, a chunk
// rarely beats a row's last key, and the insertions that dominated the
// epilogue's work almost vanish.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <new>
#include <sstream>

#include "internal.h"
#include "nn_params.h"

namespace fbc {
namespace {

constexpr int kEW = 8;           // epilogue warps
constexpr int kScanRows = 256;   // neighbours per block step of the exhaustive fallback
constexpr int kPartCap = 8;      // incomplete parts re-scanned per target before a full scan
constexpr size_t kSmemMax = 227 * 1024 - 1024;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Per-search counters in the workspace (16 bytes, zeroed before every search).
struct NnStats {
    unsigned nmax2_bits;   // max_j |n_j|^2 as FP32 bits (non-negative: integer order)
    int flagged;           // targets whose window could not be certified
    int entries;           // (target, part) re-scans listed
    int full;              // targets listed for the scan of every neighbour
};

// rows x dim FP32 -> tile-major BF16 planes [tiles][nc][tile_rows][8 values]; one
// thread per (row, plane); rows >= `rows` and dimensions >= dim are zero.  With
// n2 != nullptr (the neighbour set; nc a power of two, so a row's nc threads are
// consecutive lanes of one warp) the threads of a row also form |n|^2: each sums
// the squares of its 8 values, the row's lanes add theirs by a shuffle tree, and
// its first lane stores the sum (+inf for the padding rows) and joins the
// warp's maximum, which goes to stats->nmax2_bits.
__global__ void fbc_nn_split(const float* __restrict__ src, long long rows, int dim, int tile_rows, int nc,
                             long long padded_rows, uint8_t* __restrict__ hi, uint8_t* __restrict__ lo, int split,
                             float* __restrict__ n2, NnStats* __restrict__ stats) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < padded_rows * nc;
    const long long row = active ? i / nc : 0;
    const int c = (int)(i - row * nc);
    float sq = 0.f;
    if (active) {
        __nv_bfloat16 h[8], l[8];
        // the row's 8 values: two 16-byte loads when rows are whole 32-byte chunks
        float vv[8];
        const bool inside = row < rows && c * 8 < dim;
        if (inside && (dim & 7) == 0 && (reinterpret_cast<unsigned long long>(src) & 15) == 0) {
            const float4* s4 = reinterpret_cast<const float4*>(src + row * dim + c * 8);
            const float4 a = __ldg(s4), b = __ldg(s4 + 1);
            vv[0] = a.x; vv[1] = a.y; vv[2] = a.z; vv[3] = a.w;
            vv[4] = b.x; vv[5] = b.y; vv[6] = b.z; vv[7] = b.w;
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) vv[k] = (inside && c * 8 + k < dim) ? __ldg(src + row * dim + c * 8 + k) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float v = vv[k];
            sq = fmaf(v, v, sq);
            h[k] = __float2bfloat16_rn(v);
            l[k] = __float2bfloat16_rn(v - __bfloat162float(h[k]));
        }
        const long long tile = row / tile_rows, rr = row - tile * tile_rows;
        const long long off = ((tile * nc + c) * tile_rows + rr) * 16;
        *reinterpret_cast<uint4*>(hi + off) = *reinterpret_cast<const uint4*>(h);
        if (split) *reinterpret_cast<uint4*>(lo + off) = *reinterpret_cast<const uint4*>(l);
    }
    if (n2 == nullptr) return;   // uniform over the grid
    for (int m = 1; m < nc; m <<= 1) sq += __shfl_xor_sync(0xffffffffu, sq, m);
    const bool first = active && c == 0;
    if (first) n2[row] = row < rows ? sq : __int_as_float(0x7f800000);
    unsigned b = (first && row < rows) ? __float_as_uint(sq) : 0u;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, m));
    if ((threadIdx.x & 31) == 0 && b > *(volatile unsigned*)&stats->nmax2_bits) atomicMax(&stats->nmax2_bits, b);
}

// n2[j] = sum_k n[j][k]^2 (FP32, sequential); +inf for the padding rows; the
// maximum over the real rows into stats->nmax2_bits.  A block stages kNormRows
// rows with coalesced loads ([row][dim + 1]: conflict-free row reads), each
// thread sums one row, and the block's maximum goes out with one atomicMax
// (skipped when the stored maximum is already larger).
constexpr int kNormRows = 128;
__global__ void __launch_bounds__(kNormRows) fbc_nn_norms(const float* __restrict__ n, long long rows, int dim,
                                                          long long padded_rows, float* __restrict__ n2,
                                                          NnStats* __restrict__ stats) {
    extern __shared__ float fbc_nn_nrows[];   // [kNormRows][dim + 1]
    const long long r0 = (long long)blockIdx.x * kNormRows;
    const int tid = threadIdx.x;
    const long long left = rows - r0;
    const int real = (int)(left <= 0 ? 0 : (left < kNormRows ? left : kNormRows));
    // row = e / dim by a float reciprocal: exact here (e < 2^13, the error of the
    // product is far below the 0.5 / dim margin of e + 0.5)
    const float inv_dim = 1.f / (float)dim;
    for (int e = tid; e < real * dim; e += kNormRows) {
        const int r = (int)(((float)e + 0.5f) * inv_dim);
        fbc_nn_nrows[r * (dim + 1) + (e - r * dim)] = __ldg(n + r0 * dim + e);
    }
    __syncthreads();
    float sq = 0.f;
    if (tid < real) {
        const float* r = fbc_nn_nrows + tid * (dim + 1);
        for (int k = 0; k < dim; ++k) sq = fmaf(r[k], r[k], sq);
    }
    const long long j = r0 + tid;
    if (j < padded_rows) n2[j] = tid < real ? sq : __int_as_float(0x7f800000);
    __shared__ unsigned wmax[kNormRows / 32];
    unsigned b = __float_as_uint(sq);   // 0 for rows past the end
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, m));
    if ((tid & 31) == 0) wmax[tid >> 5] = b;
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < kNormRows / 32; ++w) b = max(b, wmax[w]);
        if (b > *(volatile unsigned*)&stats->nmax2_bits) atomicMax(&stats->nmax2_bits, b);
    }
}

__device__ __forceinline__ float fbc_nn_key_dist(unsigned long long key) {
    // inverse of the screening kernel's order-preserving map of the float
    const unsigned u = (unsigned)(key >> 32);
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Exact FP32 squared distance, one fused multiply-add per coordinate in order.
__device__ __forceinline__ float fbc_nn_exact_dist(const float* __restrict__ ti, const float* __restrict__ nj,
                                                   int dim) {
    float d = 0.f;
    for (int k = 0; k < dim; ++k) {
        const float e = __ldg(ti + k) - __ldg(nj + k);
        d = fmaf(e, e, d);
    }
    return d;
}

// One thread per target: the smallest screened key m, the window m + 2E (+ the
// rounding of the exact distances), every candidate inside it re-ranked by its
// exact FP32 distance; a part whose last kept key lies inside the window may hold
// more candidates in it than it kept, and is listed for an exact re-scan.
struct NnFinalizeArgs {
    const unsigned long long* part;
    int cands;                  // keys per target: parts x FBC_NN_KEEP
    long long rows_total;
    const float* t;
    const float* n;
    long long nt;
    int dim;
    float c_dot;                // 2 (c_prod + c_acc)
    float c_nrm;                // gamma_dim + u (norm and key rounding of Nmax^2)
    float c_key;                // u (key rounding of 2 |t| Nmax)
    float c_rr;                 // relative rounding of the exact FP32 distances
    NnStats* stats;
    int* flag_list;             // targets with at least one incomplete part
    int2* entries;              // (target, part) re-scans: kPartCap slots per target
    int* entry_list;            // the slots in use
    int* full_list;             // targets with more than kPartCap incomplete parts
    unsigned long long* best_key;
    long long* idx_out;
    float* dist_out;
};

__device__ __forceinline__ float fbc_nn_bound(const NnFinalizeArgs& A, float tn, float nb) {
    return 1.25f * (A.c_dot * tn * nb + A.c_nrm * nb * nb + A.c_key * 2.f * tn * nb);
}

// The certificate window of a target whose smallest screened key is m: m + 2E,
// E with the norm bound lowered by m (file header), widened by the rounding of
// the exact distances.  Every operation is monotone in m.
__device__ __forceinline__ float fbc_nn_window(const NnFinalizeArgs& A, float t2, float tn, float nmax, float m) {
    const float e_max = fbc_nn_bound(A, tn, nmax);
    const float nb = fminf(nmax, (tn + sqrtf(fmaxf(t2 + m + e_max, 0.f))) * 1.0001f);
    const float e = fbc_nn_bound(A, tn, nb);
    // the exact distances carry a relative FP32 rounding; the best is at most t2 + m + e
    return m + 2.f * e + A.c_rr * 2.f * fmaxf(t2 + m + e, 0.f);
}

// The key threshold of every target row (file header): U = the smallest first
// key of the sample screening's parts, T = the window at U plus one ulp; padding
// rows and targets with no sampled key get +inf.  One warp per row (the same
// |t|^2 loop as fbc_nn_finalize, so the same bits), lanes over the parts.
__global__ void __launch_bounds__(128) fbc_nn_threshold(const NnFinalizeArgs A, float* thr) {
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= A.rows_total) return;   // warp-uniform
    float T = __int_as_float(0x7f800000);
    if (i < A.nt) {
        const int nparts = A.cands / FBC_NN_KEEP;
        float u = __int_as_float(0x7f800000);
        for (int pq = lane; pq < nparts; pq += 32) {
            const unsigned long long k0 = __ldg(A.part + ((long long)pq * A.rows_total + i) * FBC_NN_KEEP);
            if (k0 != ~0ull) u = fminf(u, fbc_nn_key_dist(k0));
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) u = fminf(u, __shfl_xor_sync(0xffffffffu, u, o));
        if (u < __int_as_float(0x7f800000)) {
            const float* ti = A.t + i * A.dim;
            float t2 = 0.f;
            for (int k = 0; k < A.dim; ++k) t2 = fmaf(__ldg(ti + k), __ldg(ti + k), t2);
            const float nmax = sqrtf(__uint_as_float(A.stats->nmax2_bits));
            T = nextafterf(fbc_nn_window(A, t2, sqrtf(t2), nmax, u), __int_as_float(0x7f800000));
        }
    }
    if (lane == 0) thr[i] = T;
}

// One warp per target; lane l takes the parts l, l + 32, ...
__global__ void __launch_bounds__(128) fbc_nn_finalize(const NnFinalizeArgs A) {
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= A.nt) return;   // warp-uniform
    const float* ti = A.t + i * A.dim;
    float t2 = 0.f;
    for (int k = 0; k < A.dim; ++k) t2 = fmaf(__ldg(ti + k), __ldg(ti + k), t2);
    const float tn = sqrtf(t2);
    const float nmax = sqrtf(__uint_as_float(A.stats->nmax2_bits));
    const int nparts = A.cands / FBC_NN_KEEP;
    float m = __int_as_float(0x7f800000);
    for (int pq = lane; pq < nparts; pq += 32) {
        const unsigned long long k0 = __ldg(A.part + ((long long)pq * A.rows_total + i) * FBC_NN_KEEP);
        if (k0 != ~0ull) m = fminf(m, fbc_nn_key_dist(k0));   // a part's first key is its smallest
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const float win = fbc_nn_window(A, t2, tn, nmax, m);
    unsigned long long best = ~0ull;   // (exact distance bits, index): distances are >= 0
    int n_over = 0;
    for (int pq0 = 0; pq0 < nparts; pq0 += 32) {
        const int pq = pq0 + lane;
        bool over = false;
        if (pq < nparts) {
            const unsigned long long* pk = A.part + ((long long)pq * A.rows_total + i) * FBC_NN_KEEP;
            unsigned long long kk[FBC_NN_KEEP];
#pragma unroll
            for (int h = 0; h < FBC_NN_KEEP; ++h) kk[h] = __ldg(pk + h);
            over = kk[FBC_NN_KEEP - 1] != ~0ull && fbc_nn_key_dist(kk[FBC_NN_KEEP - 1]) <= win;
#pragma unroll
            for (int h = 0; h < FBC_NN_KEEP; ++h) {
                const unsigned long long key = kk[h];
                if (key == ~0ull || fbc_nn_key_dist(key) > win) continue;
                const long long j = (long long)(key & 0xffffffffull);
                const float d = fbc_nn_exact_dist(ti, A.n + j * A.dim, A.dim);
                const unsigned long long ek = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned long long)j;
                best = ek < best ? ek : best;
            }
        }
        // incomplete parts, in part order, up to kPartCap of them
        const unsigned ball = __ballot_sync(0xffffffffu, over);
        if (over) {
            const int slot = n_over + __popc(ball & ((1u << lane) - 1u));
            if (slot < kPartCap) A.entries[(long long)i * kPartCap + slot] = make_int2((int)i, pq);
        }
        n_over += __popc(ball);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
        best = v < best ? v : best;
    }
    if (lane != 0) return;
    if (n_over == 0) {
        A.idx_out[i] = best == ~0ull ? -1 : (long long)(best & 0xffffffffull);
        A.dist_out[i] = best == ~0ull ? __int_as_float(0x7f800000) : __uint_as_float((unsigned)(best >> 32));
        return;
    }
    // the re-scans start from the best exact candidate found so far
    A.best_key[i] = best;
    A.flag_list[atomicAdd(&A.stats->flagged, 1)] = (int)i;
    if (n_over <= kPartCap) {
        // the target's entries were written to its own kPartCap slots; list them
        const int e0 = atomicAdd(&A.stats->entries, n_over);
        for (int k = 0; k < n_over; ++k) A.entry_list[e0 + k] = (int)(i * kPartCap + k);
    } else {
        A.full_list[atomicAdd(&A.stats->full, 1)] = (int)i;
    }
}

// Exact re-scan of the incomplete parts.  A part's neighbours are the 32-column
// chunks part, part + parts, ... of the tiles of its chunk; the work units are
// (listed part, step of kScanRows of its neighbours), spread over the grid so
// that a few hundred parts keep every SM busy.  A unit stages its rows in shared
// memory (16-byte loads when the rows allow), each thread takes the exact FP32
// distance of one neighbour (the target in shared memory, the same sequential
// fmaf order as everywhere), and the smallest key of each warp goes to the
// target's best_key by atomicMin.
struct NnPartScanArgs {
    const NnStats* stats;
    const int2* entries;
    const int* entry_list;
    const float* t;
    const float* n;
    long long nn;
    int dim;
    int pre_chunks;             // chunks 0 .. pre_chunks - 1: the sample screening's,
    int pre_chunk_tiles;        //   pre_chunk_tiles tiles each from tile 0, up to sample_tiles
    int sample_tiles;
    int chunk_tiles;            // then chunk_tiles tiles each from sample_tiles, up to n_tiles
    int n_tiles;
    int parts;                  // parts per chunk (epilogue warps / 4)
    unsigned long long* best_key;
};

__global__ void __launch_bounds__(kScanRows) fbc_nn_part_scan(const NnPartScanArgs A) {
    const int cnt = A.stats->entries;
    if (cnt == 0) return;
    extern __shared__ float fbc_nn_prows[];   // [kScanRows][dim + 1], then the target [dim]
    float* tv = fbc_nn_prows + kScanRows * (A.dim + 1);
    const int tid = threadIdx.x;
    const int cols = (256 / 32) / A.parts;                  // 32-column chunks per tile in one part
    const int most = max(A.pre_chunks > 0 ? A.pre_chunk_tiles : 0, A.chunk_tiles) * cols * 32;
    const int steps = (most + kScanRows - 1) / kScanRows;   // of the largest part
    const long long units = (long long)cnt * steps;
    const bool vec = (A.dim & 3) == 0 && (reinterpret_cast<unsigned long long>(A.n) & 15) == 0;
    const float inv_dim = 1.f / (float)A.dim;
    int cur = -1;                                           // entry whose target is in tv
    for (long long w = blockIdx.x; w < units; w += gridDim.x) {
        const int e = (int)(w / steps);
        const int u0 = (int)(w - (long long)e * steps) * kScanRows;
        const int2 en = A.entries[A.entry_list[e]];
        const int c = en.y / A.parts, p = en.y - c * A.parts;
        // the tiles of chunk c
        int t0, tn;
        if (c < A.pre_chunks) {
            t0 = c * A.pre_chunk_tiles;
            tn = min(A.sample_tiles, t0 + A.pre_chunk_tiles) - t0;
        } else {
            t0 = A.sample_tiles + (c - A.pre_chunks) * A.chunk_tiles;
            tn = min(A.n_tiles, t0 + A.chunk_tiles) - t0;
        }
        const int per_part = tn * cols * 32;
        if (u0 >= per_part) continue;   // block-uniform: a step past this part's end
        // neighbour index of the part's u-th row: runs of 32 consecutive rows
        auto row_of = [&](int u) -> long long {
            const int jt = t0 + u / (cols * 32);
            const int r = u % (cols * 32);
            return (long long)jt * 256 + (p + (r >> 5) * A.parts) * 32 + (r & 31);
        };
        __syncthreads();   // the previous unit's readers are done
        if (e != cur) {    // block-uniform: w is
            for (int k = tid; k < A.dim; k += kScanRows) tv[k] = __ldg(A.t + (long long)en.x * A.dim + k);
            cur = e;
        }
        // kScanRows / 32 runs of 32 consecutive neighbours, each contiguous in memory
        for (int q = 0; q < kScanRows / 32; ++q) {
            const int u = u0 + 32 * q;
            if (u >= per_part) break;
            const long long j0 = row_of(u);
            const int nrow = (int)min(32LL, A.nn - j0);
            if (nrow <= 0) continue;
            const float* src = A.n + j0 * A.dim;
            float* dst = fbc_nn_prows + 32 * q * (A.dim + 1);
            if (vec) {
                const float4* src4 = reinterpret_cast<const float4*>(src);
                for (int f = tid; f < nrow * A.dim / 4; f += kScanRows) {
                    const int el = 4 * f;
                    // el / dim: exact, since el < 32 dim puts the quotient below 32 and at
                    // least 0.5 / dim from an integer, far above the product's rounding
                    const int r = (int)(((float)el + 0.5f) * inv_dim);
                    const float4 v = __ldg(src4 + f);
                    float* o = dst + r * (A.dim + 1) + (el - r * A.dim);
                    o[0] = v.x;
                    o[1] = v.y;
                    o[2] = v.z;
                    o[3] = v.w;
                }
            } else {
                for (int el = tid; el < nrow * A.dim; el += kScanRows) {
                    const int r = (int)(((float)el + 0.5f) * inv_dim);
                    dst[r * (A.dim + 1) + (el - r * A.dim)] = __ldg(src + el);
                }
            }
        }
        __syncthreads();
        unsigned long long key = ~0ull;
        const long long j = row_of(u0 + tid);
        if (u0 + tid < per_part && j < A.nn) {
            const float* nr = fbc_nn_prows + tid * (A.dim + 1);
            float d = 0.f;
            for (int k = 0; k < A.dim; ++k) {
                const float df = tv[k] - nr[k];
                d = fmaf(df, df, d);
            }
            key = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned long long)j;
        }
#pragma unroll
        for (int m2 = 16; m2 >= 1; m2 >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, key, m2);
            key = o < key ? o : key;
        }
        if ((tid & 31) == 0 && key != ~0ull) atomicMin(A.best_key + en.x, key);
    }
}

// Exhaustive scan for the targets with more than kPartCap incomplete parts:
// each block step stages kScanRows neighbours in shared memory ([row][dim + 1]:
// conflict-free column reads), then for every listed target each thread takes
// the exact FP32 distance of one
// neighbour; the smallest (distance, index) key of each warp goes to the
// target's best_key by atomicMin (order-independent, so deterministic).
__global__ void __launch_bounds__(kScanRows) fbc_nn_exact_scan(const NnStats* __restrict__ stats,
                                                               const int* __restrict__ full_list,
                                                               const float* __restrict__ t,
                                                               const float* __restrict__ n, long long nn, int dim,
                                                               unsigned long long* __restrict__ best_key) {
    const int cnt = stats->full;
    if (cnt == 0) return;
    extern __shared__ float fbc_nn_rows[];   // [kScanRows][dim + 1], then the target [dim]
    float* tv = fbc_nn_rows + kScanRows * (dim + 1);
    const int tid = threadIdx.x;
    for (long long r0 = (long long)blockIdx.x * kScanRows; r0 < nn; r0 += (long long)gridDim.x * kScanRows) {
        const int rows = (int)min((long long)kScanRows, nn - r0);
        __syncthreads();   // the previous step's readers are done
        for (int e = tid; e < rows * dim; e += kScanRows) {
            const int r = e / dim, k = e - r * dim;
            fbc_nn_rows[r * (dim + 1) + k] = __ldg(n + (r0 + r) * dim + k);
        }
        for (int f = 0; f < cnt; ++f) {
            const int i = __ldg(full_list + f);
            __syncthreads();   // rows staged; the previous target's readers are done
            for (int k = tid; k < dim; k += kScanRows) tv[k] = __ldg(t + (long long)i * dim + k);
            __syncthreads();
            unsigned long long key = ~0ull;
            if (tid < rows) {
                const float* nr = fbc_nn_rows + tid * (dim + 1);
                float d = 0.f;
                for (int k = 0; k < dim; ++k) {
                    const float e = tv[k] - nr[k];
                    d = fmaf(e, e, d);
                }
                key = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned long long)(r0 + tid);
            }
#pragma unroll
            for (int m2 = 16; m2 >= 1; m2 >>= 1) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, key, m2);
                key = o < key ? o : key;
            }
            if ((tid & 31) == 0 && key != ~0ull) atomicMin(best_key + i, key);
        }
    }
}

__global__ void fbc_nn_exact_write(const NnStats* __restrict__ stats, const int* __restrict__ flag_list,
                                   const unsigned long long* __restrict__ best_key, long long* __restrict__ idx_out,
                                   float* __restrict__ dist_out) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= stats->flagged) return;
    const int i = flag_list[f];
    const unsigned long long key = best_key[i];
    idx_out[i] = key == ~0ull ? -1 : (long long)(key & 0xffffffffull);
    dist_out[i] = key == ~0ull ? __int_as_float(0x7f800000) : __uint_as_float((unsigned)(key >> 32));
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
    FbcNnParams kpre{};   // the sample screening (key thresholds); kpre.n_tiles == 0: none
    int pre_grid = 0;
    size_t smem = 0, ws = 0;
    size_t off_thi = 0, off_tlo = 0, off_nhi = 0, off_nlo = 0, off_n2 = 0, off_part = 0;
    size_t off_thr = 0;
    size_t off_stats = 0, off_flag = 0, off_best = 0, off_entries = 0, off_elist = 0, off_full = 0;
    float c_dot = 0.f, c_nrm = 0.f, c_key = 0.f, c_rr = 0.f;   // screening error bound (nn.cu header)
    int scan_grid = 1;
    Kernel k;
    int* err_host = nullptr;
    int* err_dev = nullptr;
    // the last search's workspace and stream (fbcorr_nn_last_fallbacks reads its counters)
    const void* last_ws = nullptr;
    cudaStream_t last_stream = nullptr;
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
    // waves of items over the SMs, at most 16 tiles per chunk.  With the key
    // thresholds a short item costs no more insertions, and a part (and so an
    // exact re-scan) stays small: measured 4096 x 1M at 4 / 8 / 16 / 32 / 64 / 128
    // tiles 1.33 / 1.25 / 1.22 / 1.25 / 1.34 / 1.71 ms
    const long long want = 4LL * std::max(1, dev.sm_count);
    auto chunking = [&](FbcNnParams& q, int first, int end) {
        long long c = ((long long)(end - first) * k.t_tiles + want - 1) / want;
        c = std::max(1LL, std::min(16LL, c));
        q.tile0 = first;
        q.n_tiles = end;
        q.chunk_tiles = (int)c;
        q.chunks = (int)((end - first + c - 1) / c);
    };
    // the sample screening for the key thresholds (file header): the first
    // 1/FBCORR_NN_PRESCREEN of the neighbour tiles (default 16; 0: none), when
    // that is at least two tiles; the full screening then covers the other tiles,
    // and the sample's parts (kept without a threshold) join its parts
    const int n_tiles_all = k.n_tiles;
    const int pre_div = atoi(env_str("FBCORR_NN_PRESCREEN", "16").c_str());
    const int sample = (pre_div > 0 && n_tiles_all / pre_div >= 2) ? n_tiles_all / pre_div : 0;
    p->kpre = k;
    p->kpre.n_tiles = 0;
    p->kpre.chunks = 0;
    if (sample > 0) {
        chunking(p->kpre, 0, sample);
        p->kpre.chunk_base = 0;
        p->pre_grid = (int)std::min<long long>((long long)p->kpre.chunks * k.t_tiles, dev.sm_count);
    }
    chunking(k, sample, n_tiles_all);
    k.chunk_base = p->kpre.chunks;
    p->grid = (int)std::min<long long>((long long)k.chunks * k.t_tiles, dev.sm_count);
    const long long rows_total = (long long)k.t_tiles * FBC_NN_TILE_T;
    size_t off = 0;
    p->off_thi = off; off = align_up(off + (size_t)k.t_tiles * k.a_bytes, 256);
    p->off_tlo = off; if (p->split) off = align_up(off + (size_t)k.t_tiles * k.a_bytes, 256);
    p->off_nhi = off; off = align_up(off + (size_t)n_tiles_all * k.b_bytes, 256);
    p->off_nlo = off; if (p->split) off = align_up(off + (size_t)n_tiles_all * k.b_bytes, 256);
    p->off_n2 = off; off = align_up(off + (size_t)n_tiles_all * FBC_NN_TILE_N * 4, 256);
    // parts: the sample's chunks, then the full screening's
    const long long all_chunks = (long long)p->kpre.chunks + k.chunks;
    p->off_part = off; off = align_up(off + (size_t)all_chunks * (kEW / 4) * rows_total * FBC_NN_KEEP * 8, 256);
    p->off_thr = off; off = align_up(off + (size_t)rows_total * 4, 256);
    p->off_stats = off; off = align_up(off + sizeof(NnStats), 256);
    p->off_flag = off; off = align_up(off + (size_t)n_targets * 4, 256);
    p->off_best = off; off = align_up(off + (size_t)n_targets * 8, 256);
    p->off_entries = off; off = align_up(off + (size_t)n_targets * kPartCap * 8, 256);
    p->off_elist = off; off = align_up(off + (size_t)n_targets * kPartCap * 4, 256);
    p->off_full = off; off = align_up(off + (size_t)n_targets * 4, 256);
    p->ws = off;
    // the screening error bound's constants (see the file header)
    const double u = 1.0 / (1 << 24);
    const int n_mma = (p->split ? 3 : 1) * (p->nc / 2);
    const double c_prod = p->split ? 3.05 / 65536.0 : 2.0 / 256.0 + 1.0 / 65536.0;
    const double c_acc = (n_mma + 2) / (double)(1 << 22);
    const double gamma = dim * u / (1.0 - dim * u);
    p->c_dot = (float)(2.0 * (c_prod + c_acc));
    p->c_nrm = (float)(gamma + u);
    p->c_key = (float)u;
    p->c_rr = (float)((dim + 3) * u);
    p->scan_grid = std::max(1, 4 * dev.sm_count);
    const int scan_smem = (kScanRows * (int)(dim + 1) + (int)dim) * 4;
    if (cudaFuncSetAttribute((const void*)fbc_nn_exact_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, scan_smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute((const void*)fbc_nn_part_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, scan_smem) !=
            cudaSuccess) {
        cudaGetLastError();
        delete p;
        return set_error(FBCORR_ERR_CUDA, "shared memory of the exhaustive fallback kernel (%d bytes)", scan_smem);
    }
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
    NnStats* stats = reinterpret_cast<NnStats*>(base + p->off_stats);
    float* n2 = reinterpret_cast<float*>(base + p->off_n2);
    FBC_CUDA(cudaMemsetAsync(stats, 0, sizeof(NnStats), s));
    // the neighbour norms come with the split when a row's planes are lanes of one
    // warp (nc a power of two), else from their own kernel
    const bool fused_norms = (p->nc & (p->nc - 1)) == 0;
    fbc_nn_split<<<(unsigned)((tw + 255) / 256), 256, 0, s>>>(targets, p->nt, (int)p->dim, FBC_NN_TILE_T, p->nc,
                                                              t_rows, base + p->off_thi, base + p->off_tlo, p->split,
                                                              nullptr, nullptr);
    fbc_nn_split<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(neighbors, p->nn, (int)p->dim, FBC_NN_TILE_N, p->nc,
                                                              n_rows, base + p->off_nhi, base + p->off_nlo, p->split,
                                                              fused_norms ? n2 : nullptr, stats);
    if (!fused_norms)
        fbc_nn_norms<<<(unsigned)((n_rows + kNormRows - 1) / kNormRows), kNormRows,
                       (size_t)kNormRows * (p->dim + 1) * 4, s>>>(neighbors, p->nn, (int)p->dim, n_rows, n2, stats);
    FBC_CUDA(cudaGetLastError());
    NnFinalizeArgs fa;
    fa.part = reinterpret_cast<const unsigned long long*>(base + p->off_part);
    fa.cands = (p->kpre.chunks + kp.chunks) * (kEW / 4) * FBC_NN_KEEP;   // the sample's parts, then the rest
    fa.rows_total = t_rows;
    fa.t = targets;
    fa.n = neighbors;
    fa.nt = p->nt;
    fa.dim = (int)p->dim;
    fa.c_dot = p->c_dot;
    fa.c_nrm = p->c_nrm;
    fa.c_key = p->c_key;
    fa.c_rr = p->c_rr;
    fa.stats = stats;
    fa.flag_list = reinterpret_cast<int*>(base + p->off_flag);
    fa.entries = reinterpret_cast<int2*>(base + p->off_entries);
    fa.entry_list = reinterpret_cast<int*>(base + p->off_elist);
    fa.full_list = reinterpret_cast<int*>(base + p->off_full);
    fa.best_key = reinterpret_cast<unsigned long long*>(base + p->off_best);
    fa.idx_out = reinterpret_cast<long long*>(idx_out);
    fa.dist_out = dist_out;
    kp.thr = nullptr;
    if (p->kpre.n_tiles > 0) {
        // the sample screening, then the per-row key thresholds of the full one
        FbcNnParams kq = p->kpre;
        kq.thi = kp.thi;
        kq.tlo = kp.tlo;
        kq.nhi = kp.nhi;
        kq.nlo = kp.nlo;
        kq.n2 = kp.n2;
        kq.err = kp.err;
        kq.thr = nullptr;
        kq.part = kp.part;   // chunks 0 .. kpre.chunks - 1 of the part array
        void* qargs[] = {&kq};
        FBC_TRY(launch(p->k, dim3(p->pre_grid), qargs, s));
        NnFinalizeArgs qa = fa;
        qa.part = kq.part;
        qa.cands = kq.chunks * (kEW / 4) * FBC_NN_KEEP;
        float* thr = reinterpret_cast<float*>(base + p->off_thr);
        fbc_nn_threshold<<<(unsigned)((t_rows + 3) / 4), 128, 0, s>>>(qa, thr);
        FBC_CUDA(cudaGetLastError());
        kp.thr = thr;
    }
    void* args[] = {&kp};
    FBC_TRY(launch(p->k, dim3(p->grid), args, s));
    fbc_nn_finalize<<<(unsigned)((p->nt + 3) / 4), 128, 0, s>>>(fa);
    // the exact re-scans: each kernel returns at once when nothing is listed
    NnPartScanArgs pa;
    pa.stats = stats;
    pa.entries = fa.entries;
    pa.entry_list = fa.entry_list;
    pa.t = targets;
    pa.n = neighbors;
    pa.nn = p->nn;
    pa.dim = (int)p->dim;
    pa.pre_chunks = p->kpre.chunks;
    pa.pre_chunk_tiles = p->kpre.chunk_tiles;
    pa.sample_tiles = kp.tile0;
    pa.chunk_tiles = kp.chunk_tiles;
    pa.n_tiles = kp.n_tiles;
    pa.parts = kEW / 4;
    pa.best_key = fa.best_key;
    const size_t scan_smem = (size_t)(kScanRows * (p->dim + 1) + p->dim) * 4;
    fbc_nn_part_scan<<<(unsigned)p->scan_grid, kScanRows, scan_smem, s>>>(pa);
    fbc_nn_exact_scan<<<(unsigned)p->scan_grid, kScanRows, scan_smem, s>>>(
        stats, fa.full_list, targets, neighbors, p->nn, (int)p->dim, fa.best_key);
    fbc_nn_exact_write<<<(unsigned)((p->nt + 255) / 256), 256, 0, s>>>(stats, fa.flag_list, fa.best_key,
                                                                        fa.idx_out, dist_out);
    FBC_CUDA(cudaGetLastError());
    p->last_ws = ws;
    p->last_stream = s;
    return FBCORR_OK;
}

fbcorr_status_t fbcorr_nn_last_fallbacks(fbcorr_nn_plan_t p, int64_t* count) {
    clear_error();
    if (!p || !count) return set_error(FBCORR_ERR_INVALID_ARG, "NULL argument");
    *count = 0;
    if (!p->last_ws) return FBCORR_OK;
    FBC_CUDA(cudaStreamSynchronize(p->last_stream));
    NnStats st;
    FBC_CUDA(cudaMemcpy(&st, static_cast<const uint8_t*>(p->last_ws) + p->off_stats, sizeof st,
                        cudaMemcpyDeviceToHost));
    *count = st.flagged;
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
