// tc_kernel.cu -- filter-bank correlation on the sm_103a tensor cores
// (tcgen05.mma, accumulators in tensor memory), in BF16 or split-BF16.
//
// The correlation of Sec. 6.2 is an implicit GEMM: for every filter tap (i, j)
//   Y[m, n] += sum_d X[m + i*W + j, d] * Wt[n, i, j, d]
// where m = p*W + q runs over output pixels laid out with the INPUT width W
// (columns q >= W' are computed and discarded: (fw-1)/W extra work).  With
// that layout the A operand of every tap is a contiguous run of 128 input
// pixels, so one shared-memory "slab" of 128+fw-1 pixels per filter row i
// serves all fw taps of that row: tap j is the same slab started j rows later.
//
// Data path per CTA (persistent, one per SM, 192 threads):
//   warp 0     : producer -- cp.async.bulk (1D TMA) of A slabs and B slices of
//                `bt` consecutive taps into multi-stage rings, mbarrier complete_tx;
//   warp 1     : allocates 512 TMEM columns and issues tcgen05.mma
//                (M=128, N<=256, K=16, kind::f16 BF16 inputs, FP32 accumulate)
//                into one of two accumulators; tcgen05.commit frees ring
//                slots and hands finished accumulators to the epilogue;
//   warps 2..5 : epilogue, one warp per TMEM lane quarter -- tcgen05.ld 32x32b,
//                optional clamp, transpose
//                through shared memory, coalesced float4 streaming stores;
//                overlaps the MMAs of the next tile (double-buffered TMEM).
// Operands use the no-swizzle K-major canonical layout: a core matrix is 8
// rows x 16 bytes (8 BF16 along K), rows contiguous; LBO = byte stride between
// the two K-adjacent core matrices (one "chunk plane"), SBO = 128 bytes between
// 8-row groups.  The split pre-pass writes x and w straight into that layout.
//
// Split BF16 (FBCORR_BF16X3): v = hi + lo, hi = bf16_rn(v), lo = bf16_rn(v - hi);
// each K step issues hi*hi + hi*lo + lo*hi into the same FP32 accumulator (the
// lo*lo term, ~2^-16 relative, is dropped).
//
// Every mbarrier wait is bounded in time (%globaltimer); on expiry the kernel
// records an error code in host-mapped memory, stops every role, waits (again
// bounded) for its own copies and MMAs in flight, frees TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <new>
#include <sstream>

#include "internal.h"

namespace fbc {

namespace {

constexpr int kEpiWarps = 4;      // one epilogue warp per TMEM lane quarter (4 or 8)
constexpr int kConvWarps = 2;     // FP32 -> BF16 converters of the fused mode
constexpr int kThreads = 64 + 32 * kEpiWarps + 32 * kConvWarps;
constexpr int kTileM = 128;
constexpr int kAccCols = 256;     // TMEM columns reserved per accumulator
constexpr int kTmemCols = 512;
constexpr int kStgPitch = 36;     // floats per staged row (16-byte aligned, conflict-free)
constexpr int kStgBytes = kEpiWarps * 32 * kStgPitch * 4;
constexpr size_t kSmemMax = 227 * 1024 - 1024;   // leave room for static shared memory

enum : int { kErrWaitA = 1, kErrWaitB = 2, kErrWaitAcc = 3, kErrWaitEmpty = 4 };

struct TcParams {
    const uint8_t* xhi;   // [nc][npix_pad][16 B]
    const uint8_t* xlo;
    const uint8_t* whi;   // [ntn][taps][nc][nt][16 B]
    const uint8_t* wlo;
    float* y;             // [Ho][Wo][N]
    int* err;             // host-mapped error word
    long long npix_pad;
    unsigned long long wait_ns;
    int W, Ho, Wo, N;
    int fh, fw, nc, nt, ntn, mtiles;
    int lp;               // pixels per chunk plane of an A slot
    int split;
    int na, nb;
    int bt;               // filter taps per B stage (one wait + one commit per stage)
    uint32_t a_slot, b_stage;   // bytes per A slot / B stage (hi [+ lo])
    uint32_t a_tx, b_tx;        // bytes copied per A slot / per filter tap of a B stage
    uint32_t a_off, b_off, stg_off, bar_off;
    int epi;
    float lo, hi;
    int drop_b;           // fault injection: B load index whose copy is skipped (-1: none)
    // fused conversion of x (fuse = 1): raw FP32 slab rows are staged in nr slots
    // and turned into the BF16 hi / lo A slots by the converter warps
    const float* xraw;    // x itself [H*W][D]
    long long npix;       // H*W
    int D, fuse, nr;
    uint32_t raw_slot, raw_off;
    int alook;            // rows by which the A side runs ahead of the B stages (0 or 1)
};

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// 1D bulk copy global -> shared, completion counted on `bar` (bytes % 16 == 0).
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// K-major, no-swizzle shared-memory matrix descriptor.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------- bounded waits
struct Ctl {
    int abort;
};

__device__ __noinline__ bool wait_slow(uint32_t bar, uint32_t parity, const TcParams& P,
                                       volatile int* abort_flag, int code) {
    const unsigned long long t0 = globaltimer();
    for (;;) {
#pragma unroll 1
        for (int k = 0; k < 64; ++k)
            if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > P.wait_ns) {
            *abort_flag = 1;
            *(volatile int*)P.err = code;
            __threadfence_system();
            return false;
        }
    }
}

__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, const TcParams& P,
                                         volatile int* abort_flag, int code) {
    if (mbar_try_wait(bar, parity)) return true;
    return wait_slow(bar, parity, P, abort_flag, code);
}

// Drain wait after an abort: bounded, ignores the abort flag.
__device__ __noinline__ void wait_drain(uint32_t bar, uint32_t parity, const TcParams& P) {
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() - t0 > P.wait_ns) return;
}

// hi = bf16_rn(v), lo = bf16_rn(v - hi) for 8 values; v - hi is exact in FP32.
__device__ __forceinline__ void split8(const float (&v)[8], uint4* hi_out, uint4* lo_out, int split) {
    __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        h[k] = __float2bfloat16_rn(v[k]);
        l[k] = __float2bfloat16_rn(v[k] - __bfloat162float(h[k]));
    }
    *hi_out = *reinterpret_cast<const uint4*>(h);
    if (split) *lo_out = *reinterpret_cast<const uint4*>(l);
}

// All MMAs of one filter tap: K = 16 per instruction over the NC/2 pairs of
// chunk planes; split mode adds hi*lo and lo*hi before hi*hi.
template <int NC, int SPLIT>
__device__ __forceinline__ void issue_tap(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint64_t ak,
                                          uint64_t bk, uint64_t alo, uint64_t blo, uint32_t idesc,
                                          uint32_t& accumulate) {
#pragma unroll
    for (int kk = 0; kk < NC / 2; ++kk) {
        const uint64_t a = ad + kk * ak;
        const uint64_t b = bd + kk * bk;
        if (SPLIT) {
            // small terms first, then hi*hi
            umma_bf16(d_tmem, a, b + blo, idesc, accumulate);
            umma_bf16(d_tmem, a + alo, b, idesc, 1);
            umma_bf16(d_tmem, a, b, idesc, 1);
        } else {
            umma_bf16(d_tmem, a, b, idesc, accumulate);
        }
        accumulate = 1;
    }
}

// ---------------------------------------------------------------- the kernel
// NC = 16-byte chunk planes per pixel (D rounded up to 16, / 8); SPLIT = 3-product mode.
// Both are compile-time so that the single MMA-issuing thread runs a short,
// fully unrolled instruction chain per tap: ring indices advance incrementally
// and descriptors are advanced by adding to their start-address field.
// LF selects the shape of the issuing loop: 0 = one iteration per tap with the
// stage wait / release as branches, 1 = one iteration per B stage with an inner
// tap loop.  Both issue the same MMAs; which schedules better depends on the
// taps per stage, so the auto-tuner measures both.
template <int NC, int SPLIT, int LF>
__global__ void __launch_bounds__(kThreads, 1) fbc_tc_corr(const __grid_constant__ TcParams P) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ int s_abort;
    __shared__ uint32_t s_tmem;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t sbase = smem_u32(smem);
    // barrier table: a_full[na] a_empty[na] b_full[nb] b_empty[nb] acc_full[2] acc_empty[2] drain
    const uint32_t a_full0 = sbase + P.bar_off;
    const uint32_t a_empty0 = a_full0 + 8u * P.na;
    const uint32_t b_full0 = a_empty0 + 8u * P.na;
    const uint32_t b_empty0 = b_full0 + 8u * P.nb;
    const uint32_t acc_full0 = b_empty0 + 8u * P.nb;
    const uint32_t acc_empty0 = acc_full0 + 16u;
    const uint32_t drain_bar = acc_empty0 + 16u;
    const uint32_t raw_full0 = drain_bar + 8u;        // fused mode only: raw_full[nr] raw_empty[nr]
    const uint32_t raw_empty0 = raw_full0 + 8u * P.nr;

    if (threadIdx.x == 0) {
        for (int s = 0; s < P.na; ++s) {
            mbar_init(a_full0 + 8u * s, P.fuse ? kConvWarps : 1);
            mbar_init(a_empty0 + 8u * s, 1);
        }
        for (int s = 0; s < P.nr; ++s) {
            mbar_init(raw_full0 + 8u * s, 1);
            mbar_init(raw_empty0 + 8u * s, kConvWarps);
        }
        for (int s = 0; s < P.nb; ++s) {
            mbar_init(b_full0 + 8u * s, 1);
            mbar_init(b_empty0 + 8u * s, 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(acc_full0 + 8u * s, 1);
            mbar_init(acc_empty0 + 8u * s, kEpiWarps);
        }
        mbar_init(drain_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    volatile int* abort_flag = &s_abort;
    const int ntiles = P.mtiles * P.ntn;
    const uint32_t plane = (uint32_t)P.lp * 16u;      // bytes per A chunk plane (shared)
    const uint32_t bplane = (uint32_t)P.nt * 16u;     // bytes per B chunk plane (shared)
    const uint32_t a_half = NC * plane;               // offset of the lo planes in an A slot
    const uint32_t b_half = NC * bplane;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            uint32_t a_it = 0, b_it = 0, r_it = 0;
            int as = 0, bs = 0, rs = 0;
            uint32_t aph = 0, bph = 0, rph = 0;
            bool ok = true;
            const uint32_t a_copy = (uint32_t)(kTileM + P.fw - 1) * 16u;
            const long long tap_bytes = (long long)NC * P.nt * 16;
            // The rows of this CTA's tiles in order: row r = (tile k, filter row i).
            // The A side of row r (+ alook) is issued before the B stages of row r,
            // so a slab (or, fused, a raw row and its conversion) is in flight while
            // the MMAs of the previous row run.
            const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
            const int R = my_tiles * P.fh;
            auto issue_a = [&](int r) -> bool {
                const int tile = blockIdx.x + (r / P.fh) * gridDim.x;
                const int i = r % P.fh;
                const long long p0 = (long long)(tile % P.mtiles) * kTileM + (long long)i * P.W;
                if (P.fuse) {
                    // raw FP32 pixels [p0, p0 + 128 + fw - 1); the part past the end of
                    // x is zero-filled by the converters
                    if (!wait_bar(raw_empty0 + 8u * rs, rph ^ 1, P, abort_flag, kErrWaitEmpty)) return false;
                    const uint32_t rfull = raw_full0 + 8u * rs;
                    long long valid = P.npix - p0;
                    valid = valid < 0 ? 0 : (valid > kTileM + P.fw - 1 ? kTileM + P.fw - 1 : valid);
                    const uint32_t bytes = (uint32_t)(valid * P.D * 4);
                    mbar_expect_tx(rfull, bytes);
                    if (bytes) bulk_g2s(sbase + P.raw_off + rs * P.raw_slot, P.xraw + p0 * P.D, bytes, rfull);
                    ++r_it;
                    if (++rs == P.nr) { rs = 0; rph ^= 1; }
                } else {
                    if (!wait_bar(a_empty0 + 8u * as, aph ^ 1, P, abort_flag, kErrWaitEmpty)) return false;
                    const uint32_t afull = a_full0 + 8u * as;
                    mbar_expect_tx(afull, P.a_tx);
                    const uint32_t dst = sbase + P.a_off + as * P.a_slot;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const long long src = (c * P.npix_pad + p0) * 16;
                        bulk_g2s(dst + c * plane, P.xhi + src, a_copy, afull);
                        if (SPLIT) bulk_g2s(dst + a_half + c * plane, P.xlo + src, a_copy, afull);
                    }
                    ++a_it;
                    if (++as == P.na) { as = 0; aph ^= 1; }
                }
                return true;
            };
            auto issue_b_row = [&](int r) -> bool {
                const int tile = blockIdx.x + (r / P.fh) * gridDim.x;
                const int i = r % P.fh;
                const long long woff = (((long long)(tile / P.mtiles) * P.fh + i) * P.fw) * tap_bytes;
                const uint8_t* wtap_hi = P.whi + woff;
                const uint8_t* wtap_lo = P.wlo + woff;
                for (int j0 = 0; j0 < P.fw; j0 += P.bt) {
                    // taps j0 .. j0+tcnt-1 of this filter row are contiguous in the
                    // operand layout: one copy per half for the whole stage
                    const int tcnt = min(P.bt, P.fw - j0);
                    if (!wait_bar(b_empty0 + 8u * bs, bph ^ 1, P, abort_flag, kErrWaitEmpty)) return false;
                    const uint32_t bfull = b_full0 + 8u * bs;
                    const uint32_t bytes = (uint32_t)tcnt * b_half;
                    mbar_expect_tx(bfull, SPLIT ? 2u * bytes : bytes);
                    if ((int)b_it != P.drop_b) {
                        const uint32_t bdst = sbase + P.b_off + bs * P.b_stage;
                        bulk_g2s(bdst, wtap_hi, bytes, bfull);
                        if (SPLIT) bulk_g2s(bdst + (uint32_t)P.bt * b_half, wtap_lo, bytes, bfull);
                    }
                    wtap_hi += tcnt * tap_bytes;
                    wtap_lo += tcnt * tap_bytes;
                    ++b_it;
                    if (++bs == P.nb) { bs = 0; bph ^= 1; }
                }
                return true;
            };
            int next_a = 0;
            for (int r = 0; r < R && ok; ++r) {
                while (ok && next_a < R && next_a <= r + P.alook) ok = issue_a(next_a++);
                if (ok) ok = issue_b_row(r);
            }
            if (!ok) {
                // wait (bounded) for the copies still in flight into each ring slot
                const uint32_t a0 = a_it > (uint32_t)P.na ? a_it - P.na : 0;
                for (uint32_t k = a0; k < a_it; ++k) wait_drain(a_full0 + 8u * (k % P.na), (k / P.na) & 1, P);
                const uint32_t b0 = b_it > (uint32_t)P.nb ? b_it - P.nb : 0;
                for (uint32_t k = b0; k < b_it; ++k) wait_drain(b_full0 + 8u * (k % P.nb), (k / P.nb) & 1, P);
                const uint32_t r0 = r_it > (uint32_t)P.nr ? r_it - P.nr : 0;
                for (uint32_t k = r0; k < r_it; ++k) wait_drain(raw_full0 + 8u * (k % P.nr), (k / P.nr) & 1, P);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = (1u << 4)                          // D: FP32
                                   | (1u << 7) | (1u << 10)           // A, B: BF16
                                   | ((uint32_t)(P.nt >> 3) << 17)    // N
                                   | ((uint32_t)(kTileM >> 4) << 24); // M
            // descriptor arithmetic: the start address sits in the low 14 bits as
            // (addr >> 4); every shared address is < 2^18, so adding (offset >> 4)
            // to the descriptor never carries out of that field
            const uint64_t adesc0 = smem_desc(sbase + P.a_off, plane, 128);
            const uint64_t bdesc0 = smem_desc(sbase + P.b_off, bplane, 128);
            const uint64_t a_step = P.a_slot >> 4, b_step = P.b_stage >> 4;
            const uint64_t ak = (2 * plane) >> 4, bk = (2 * bplane) >> 4;
            const uint64_t alo = a_half >> 4, blo = ((uint64_t)P.bt * b_half) >> 4;
            const uint64_t btap = b_half >> 4;   // next tap inside a stage
            int as = 0, bs = 0;
            uint32_t aph = 0, bph = 0, acc_it = 0;
            uint64_t adesc = adesc0, bdesc = bdesc0;
            bool ok = true;
            bool issued = false;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                const int acc = acc_it & 1;
                if (!(ok = wait_bar(acc_empty0 + 8u * acc, ((acc_it >> 1) & 1) ^ 1, P, abort_flag, kErrWaitAcc)))
                    break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(acc * kAccCols);
                uint32_t accumulate = 0;
                for (int i = 0; i < P.fh && ok; ++i) {
                    if (!(ok = wait_bar(a_full0 + 8u * as, aph, P, abort_flag, kErrWaitA))) break;
                    if (LF == 0) {
                        // one iteration per tap; a B stage holds bt consecutive taps:
                        // wait for it at its first tap, release it after its last
                        int t = 0;
                        for (int j = 0; j < P.fw; ++j) {
                            if (t == 0 && !(ok = wait_bar(b_full0 + 8u * bs, bph, P, abort_flag, kErrWaitB)))
                                break;
                            issue_tap<NC, SPLIT>(d_tmem, adesc + (uint64_t)j, bdesc + (uint64_t)t * btap, ak, bk,
                                                 alo, blo, idesc, accumulate);
                            issued = true;
                            if (++t == P.bt || j == P.fw - 1) {
                                umma_commit(b_empty0 + 8u * bs);
                                if (++bs == P.nb) { bs = 0; bph ^= 1; bdesc = bdesc0; } else { bdesc += b_step; }
                                t = 0;
                            }
                        }
                    } else {
                        // one iteration per B stage, inner loop over its taps
                        for (int j0 = 0; j0 < P.fw; j0 += P.bt) {
                            const int tcnt = min(P.bt, P.fw - j0);
                            if (!(ok = wait_bar(b_full0 + 8u * bs, bph, P, abort_flag, kErrWaitB))) break;
                            for (int t = 0; t < tcnt; ++t)
                                issue_tap<NC, SPLIT>(d_tmem, adesc + (uint64_t)(j0 + t), bdesc + (uint64_t)t * btap,
                                                     ak, bk, alo, blo, idesc, accumulate);
                            issued = true;
                            umma_commit(b_empty0 + 8u * bs);
                            if (++bs == P.nb) { bs = 0; bph ^= 1; bdesc = bdesc0; } else { bdesc += b_step; }
                        }
                    }
                    if (!ok) break;
                    umma_commit(a_empty0 + 8u * as);
                    if (++as == P.na) { as = 0; aph ^= 1; adesc = adesc0; } else { adesc += a_step; }
                }
                if (!ok) break;
                umma_commit(acc_full0 + 8u * acc);
                ++acc_it;
            }
            if (!ok && issued) {
                umma_commit(drain_bar);
                wait_drain(drain_bar, 0, P);
            }
        }
    } else if (warp >= 2 + kEpiWarps) {
        // ------------------------------------------------------------ converters (fused mode)
        // FP32 slab row -> BF16 hi (and lo) chunk planes of an A slot.  Generic-proxy
        // shared-memory writes are made visible to the tensor core's async proxy by
        // fence.proxy.async before the arrival on a_full.
        if (P.fuse) {
            const int ct = threadIdx.x - (2 + kEpiWarps) * 32;
            constexpr int NCT = kConvWarps * 32;
            const int L = kTileM + P.fw - 1;
            int as = 0, rs = 0;
            uint32_t aph = 0, rph = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                const int mt = tile % P.mtiles;
                for (int i = 0; i < P.fh && ok; ++i) {
                    if (!(ok = wait_bar(raw_full0 + 8u * rs, rph, P, abort_flag, kErrWaitA))) break;
                    if (!(ok = wait_bar(a_empty0 + 8u * as, aph ^ 1, P, abort_flag, kErrWaitEmpty))) break;
                    const long long p0 = (long long)mt * kTileM + (long long)i * P.W;
                    long long vl = P.npix - p0;
                    const int valid = (int)(vl < 0 ? 0 : (vl > L ? L : vl));
                    const float* raw = reinterpret_cast<const float*>(smem + P.raw_off + rs * P.raw_slot);
                    uint8_t* dst = smem + P.a_off + as * P.a_slot;
                    const bool vec = (P.D & 7) == 0;
                    for (int item = ct; item < L * NC; item += NCT) {
                        const int px = item / NC;
                        const int c = item - px * NC;
                        float v[8];
                        if (px < valid && vec && c * 8 + 8 <= P.D) {
                            const float4* r4 = reinterpret_cast<const float4*>(raw + px * P.D + c * 8);
                            const float4 a = r4[0], b = r4[1];
                            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
                            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
                        } else {
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const int d = c * 8 + k;
                                v[k] = (px < valid && d < P.D) ? raw[px * P.D + d] : 0.f;
                            }
                        }
                        split8(v, reinterpret_cast<uint4*>(dst + c * plane + px * 16),
                               reinterpret_cast<uint4*>(dst + a_half + c * plane + px * 16), SPLIT);
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive(a_full0 + 8u * as);
                        mbar_arrive(raw_empty0 + 8u * rs);
                    }
                    if (++as == P.na) { as = 0; aph ^= 1; }
                    if (++rs == P.nr) { rs = 0; rph ^= 1; }
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - 2;         // staging buffer
        const int lq = warp & 3;         // TMEM lane quarter this warp may access
        const int part = ew >> 2;        // with 8 epilogue warps: even / odd chunks of this quarter
        float* stg = reinterpret_cast<float*>(smem + P.stg_off) + ew * 32 * kStgPitch;
        uint32_t acc_it = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int mt = tile % P.mtiles;
            const int nti = tile / P.mtiles;
            const int acc = acc_it & 1;
            if (!wait_bar(acc_full0 + 8u * acc, (acc_it >> 1) & 1, P, abort_flag, kErrWaitAcc)) break;
            tc_fence_after();
            // output offsets of the 8 rows this lane stores (row = it*4 + lane/8)
            int obase[8];
            const int mrow0 = mt * kTileM + lq * 32;
#pragma unroll
            for (int it = 0; it < 8; ++it) {
                const int m = mrow0 + it * 4 + (lane >> 3);
                const int p = m / P.W;
                const int q = m - p * P.W;
                obase[it] = (p < P.Ho && q < P.Wo) ? (p * P.Wo + q) * P.N : -1;
            }
            const int ncol = (P.nt + 31) / 32;   // a 16-wide tile still loads one 32-column chunk
            for (int cc = part; cc < ncol; cc += kEpiWarps / 4) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(acc * kAccCols + cc * 32), r);
                float4* srow = reinterpret_cast<float4*>(stg + lane * kStgPitch);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    float4 v = make_float4(__uint_as_float(r[4 * k]), __uint_as_float(r[4 * k + 1]),
                                           __uint_as_float(r[4 * k + 2]), __uint_as_float(r[4 * k + 3]));
                    if (P.epi == 1) {
                        v.x = fminf(fmaxf(v.x, P.lo), P.hi);
                        v.y = fminf(fmaxf(v.y, P.lo), P.hi);
                        v.z = fminf(fmaxf(v.z, P.lo), P.hi);
                        v.w = fminf(fmaxf(v.w, P.lo), P.hi);
                    }
                    srow[k] = v;
                }
                __syncwarp();
                // columns past this tile's last filter (nt is a multiple of 16, the
                // chunk 32 wide) hold no result: stop at the tile end as well as N
                const int nend = min(P.N, (nti + 1) * P.nt);
                const int n0 = nti * P.nt + cc * 32 + (lane & 7) * 4;
                const bool vec = ((P.N & 3) == 0) && (n0 + 4 <= nend);
#pragma unroll
                for (int it = 0; it < 8; ++it) {
                    const int row = it * 4 + (lane >> 3);
                    if (obase[it] < 0 || n0 >= nend) continue;
                    const float4 v = *reinterpret_cast<const float4*>(stg + row * kStgPitch + (lane & 7) * 4);
                    float* dst = P.y + (long long)obase[it] + n0;
                    if (vec) {
                        __stcs(reinterpret_cast<float4*>(dst), v);
                    } else {
                        const float vv[4] = {v.x, v.y, v.z, v.w};
                        for (int e = 0; e < 4; ++e)
                            if (n0 + e < nend) dst[e] = vv[e];
                    }
                }
                __syncwarp();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty0 + 8u * acc);
            ++acc_it;
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// ---------------------------------------------------------------- split pre-pass
// Blocks [0, xblocks) convert x, the rest convert w, into the BF16 chunk-plane
// layouts read by fbc_tc_corr (zero padding for channels >= D, pixels >= H*W,
// filters >= N).  hi = bf16_rn(v); lo = bf16_rn(v - hi) (v - hi is exact in FP32).
struct SplitParams {
    const float* x;
    const float* w;
    uint8_t* xhi;
    uint8_t* xlo;
    uint8_t* whi;
    uint8_t* wlo;
    long long npix, npix_pad;
    int D, nc, N, fh, fw, nt, ntn, split;
    long long xblocks;
};


__global__ void __launch_bounds__(256) fbc_tc_split(const __grid_constant__ SplitParams S) {
    if ((long long)blockIdx.x < S.xblocks) {
        // one thread per pixel: contiguous reads of its D channels, and for
        // every chunk plane a 16-byte store that is contiguous across the warp
        const long long pix = (long long)blockIdx.x * 256 + threadIdx.x;
        if (pix >= S.npix_pad) return;
        const bool inside = pix < S.npix;
        const float* src = S.x + pix * S.D;
        // all loads first (up to 8 planes, 64 registers), then convert and store,
        // so the loads of one pixel are in flight together
        float v[8][8];
        const bool vec = inside && (S.D & 7) == 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (c < S.nc) {
                if (vec && c * 8 + 8 <= S.D) {
                    const float4* s4 = reinterpret_cast<const float4*>(src + c * 8);
                    const float4 a = __ldg(s4), b = __ldg(s4 + 1);
                    v[c][0] = a.x; v[c][1] = a.y; v[c][2] = a.z; v[c][3] = a.w;
                    v[c][4] = b.x; v[c][5] = b.y; v[c][6] = b.z; v[c][7] = b.w;
                } else {
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int d = c * 8 + k;
                        v[c][k] = (inside && d < S.D) ? __ldg(src + d) : 0.f;
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (c < S.nc) {
                const long long idx = (long long)c * S.npix_pad + pix;
                split8(v[c], reinterpret_cast<uint4*>(S.xhi) + idx, reinterpret_cast<uint4*>(S.xlo) + idx,
                       S.split);
            }
        }
    } else {
        const long long idx = ((long long)blockIdx.x - S.xblocks) * 256 + threadIdx.x;
        const int taps = S.fh * S.fw;
        const long long total = (long long)S.ntn * taps * S.nc * S.nt;
        if (idx >= total) return;
        const int nl = (int)(idx % S.nt);
        long long t = idx / S.nt;
        const int c = (int)(t % S.nc);
        t /= S.nc;
        const int tap = (int)(t % taps);
        const int nti = (int)(t / taps);
        const int n = nti * S.nt + nl;
        const int i = tap / S.fw, j = tap % S.fw;
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int d = c * 8 + k;
            v[k] = (n < S.N && d < S.D) ? __ldg(S.w + (((long long)n * S.fh + i) * S.fw + j) * S.D + d) : 0.f;
        }
        split8(v, reinterpret_cast<uint4*>(S.whi) + idx, reinterpret_cast<uint4*>(S.wlo) + idx, S.split);
    }
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

typedef void (*TcKernelFn)(const TcParams);

template <int LF>
TcKernelFn tc_kernel_lf(int nc, int split) {
    switch (nc * 2 + (split ? 1 : 0)) {
        case 4: return fbc_tc_corr<2, 0, LF>;
        case 5: return fbc_tc_corr<2, 1, LF>;
        case 8: return fbc_tc_corr<4, 0, LF>;
        case 9: return fbc_tc_corr<4, 1, LF>;
        case 12: return fbc_tc_corr<6, 0, LF>;
        case 13: return fbc_tc_corr<6, 1, LF>;
        case 16: return fbc_tc_corr<8, 0, LF>;
        case 17: return fbc_tc_corr<8, 1, LF>;
    }
    return nullptr;
}

TcKernelFn tc_kernel_for(int nc, int split, int lf) {
    return lf ? tc_kernel_lf<1>(nc, split) : tc_kernel_lf<0>(nc, split);
}

}  // namespace

struct TcConfig {
    int na = 2, nb = 5, ntmax = 256;   // A slots, B stages, widest filter tile
    int bt = 1;                        // filter taps per B stage
    int lf = 0;                        // issuing-loop form (see fbc_tc_corr)
    int fuse = 0;                      // convert x inside the kernel (no x pre-pass)
};

struct TcPlan {
    TcParams kp;          // pointers filled per call
    SplitParams sp;
    TcConfig cfg;
    size_t smem = 0;
    size_t ws_bytes = 0;  // the largest any candidate configuration needs
    size_t off_xhi = 0, off_xlo = 0, off_whi = 0, off_wlo = 0;
    int grid = 0;
    int split_blocks = 0;
    int H = 0, W = 0, D = 0, N = 0, fh = 0, fw = 0, split = 0, epi = 0;
    float lo = 0.f, hi = 0.f;
    int sm_count = 1;
    unsigned long long wait_ns = 0;
    int drop_b = -1;
    TcKernelFn kfn = nullptr;
};

namespace {

// Filter-tile width for a widest tile of `ntmax` columns: equal tiles, multiples of 16.
void filter_tiles(int N, int ntmax, int* nt, int* ntn) {
    const int npad = (N + 15) / 16 * 16;
    *ntn = (npad + ntmax - 1) / ntmax;
    *nt = ((npad + *ntn - 1) / *ntn + 15) / 16 * 16;
}

// Lay out shared memory, pipeline depths and the workspace for one configuration.
bool tc_layout(TcPlan* p, const TcConfig& c, bool commit) {
    const int Dp = (p->D + 15) / 16 * 16;
    const int nc = Dp / 8;
    const int Ho = p->H - p->fh + 1, Wo = p->W - p->fw + 1;
    int nt, ntn;
    filter_tiles(p->N, c.ntmax, &nt, &ntn);
    const long long mvirt = (long long)Ho * p->W;
    const int mtiles = (int)((mvirt + kTileM - 1) / kTileM);
    const int lp = (kTileM + p->fw - 1 + 7) / 8 * 8;
    const int halves = p->split ? 2 : 1;
    const uint32_t a_slot = (uint32_t)align_up((size_t)nc * lp * 16 * halves, 128);
    if (c.bt < 1 || c.bt > p->fw) return false;
    if (c.fuse && (p->D % 4) != 0) return false;   // raw rows are copied in 16-byte units
    const int L = kTileM + p->fw - 1;
    const int nr = c.fuse ? 2 : 0;
    const uint32_t raw_slot = c.fuse ? (uint32_t)align_up((size_t)L * p->D * 4, 128) : 0;
    const uint32_t b_stage = (uint32_t)align_up((size_t)c.bt * nc * nt * 16 * halves, 128);
    if (c.na < 2 || c.nb < 2) return false;
    const size_t need = (size_t)c.na * a_slot + (size_t)c.nb * b_stage + kStgBytes + (size_t)nr * raw_slot + 512;
    if (need > kSmemMax) return false;
    if (!commit) return true;
    p->cfg = c;
    TcParams& k = p->kp;
    k = TcParams{};
    k.npix_pad = (long long)align_up((size_t)p->H * p->W + kTileM + p->fw + 8, 8);
    k.W = p->W; k.Ho = Ho; k.Wo = Wo; k.N = p->N;
    k.fh = p->fh; k.fw = p->fw; k.nc = nc; k.nt = nt; k.ntn = ntn; k.mtiles = mtiles;
    k.lp = lp; k.split = p->split; k.na = c.na; k.nb = c.nb; k.bt = c.bt;
    k.a_slot = a_slot; k.b_stage = b_stage;
    k.a_tx = (uint32_t)(nc * (kTileM + p->fw - 1) * 16 * halves);
    k.b_tx = (uint32_t)(nc * nt * 16 * halves);
    k.a_off = 0;
    k.b_off = (uint32_t)(c.na * a_slot);
    k.stg_off = (uint32_t)(k.b_off + c.nb * b_stage);
    k.raw_off = (uint32_t)(k.stg_off + kStgBytes);
    k.raw_slot = raw_slot;
    k.nr = nr;
    k.fuse = c.fuse;
    k.npix = (long long)p->H * p->W;
    k.D = p->D;
    // A-side look-ahead needs a free slot beyond the one the MMAs of the previous
    // row still read: the raw ring (fused), or three A slots
    k.alook = (c.fuse || c.na >= 3) ? 1 : 0;
    k.bar_off = (uint32_t)(k.raw_off + (size_t)nr * raw_slot);
    k.epi = p->epi; k.lo = p->lo; k.hi = p->hi;
    k.wait_ns = p->wait_ns;
    k.drop_b = p->drop_b;
    p->smem = k.bar_off + 512;

    const size_t xplanes = (size_t)nc * k.npix_pad * 16;
    const size_t wplanes = (size_t)ntn * p->fh * p->fw * nc * nt * 16;
    size_t off = 0;
    p->off_xhi = off; off = align_up(off + xplanes, 256);
    p->off_xlo = off; if (p->split) off = align_up(off + xplanes, 256);
    p->off_whi = off; off = align_up(off + wplanes, 256);
    p->off_wlo = off; if (p->split) off = align_up(off + wplanes, 256);

    SplitParams& sp = p->sp;
    sp = SplitParams{};
    sp.npix = (long long)p->H * p->W;
    sp.npix_pad = k.npix_pad;
    sp.D = p->D; sp.nc = nc; sp.N = p->N; sp.fh = p->fh; sp.fw = p->fw; sp.nt = nt; sp.ntn = ntn;
    sp.split = p->split;
    sp.xblocks = (k.npix_pad + 255) / 256;
    const long long wblocks = ((long long)ntn * p->fh * p->fw * nc * nt + 255) / 256;
    if (c.fuse) sp.xblocks = 0;   // x is converted inside the correlation kernel
    p->split_blocks = (int)(sp.xblocks + wblocks);
    p->grid = std::min(mtiles * ntn, std::max(1, p->sm_count));
    p->kfn = tc_kernel_for(nc, p->split, c.lf);
    return true;
}

size_t tc_ws_need(TcPlan* p, const TcConfig& c) {
    TcPlan tmp = *p;
    if (!tc_layout(&tmp, c, true)) return 0;
    const size_t wplanes = (size_t)tmp.kp.ntn * p->fh * p->fw * tmp.kp.nc * tmp.kp.nt * 16;
    return align_up(tmp.off_wlo + (p->split ? wplanes : 0), 256);
}

std::vector<TcConfig> tc_candidate_configs(TcPlan* p) {
    // widest filter tile first; within it, taps per stage from the most (fewest
    // barrier handoffs) down, each with the deepest B ring that fits
    std::vector<TcConfig> out;
    const int widths[] = {256, 128};
    for (int ntmax : widths) {
        if (ntmax == 128 && p->N <= 128) continue;
        for (int fuse = (p->D % 4 == 0) ? 1 : 0; fuse >= 0; --fuse)
            for (int bt = std::min(p->fw, 5); bt >= 1; --bt)
                for (int na = 2; na <= 3; ++na) {
                    int best = 0;
                    for (int nb = 2; nb <= 10; ++nb)
                        if (tc_layout(p, TcConfig{na, nb, ntmax, bt, 0, fuse}, false)) best = nb;
                    if (!best) continue;
                    out.push_back(TcConfig{na, best, ntmax, bt, 0, fuse});
                    if (bt > 1) out.push_back(TcConfig{na, best, ntmax, bt, 1, fuse});
                }
    }
    return out;
}

bool parse_tc_spec(const std::string& s, TcConfig* c) {
    TcConfig t;
    const int n = sscanf(s.c_str(), "tcgen05:na=%d,nb=%d,nt=%d,bt=%d,lf=%d,fz=%d", &t.na, &t.nb,
                         &t.ntmax, &t.bt, &t.lf, &t.fuse);
    if (n == 3) t.bt = 1;
    if (n <= 4) t.lf = 0;
    if (n <= 5) t.fuse = 0;
    if (n < 3 || t.lf < 0 || t.lf > 1 || t.fuse < 0 || t.fuse > 1) return false;
    if (t.ntmax != 256 && t.ntmax != 128 && t.ntmax != 64) return false;
    *c = t;
    return true;
}

}  // namespace

std::string tc_spec(const TcPlan* p) {
    char b[96];
    snprintf(b, sizeof b, "tcgen05:na=%d,nb=%d,nt=%d,bt=%d,lf=%d,fz=%d", p->cfg.na, p->cfg.nb,
             p->cfg.ntmax, p->cfg.bt, p->cfg.lf, p->cfg.fuse);
    return b;
}

std::vector<std::string> tc_candidates(TcPlan* p) {
    std::vector<std::string> out;
    for (const auto& c : tc_candidate_configs(p)) {
        char b[96];
        snprintf(b, sizeof b, "tcgen05:na=%d,nb=%d,nt=%d,bt=%d,lf=%d,fz=%d", c.na, c.nb, c.ntmax, c.bt,
                 c.lf, c.fuse);
        out.push_back(b);
    }
    return out;
}

fbcorr_status_t tc_set_spec(TcPlan* p, const std::string& spec) {
    TcConfig c;
    if (!parse_tc_spec(spec, &c)) return set_error(FBCORR_ERR_INVALID_ARG, "unknown tcgen05 spec '%s'", spec.c_str());
    if (!tc_layout(p, c, false) || tc_ws_need(p, c) > p->ws_bytes)
        return set_error(FBCORR_ERR_UNSUPPORTED, "tcgen05 spec '%s' does not fit this shape", spec.c_str());
    tc_layout(p, c, true);
    return FBCORR_OK;
}

fbcorr_status_t tc_plan_create(TcPlan** out, int H, int W, int D, int N, int fh, int fw, int split,
                               int epi, float lo, float hi, const DeviceInfo& dev) {
    *out = nullptr;
    if ((D + 15) / 16 * 16 / 8 > 8)
        return set_error(FBCORR_ERR_UNSUPPORTED,
                         "tensor-core modes support depth D <= 64 (got %d); use FBCORR_F32", D);
    TcPlan* p = new (std::nothrow) TcPlan();
    if (!p) return set_error(FBCORR_ERR_OOM, "host allocation failed");
    p->H = H; p->W = W; p->D = D; p->N = N; p->fh = fh; p->fw = fw;
    p->split = split; p->epi = epi; p->lo = lo; p->hi = hi;
    p->sm_count = dev.sm_count;
    const long long wait_ms = atoll(env_str("FBCORR_WAIT_MS", "4000").c_str());
    p->wait_ns = (unsigned long long)std::max(1LL, wait_ms) * 1000000ull;
    p->drop_b = fault_injected("tcdrop") ? 0 : -1;   // the first B stage: every CTA has one
    const std::vector<TcConfig> cands = tc_candidate_configs(p);
    if (cands.empty()) {
        delete p;
        return set_error(FBCORR_ERR_UNSUPPORTED, "shape needs more shared memory than one SM has");
    }
    for (const auto& c : cands) p->ws_bytes = std::max(p->ws_bytes, tc_ws_need(p, c));
    // default: the fewest A slots (2) with the deepest B ring, widest filter tile
    tc_layout(p, cands.front(), true);
    // one attribute for every plan: the largest dynamic shared memory any plan uses
    cudaError_t e = cudaSuccess;
    for (int lf = 0; lf <= 1 && e == cudaSuccess; ++lf) {
        TcKernelFn f = tc_kernel_for(p->kp.nc, p->split, lf);
        e = f ? cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSmemMax)
              : cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) {
        delete p;
        return set_error(FBCORR_ERR_CUDA, "cudaFuncSetAttribute(tc smem): %s", cudaGetErrorString(e));
    }
    logf("tc plan: nc=%d nt=%d ntn=%d mtiles=%d lp=%d na=%d nb=%d smem=%zu ws=%zu grid=%d", p->kp.nc,
         p->kp.nt, p->kp.ntn, p->kp.mtiles, p->kp.lp, p->kp.na, p->kp.nb, p->smem, p->ws_bytes, p->grid);
    *out = p;
    return FBCORR_OK;
}

void tc_plan_destroy(TcPlan* p) { delete p; }

size_t tc_workspace_bytes(const TcPlan* p) { return p->ws_bytes; }

int tc_launches(const TcPlan*) { return 2; }

std::string tc_describe(const TcPlan* p) {
    std::ostringstream o;
    o << "{\"precision\":\"" << (p->kp.split ? "bf16x3" : "bf16") << "\",\"mma\":\"128x" << p->kp.nt
      << "x16\",\"filter_tiles\":" << p->kp.ntn << ",\"tiles\":" << p->kp.mtiles * p->kp.ntn
      << ",\"smem\":" << p->smem << ",\"grid\":" << p->grid << "}";
    return o.str();
}

fbcorr_status_t tc_forward(TcPlan* p, const float* x, const float* w, float* y, void* ws,
                           int* err_word, cudaStream_t s, cudaEvent_t ev_start, cudaEvent_t ev_stop) {
    uint8_t* base = static_cast<uint8_t*>(ws);
    SplitParams sp = p->sp;
    sp.x = x;
    sp.w = w;
    sp.xhi = base + p->off_xhi;
    sp.xlo = base + p->off_xlo;
    sp.whi = base + p->off_whi;
    sp.wlo = base + p->off_wlo;
    fbc_tc_split<<<p->split_blocks, 256, 0, s>>>(sp);
    FBC_CUDA(cudaGetLastError());
    TcParams kp = p->kp;
    kp.xhi = sp.xhi;
    kp.xlo = sp.xlo;
    kp.whi = sp.whi;
    kp.wlo = sp.wlo;
    kp.y = y;
    kp.err = err_word;
    kp.xraw = x;
    if (ev_start) FBC_CUDA(cudaEventRecord(ev_start, s));
    void* args[] = {&kp};
    FBC_CUDA(cudaLaunchKernel((const void*)p->kfn, dim3(p->grid), dim3(kThreads), args, p->smem, s));
    if (ev_stop) FBC_CUDA(cudaEventRecord(ev_stop, s));
    return FBCORR_OK;
}

}  // namespace fbc
