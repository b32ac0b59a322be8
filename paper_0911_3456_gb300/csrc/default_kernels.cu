// default_kernels.cu -- prebuilt (nvcc) kernels that need no code generation.
//
//  * fbc_default_direct: the generic "default" correlation kernel.  The paper
//    compares its auto-tuned kernels with a hand-written default that runs
//    correctly for every input range (Sec. 6.2, Table "Performance of RTCG
//    auto-tuning on 3D filter-bank convolutions", column "Default").  This one
//    takes every size at run time, so it serves any shape without NVRTC; it is
//    the baseline of the Boost report and the fallback when code generation
//    fails.  Thread = 4 output rows x 8 output channels at one column; input
//    values come through the read-only cache, filter values are warp-uniform
//    (broadcast) loads.
//  * fbc_default_dw: generic per-chunk partial sums of dL/dw (one thread per
//    filter element and chunk of output rows).
//  * fbc_dw_reduce: the deterministic second stage of dL/dw: for every filter
//    element, a fixed-order pairwise sum over the chunk partials (trees over
//    groups of 8 in registers, then over the group sums in shared memory).
#include "internal.h"

namespace fbc {

namespace {

constexpr int kDefTR = 4;   // output rows per thread
constexpr int kDefTF = 8;   // output channels per thread

__global__ void __launch_bounds__(256) fbc_default_direct(DirectArgsRT a) {
    const int q = blockIdx.x * 32 + (threadIdx.x & 31);
    const int p0 = (blockIdx.y * 8 + (threadIdx.x >> 5)) * kDefTR;
    const int n0 = blockIdx.z * kDefTF;
    float acc[kDefTR][kDefTF];
#pragma unroll
    for (int r = 0; r < kDefTR; ++r)
#pragma unroll
        for (int f = 0; f < kDefTF; ++f) acc[r][f] = 0.f;
    if (q < a.out_w && p0 < a.out_h) {
        for (int i = 0; i < a.fh; ++i)
            for (int j = 0; j < a.fw; ++j) {
                const int gx = q - a.pad_x + j;
                const bool xin = gx >= 0 && gx < a.in_w;
                for (int c = 0; c < a.c; ++c) {
                    float wv[kDefTF];
#pragma unroll
                    for (int f = 0; f < kDefTF; ++f) {
                        const int n = n0 + f;
                        float v = 0.f;
                        if (n < a.nf) {
                            const long long off =
                                a.flip ? (((long long)c * a.fh + (a.fh - 1 - i)) * a.fw + (a.fw - 1 - j)) * a.nf + n
                                       : (((long long)n * a.fh + i) * a.fw + j) * a.c + c;
                            v = __ldg(a.w + off);
                        }
                        wv[f] = v;
                    }
#pragma unroll
                    for (int r = 0; r < kDefTR; ++r) {
                        const int gy = p0 + r - a.pad_y + i;
                        float xv = 0.f;
                        if (xin && gy >= 0 && gy < a.in_h) {
                            const long long off = ((long long)gy * a.in_w + gx) * a.c + c;
                            xv = __ldg(a.x + off);
                            if (a.mask) {
                                const float mv = __ldg(a.m + off);
                                if (!(mv > a.lo && mv < a.hi)) xv = 0.f;
                            }
                        }
#pragma unroll
                        for (int f = 0; f < kDefTF; ++f) acc[r][f] = fmaf(xv, wv[f], acc[r][f]);
                    }
                }
            }
    }
    if (q >= a.out_w) return;
#pragma unroll
    for (int r = 0; r < kDefTR; ++r) {
        const int p = p0 + r;
        if (p >= a.out_h) continue;
        float* yp = a.y + ((long long)p * a.out_w + q) * a.nf;
#pragma unroll
        for (int f = 0; f < kDefTF; ++f) {
            const int n = n0 + f;
            if (n >= a.nf) continue;
            float v = acc[r][f];
            if (a.epi == 1) v = fminf(fmaxf(v, a.lo), a.hi);
            yp[n] = v;
        }
    }
}

__global__ void __launch_bounds__(256) fbc_default_dw(const float* __restrict__ x,
                                                      const float* __restrict__ g,
                                                      const float* __restrict__ m,
                                                      float* __restrict__ part, int H, int W, int C,
                                                      int Ho, int Wo, int N, int fh, int fw,
                                                      int rows_per_chunk, int mask, float lo,
                                                      float hi) {
    const long long E = (long long)N * fh * fw * C;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    if (e >= E) return;
    const int c = (int)(e % C);
    const int j = (int)((e / C) % fw);
    const int i = (int)((e / ((long long)C * fw)) % fh);
    const int n = (int)(e / ((long long)C * fw * fh));
    const int pb = chunk * rows_per_chunk;
    const int pe = min(pb + rows_per_chunk, Ho);
    float tot = 0.f;
    for (int p = pb; p < pe; ++p) {
        float row = 0.f;
        const float* xr = x + ((long long)(p + i) * W + j) * C + c;
        const float* gr = g + (long long)p * Wo * N + n;
        for (int q = 0; q < Wo; ++q) {
            float gv = __ldg(gr + (long long)q * N);
            if (mask) {
                const float mv = __ldg(m + (long long)p * Wo * N + (long long)q * N + n);
                if (!(mv > lo && mv < hi)) gv = 0.f;
            }
            row = fmaf(gv, __ldg(xr + (long long)q * C), row);
        }
        tot += row;
    }
    part[(long long)chunk * E + e] = tot;
}

constexpr int kRedElems = 128;    // filter elements per block
constexpr int kRedSlices = 4;     // threads per element, each summing every kRedSlices-th group
constexpr int kMaxChunks = 256;   // the plan keeps the chunk count at or below this

// Fixed-order pairwise sum over the S chunk partials of every filter element e:
// groups of 8 consecutive partials are summed as a balanced tree in registers
// (8 independent loads in flight per thread; kRedSlices threads per element take
// the groups in turn), the group sums (the last group padded with zeros) are kept
// in shared memory, one column per element, and added by a balanced tree over
// the groups.  No dynamically indexed register arrays.
__global__ void __launch_bounds__(kRedElems * kRedSlices) fbc_dw_reduce(const float* __restrict__ part,
                                                                        float* __restrict__ dw, int S,
                                                                        long long E) {
    extern __shared__ float gsum[];   // [ceil(S / 8)][kRedElems]
    // launched as the programmatic dependent of the partial-sum kernel: wait for
    // that grid to complete and its partials to be visible before reading them
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int el = threadIdx.x % kRedElems;
    const int slice = threadIdx.x / kRedElems;
    const long long e = (long long)blockIdx.x * kRedElems + el;
    const bool valid = e < E;
    const int G = (S + 7) / 8;
    for (int gi = slice; gi < G; gi += kRedSlices) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int sidx = gi * 8 + k;
            v[k] = (valid && sidx < S) ? __ldg(part + (long long)sidx * E + e) : 0.f;
        }
        gsum[gi * kRedElems + el] = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    }
    __syncthreads();
    if (slice != 0) return;
    for (int step = 1; step < G; step *= 2)
        for (int g = 0; g + step < G; g += 2 * step) gsum[g * kRedElems + el] += gsum[(g + step) * kRedElems + el];
    if (valid) dw[e] = gsum[el];
}

}  // namespace

cudaError_t launch_default_direct(const DirectArgsRT& a, cudaStream_t s) {
    dim3 grid((a.out_w + 31) / 32, (a.out_h + 8 * kDefTR - 1) / (8 * kDefTR),
              (a.nf + kDefTF - 1) / kDefTF);
    fbc_default_direct<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_default_dw(const float* x, const float* g, const float* m, float* part, int H,
                              int W, int C, int Ho, int Wo, int N, int fh, int fw, int chunks,
                              int rows_per_chunk, int mask, float lo, float hi, cudaStream_t s) {
    const long long E = (long long)N * fh * fw * C;
    dim3 grid((unsigned)((E + 255) / 256), (unsigned)chunks);
    fbc_default_dw<<<grid, 256, 0, s>>>(x, g, m, part, H, W, C, Ho, Wo, N, fh, fw, rows_per_chunk,
                                        mask, lo, hi);
    return cudaGetLastError();
}

cudaError_t launch_dw_reduce(const float* part, float* dw, int S, long long E, cudaStream_t s) {
    if (S < 1 || S > kMaxChunks) return cudaErrorInvalidValue;
    const size_t smem = (size_t)((S + 7) / 8) * kRedElems * sizeof(float);
    // programmatic dependent launch: the reduction's launch and CTA set-up overlap
    // the tail of the partial-sum kernel (which triggers it once its sums are done)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((E + kRedElems - 1) / kRedElems));
    cfg.blockDim = dim3(kRedElems * kRedSlices);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fbc_dw_reduce, part, dw, S, E);
}

}  // namespace fbc
