// rtcg_direct.cuh -- kernel templates compiled at plan time by NVRTC for sm_103a.
//
// This file is embedded as a string into libfbcorr and compiled with the
// filter size, depth and tile of one plan baked in as template arguments --
// the "hardcoding" specialisation that the paper obtains from run-time code
// generation (Sec. 4.2, Sec. 6.2): fixed loop trip counts, fully unrolled
// inner loops, register blocking chosen per shape by the auto-tuner.
// It is self-contained: NVRTC compiles it without any system header.
//
// Operation (Sec. 6.2, Table "Performance of RTCG auto-tuning on 3D
// filter-bank convolutions"), all tensors FP32 with the last index fastest:
//   forward:  y[p][q][n] = epi( sum_{i,j,c} x[p+i][q+j][c] * w[n][i][j][c] )
//   dL/dx:    the same correlation run over the zero-padded upstream gradient
//             g~ with the flipped, transposed bank  w'[d][i][j][n] =
//             w[n][fh-1-i][fw-1-j][d]  (FLIP = 1, pad = (fh-1, fw-1));
//   dL/dw:    dw[n][i][j][c] = sum_{p,q} g~[p][q][n] * x[p+i][q+j][c], as
//             per-chunk partial sums followed by a fixed-order pairwise
//             reduction (deterministic, no atomics).

typedef unsigned int fbc_u32;

// Snippet epilogue (EPI = 2): defined by the generated source after this file.
__device__ float fbc_user_epi(float y, int n, float lo, float hi);

struct FbcDirectArgs {
    const float* __restrict__ x;   // input  [in_h][in_w][C]
    const float* __restrict__ m;   // clamp-mask source, same shape as x (FLIP with MASK only)
    const float* __restrict__ w;   // bank in its original [N][fh][fw][D] layout
    float* __restrict__ y;         // output [out_h][out_w][nf]
    int in_h, in_w, out_h, out_w, nf;
    int pad_y, pad_x;              // output (p, q) reads input (p - pad_y + i, q - pad_x + j)
    float lo, hi;                  // clamp bounds (EPI) or mask bounds (MASK)
};

template <int V>
struct FbcOdd { static constexpr int value = (V % 2 == 1) ? V : V + 1; };

// One CTA computes an output block of BH = TR*WR rows x 32 columns x BN = TF*WF
// output channels.  Lane l of a warp owns output column q0 + l; warp (wr, wf)
// owns rows wr*TR .. +TR and channels wf*TF .. +TF, so each thread holds a
// TR x TF accumulator block.  The input depth is processed in chunks of CC
// channels: per chunk the input halo is staged in shared memory as
// [row][channel][column] (odd column pitch: conflict-free column reads) and
// the CTA's slice of the bank as [i][j][channel][BN+4], so that a warp's TF
// filter values are one broadcast float4 read per 4 filters.  For a fixed
// (j, c) a thread loads TR+FH-1 input values once and reuses them for all FH
// filter rows: TR*TF*FH FMAs per TR+FH-1 scalar and FH*TF/4 vector shared loads.
// Chunking bounds shared memory by CC instead of the full depth C, so large
// filters (11x11x32) and deep inputs (the 64-channel gradient of dL/dx) keep
// several CTAs resident per SM.
// PK = 1 issues the TR x TF multiply-adds as packed pairs over adjacent filters
// (fma.rn.f32x2, sm_100 and later): one instruction per two FMAs, each lane
// rounded exactly like fmaf, so the results are bit-identical to PK = 0 and
// only the issue pressure differs.  The input value is broadcast into both
// halves once per (j, c) and reused for all FH filter rows.
template <int FH, int FW, int C, int TR, int TF, int WR, int WF, int FLIP, int EPI, int MASK, int CC,
          int PK = 0, int PF = 0>
struct FbcDirect {
    static constexpr int BW = 32;
    static constexpr int BH = TR * WR;
    static constexpr int BN = TF * WF;
    static constexpr int NT = 32 * WR * WF;
    static constexpr int HR = BH + FH - 1;
    static constexpr int HC = BW + FW - 1;
    static constexpr int COLP = FbcOdd<HC>::value;
    static constexpr int BNP = BN + 4;
    static constexpr int NCHUNK = (C + CC - 1) / CC;
    static constexpr int XS = ((HR * CC * COLP + 3) / 4) * 4;   // floats, 16-byte multiple
    static constexpr int WS = FH * FW * CC * BNP;
    static constexpr int SMEM_BYTES = (XS + WS) * 4;
    static_assert(TF % 4 == 0, "TF must be a multiple of 4");

    // Staging elements: the halo in 4-channel groups (XV) or single channels, the
    // forward bank in 4-channel groups (WV) or single values.  Each element is
    // loaded from global memory (x_load / w_load) and stored transposed into
    // shared memory (x_store / w_store).
    static constexpr bool XV = (C % 4 == 0) && (CC % 4 == 0);
    static constexpr bool WV = !FLIP && (C % 4 == 0) && (CC % 4 == 0);
    static constexpr int NXE = XV ? HR * HC * (CC / 4) : HR * HC * CC;
    static constexpr int NWE = WV ? BN * FH * FW * (CC / 4) : BN * FH * FW * CC;
    static constexpr int PX = (NXE + NT - 1) / NT;   // elements per thread
    static constexpr int PW = (NWE + NT - 1) / NT;

    static __device__ __forceinline__ float mask_val(float v, float mv, float lo, float hi) {
        return (mv > lo && mv < hi) ? v : 0.0f;
    }

    static __device__ __forceinline__ float4 x_load4(const FbcDirectArgs& a, int e, int c0, int p0, int q0) {
        constexpr int C4 = CC / 4;
        const int c4 = e % C4;
        const int t = e / C4;
        const int col = t % HC;
        const int row = t / HC;
        const int gy = p0 - a.pad_y + row;
        const int gx = q0 - a.pad_x + col;
        const int c = c0 + c4 * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gy >= 0 && gy < a.in_h && gx >= 0 && gx < a.in_w && c < C) {
            const long long off = ((long long)gy * a.in_w + gx) * C + c;
            v = __ldg(reinterpret_cast<const float4*>(a.x + off));
            if (MASK) {
                const float4 mv = __ldg(reinterpret_cast<const float4*>(a.m + off));
                v.x = mask_val(v.x, mv.x, a.lo, a.hi);
                v.y = mask_val(v.y, mv.y, a.lo, a.hi);
                v.z = mask_val(v.z, mv.z, a.lo, a.hi);
                v.w = mask_val(v.w, mv.w, a.lo, a.hi);
            }
        }
        return v;
    }
    static __device__ __forceinline__ void x_store4(float* xs, int e, float4 v) {
        constexpr int C4 = CC / 4;
        const int c4 = e % C4;
        const int t = e / C4;
        const int col = t % HC;
        const int row = t / HC;
        float* dst = xs + (row * CC + c4 * 4) * COLP + col;
        dst[0] = v.x;
        dst[COLP] = v.y;
        dst[2 * COLP] = v.z;
        dst[3 * COLP] = v.w;
    }
    static __device__ __forceinline__ float x_load1(const FbcDirectArgs& a, int e, int c0, int p0, int q0) {
        const int cl = e % CC;
        const int t = e / CC;
        const int col = t % HC;
        const int row = t / HC;
        const int gy = p0 - a.pad_y + row;
        const int gx = q0 - a.pad_x + col;
        const int c = c0 + cl;
        float v = 0.f;
        if (gy >= 0 && gy < a.in_h && gx >= 0 && gx < a.in_w && c < C) {
            const long long off = ((long long)gy * a.in_w + gx) * C + c;
            v = __ldg(a.x + off);
            if (MASK) v = mask_val(v, __ldg(a.m + off), a.lo, a.hi);
        }
        return v;
    }
    static __device__ __forceinline__ void x_store1(float* xs, int e, float v) {
        const int cl = e % CC;
        const int t = e / CC;
        const int col = t % HC;
        const int row = t / HC;
        xs[(row * CC + cl) * COLP + col] = v;
    }
    // forward, 4-channel groups: ws[i][j][cl][f] = w[f0+f][i][j][c0+cl]; filters
    // fastest across the threads, each reading 4 channels of one tap with a
    // 16-byte load and storing them down 4 rows of ws, so that a warp's stores of
    // one component cover consecutive filters
    static __device__ __forceinline__ float4 w_load4(const FbcDirectArgs& a, int e, int c0, int f0) {
        constexpr int C4 = CC / 4;
        const int f = e % BN;
        const int r = e / BN;   // (i*FW + j)*C4 + c4
        const int tap = r / C4;
        const int cl = (r - tap * C4) * 4;
        const int n = f0 + f;
        const int c = c0 + cl;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n < a.nf && c < C) v = __ldg(reinterpret_cast<const float4*>(a.w + ((long long)n * FH * FW + tap) * C + c));
        return v;
    }
    static __device__ __forceinline__ void w_store4(float* ws, int e, float4 v) {
        constexpr int C4 = CC / 4;
        const int f = e % BN;
        const int r = e / BN;
        const int tap = r / C4;
        const int cl = (r - tap * C4) * 4;
        float* dst = ws + (tap * CC + cl) * BNP + f;
        dst[0] = v.x;
        dst[BNP] = v.y;
        dst[2 * BNP] = v.z;
        dst[3 * BNP] = v.w;
    }
    // single values: forward with filters fastest (w[f0+f][i][j][c0+cl]); dL/dx
    // with output channels fastest, reading along them: output channel f is the
    // bank's depth index, input channel c its filter index, ws[i][j][cl][f] =
    // w[c0+cl][FH-1-i][FW-1-j][f0+f]
    static __device__ __forceinline__ float w_load1(const FbcDirectArgs& a, int e, int c0, int f0) {
        const int f = e % BN;
        const int r = e / BN;   // (i*FW + j)*CC + cl
        const int tap = r / CC;
        const int cl = r - tap * CC;
        const int n = f0 + f;
        const int c = c0 + cl;
        if (n >= a.nf || c >= C) return 0.f;
        if (!FLIP) return __ldg(a.w + ((long long)n * FH * FW + tap) * C + c);
        const int i = tap / FW, j = tap - i * FW;
        return __ldg(a.w + (((long long)c * FH + (FH - 1 - i)) * FW + (FW - 1 - j)) * a.nf + n);
    }
    static __device__ __forceinline__ void w_store1(float* ws, int e, float v) {
        const int f = e % BN;
        const int r = e / BN;
        ws[r * BNP + f] = v;   // r = (i*FW + j)*CC + cl
    }

    // Stage input channels [c0, c0+CC) of the halo and the matching bank slice.
    static __device__ __forceinline__ void stage(const FbcDirectArgs& a, float* xs, float* ws, int c0,
                                                 int p0, int q0, int f0) {
        const int tid = threadIdx.x;
        if constexpr (XV) {
            for (int e = tid; e < NXE; e += NT) x_store4(xs, e, x_load4(a, e, c0, p0, q0));
        } else {
            for (int e = tid; e < NXE; e += NT) x_store1(xs, e, x_load1(a, e, c0, p0, q0));
        }
        if constexpr (WV) {
            for (int e = tid; e < NWE; e += NT) w_store4(ws, e, w_load4(a, e, c0, f0));
        } else {
            for (int e = tid; e < NWE; e += NT) w_store1(ws, e, w_load1(a, e, c0, f0));
        }
    }

    // PF = 1: the next chunk's staging elements are loaded into registers before
    // the current chunk is summed (their latency hides behind its FMAs) and
    // stored into shared memory after it.
    struct Pre {
        float4 x4[XV ? PX : 1];
        float x1[XV ? 1 : PX];
        float4 w4[WV ? PW : 1];
        float w1[WV ? 1 : PW];
    };
    static __device__ __forceinline__ void prefetch(const FbcDirectArgs& a, Pre& pre, int c0, int p0, int q0,
                                                    int f0) {
        const int tid = threadIdx.x;
#pragma unroll
        for (int k = 0; k < PX; ++k) {
            const int e = tid + k * NT;
            if constexpr (XV) {
                if (e < NXE) pre.x4[k] = x_load4(a, e, c0, p0, q0);
            } else {
                if (e < NXE) pre.x1[k] = x_load1(a, e, c0, p0, q0);
            }
        }
#pragma unroll
        for (int k = 0; k < PW; ++k) {
            const int e = tid + k * NT;
            if constexpr (WV) {
                if (e < NWE) pre.w4[k] = w_load4(a, e, c0, f0);
            } else {
                if (e < NWE) pre.w1[k] = w_load1(a, e, c0, f0);
            }
        }
    }
    static __device__ __forceinline__ void commit(const Pre& pre, float* xs, float* ws) {
        const int tid = threadIdx.x;
#pragma unroll
        for (int k = 0; k < PX; ++k) {
            const int e = tid + k * NT;
            if constexpr (XV) {
                if (e < NXE) x_store4(xs, e, pre.x4[k]);
            } else {
                if (e < NXE) x_store1(xs, e, pre.x1[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < PW; ++k) {
            const int e = tid + k * NT;
            if constexpr (WV) {
                if (e < NWE) w_store4(ws, e, pre.w4[k]);
            } else {
                if (e < NWE) w_store1(ws, e, pre.w1[k]);
            }
        }
    }

    static __device__ __forceinline__ void run(const FbcDirectArgs& a, float* smem,
                                               int tile_x, int tile_y, int tile_f) {
        const int tid = threadIdx.x;
        const int lane = tid & 31;
        const int warp = tid >> 5;
        const int wr = warp % WR;
        const int wf = warp / WR;
        const int q0 = tile_x * BW;
        const int p0 = tile_y * BH;
        const int f0 = tile_f * BN;
        float* xs = smem;
        float* ws = smem + XS;

        float acc[TR][TF];       // PK = 0
        float2 acc2[TR][TF / 2]; // PK = 1: filters (2k, 2k+1) in one register pair
#pragma unroll
        for (int r = 0; r < TR; ++r) {
#pragma unroll
            for (int f = 0; f < TF; ++f) acc[r][f] = 0.f;
#pragma unroll
            for (int f = 0; f < TF / 2; ++f) acc2[r][f] = make_float2(0.f, 0.f);
        }

        const float* xb = xs + (wr * TR) * CC * COLP + lane;
        const float* wb = ws + wf * TF;
        Pre pre;
        if constexpr (PF) stage(a, xs, ws, 0, p0, q0, f0);
#pragma unroll 1
        for (int ch = 0; ch < NCHUNK; ++ch) {
            if constexpr (PF) {
                __syncthreads();   // chunk ch is staged
                if (ch + 1 < NCHUNK) prefetch(a, pre, (ch + 1) * CC, p0, q0, f0);
            } else {
                if (ch > 0) __syncthreads();   // every thread is done reading the previous chunk
                stage(a, xs, ws, ch * CC, p0, q0, f0);
                __syncthreads();
            }
#pragma unroll 1
            for (int j = 0; j < FW; ++j) {
#pragma unroll 2
                for (int c = 0; c < CC; ++c) {
                    if constexpr (PK) {
                        float2 xv2[TR + FH - 1];
#pragma unroll
                        for (int k = 0; k < TR + FH - 1; ++k) {
                            const float v = xb[(k * CC + c) * COLP + j];
                            xv2[k] = make_float2(v, v);
                        }
#pragma unroll
                        for (int i = 0; i < FH; ++i) {
                            float2 wv2[TF / 2];
                            const float4* wp = reinterpret_cast<const float4*>(wb + ((i * FW + j) * CC + c) * BNP);
#pragma unroll
                            for (int f4 = 0; f4 < TF / 4; ++f4) {
                                const float4 t4 = wp[f4];
                                wv2[2 * f4 + 0] = make_float2(t4.x, t4.y);
                                wv2[2 * f4 + 1] = make_float2(t4.z, t4.w);
                            }
#pragma unroll
                            for (int r = 0; r < TR; ++r)
#pragma unroll
                                for (int f = 0; f < TF / 2; ++f)
                                    acc2[r][f] = __ffma2_rn(xv2[r + i], wv2[f], acc2[r][f]);
                        }
                    } else {
                        float xv[TR + FH - 1];
#pragma unroll
                        for (int k = 0; k < TR + FH - 1; ++k) xv[k] = xb[(k * CC + c) * COLP + j];
#pragma unroll
                        for (int i = 0; i < FH; ++i) {
                            float wv[TF];
                            const float4* wp = reinterpret_cast<const float4*>(wb + ((i * FW + j) * CC + c) * BNP);
#pragma unroll
                            for (int f4 = 0; f4 < TF / 4; ++f4) {
                                const float4 t4 = wp[f4];
                                wv[4 * f4 + 0] = t4.x;
                                wv[4 * f4 + 1] = t4.y;
                                wv[4 * f4 + 2] = t4.z;
                                wv[4 * f4 + 3] = t4.w;
                            }
#pragma unroll
                            for (int r = 0; r < TR; ++r)
#pragma unroll
                                for (int f = 0; f < TF; ++f) acc[r][f] = fmaf(xv[r + i], wv[f], acc[r][f]);
                        }
                    }
                }
            }
            if constexpr (PF) {
                if (ch + 1 < NCHUNK) {
                    __syncthreads();   // every thread is done reading chunk ch
                    commit(pre, xs, ws);
                }
            }
        }

        // ---- epilogue: optional clamp, then store
        const int q = q0 + lane;
        const int nb = f0 + wf * TF;
        const bool vec = ((a.nf & 3) == 0) && (nb + TF <= a.nf);
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            const int p = p0 + wr * TR + r;
            if (p >= a.out_h || q >= a.out_w) continue;
            float* yp = a.y + ((long long)p * a.out_w + q) * a.nf + nb;
            float v[TF];
#pragma unroll
            for (int f = 0; f < TF; ++f) {
                v[f] = PK ? ((f & 1) ? acc2[r][f / 2].y : acc2[r][f / 2].x) : acc[r][f];
                if constexpr (EPI == 2) v[f] = fbc_user_epi(v[f], nb + f, a.lo, a.hi);
                if (EPI == 1) v[f] = fminf(fmaxf(v[f], a.lo), a.hi);
            }
            if (vec) {
#pragma unroll
                for (int f4 = 0; f4 < TF / 4; ++f4)
                    reinterpret_cast<float4*>(yp)[f4] =
                        make_float4(v[4 * f4], v[4 * f4 + 1], v[4 * f4 + 2], v[4 * f4 + 3]);
            } else {
#pragma unroll
                for (int f = 0; f < TF; ++f)
                    if (nb + f < a.nf) yp[f] = v[f];
            }
        }
    }
};

// ---- K-split forward tile for small fh*fw*D --------------------------------
// When the reduction K = FH*FW*C is short (e.g. 9x9x8 = 648) and the output is
// small, one output column per lane leaves most of the GPU idle: 120x120x16
// outputs in 8-output register blocks are under 30 k threads for a machine of
// 311 k.  Here the KS lanes of a lane group share the same outputs and split
// the depth: lane (qs, s) of a warp -- qs = lane / KS, s = lane % KS -- owns
// output column qs of the warp's LQ = 32 / KS columns and accumulates the
// channels c = s, s + KS, ... (channels C..CPAD-1 are zero padding) over all
// FH x FW taps of its TR x TF register block.  The KS partial blocks are then
// combined by a reduce-scatter over the lane bits of s with __shfl_xor_sync:
// at every step a lane keeps one half of its values, receives the partner's
// copy of that half and adds it, so after log2(KS) steps lane s holds the
// complete sums of its share (block entries s*n/KS .. (s+1)*n/KS - 1 of the
// n = TR*TF entries, row-major over (row, filter)).  The summation tree is
// fixed, so the results are deterministic run to run.
// Shared memory keeps the natural layout of x: the halo as [row][column][CP]
// with the pixel pitch CP = CPAD rounded up to KS modulo 32, so that the 32
// lanes of a warp (LQ columns x KS channels) read 32 distinct banks; the bank
// slice as [i][j][c][BNP], one float4 per 4 filters, whose KS distinct channel
// rows fall into distinct bank quads (BNP / 4 odd).  Staging issues all of a
// thread's 16-byte loads of a batch before storing any, so the halo and the
// bank stream in with many loads in flight.
// SHI = 1 takes s from the high lane bits instead (qs = lane % LQ, s = lane / LQ),
// so that the lanes of a quarter warp read the same filter values; the tuner
// measures both.  Forward only (no flip, no mask).  PK = 1 issues packed-pair FMAs.
template <int FH, int FW, int C, int TR, int TF, int KS, int WQ, int WR, int WF, int EPI, int PK = 0,
          int SHI = 0>
struct FbcDirectKS {
    static constexpr int LQ = 32 / KS;
    static constexpr int BW = LQ * WQ;
    static constexpr int BH = TR * WR;
    static constexpr int BN = TF * WF;
    static constexpr int NT = 32 * WQ * WR * WF;
    static constexpr int HR = BH + FH - 1;
    static constexpr int HC = BW + FW - 1;
    static constexpr int CPAD = (C + KS - 1) / KS * KS;
    static constexpr int CPL = CPAD / KS;                          // channels per lane
    static constexpr int CP = CPAD + (((KS - CPAD) % 32) + 32) % 32;   // CP = KS (mod 32)
    static constexpr int BNP = ((BN / 4) % 2 == 1) ? BN : BN + 4;
    static constexpr int XS = HR * HC * CP;
    static constexpr int WS = FH * FW * CPAD * BNP;
    static constexpr int SMEM_BYTES = (XS + WS) * 4;
    static constexpr int NPAIR = TR * TF / 2;                      // accumulator pairs per lane
    static constexpr int NOWN = NPAIR / KS;                        // pairs each lane ends with
    static constexpr int BATCH = 8;                                // 16-byte loads in flight per thread
    static_assert(KS == 4 || KS == 8 || KS == 16 || KS == 32, "KS must be 4, 8, 16 or 32");
    static_assert(TF % 4 == 0, "TF must be a multiple of 4");
    static_assert(NPAIR % KS == 0, "TR*TF/2 must be a multiple of KS");

    // Halo and bank together (C % 4 == 0): one index space over the halo's
    // float4s followed by the bank's, so that a batch issues the loads of both
    // before storing any and the whole staging costs one memory round trip when
    // it fits one batch (first configuration: 1024 + 1296 float4s for 384
    // threads), where staging them one after the other costs two.
    static __device__ __forceinline__ void stage_joint(const FbcDirectArgs& a, float* xs, float* ws, int p0,
                                                       int q0, int f0) {
        const int tid = threadIdx.x;
        constexpr int C4 = C / 4;
        constexpr int NX = HR * HC * C4;
        constexpr int NV = NX + BN * FH * FW * C4;
#pragma unroll 1
        for (int b0 = 0; b0 < NV; b0 += NT * BATCH) {
            float4 v[BATCH];
#pragma unroll
            for (int k = 0; k < BATCH; ++k) {
                const int e = b0 + tid + k * NT;
                v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (e < NX) {
                    const int c4 = e % C4;
                    const int t = e / C4;
                    const int gy = p0 + t / HC, gx = q0 + t % HC;
                    if (gy < a.in_h && gx < a.in_w)
                        v[k] = __ldg(reinterpret_cast<const float4*>(a.x + ((long long)gy * a.in_w + gx) * C) + c4);
                } else if (e < NV) {
                    const int f = (e - NX) % BN;
                    const int r = (e - NX) / BN;   // (i*FW + j)*C4 + c4
                    if (f0 + f < a.nf)
                        v[k] = __ldg(reinterpret_cast<const float4*>(a.w + (long long)(f0 + f) * (FH * FW * C)) + r);
                }
            }
#pragma unroll
            for (int k = 0; k < BATCH; ++k) {
                const int e = b0 + tid + k * NT;
                if (e < NX) {
                    reinterpret_cast<float4*>(xs + (e / C4) * CP)[e % C4] = v[k];
                } else if (e < NV) {
                    const int f = (e - NX) % BN;
                    const int r = (e - NX) / BN;
                    const int tap = r / C4;
                    const int c = (r - tap * C4) * 4;
                    float* dst = ws + (tap * CPAD + c) * BNP + f;
                    dst[0] = v[k].x;
                    dst[BNP] = v[k].y;
                    dst[2 * BNP] = v[k].z;
                    dst[3 * BNP] = v[k].w;
                }
            }
        }
    }

    static __device__ __forceinline__ void stage(const FbcDirectArgs& a, float* xs, float* ws, int p0,
                                                 int q0, int f0) {
        const int tid = threadIdx.x;
        if constexpr (C % 4 == 0 && CPAD == C) {
            stage_joint(a, xs, ws, p0, q0, f0);
            return;
        }
        // ---- input halo [HR][HC][CP]; channels C..CPAD-1 zero
        if constexpr (C % 4 == 0) {
            constexpr int C4 = C / 4;
            constexpr int NV = HR * HC * C4;
#pragma unroll 1
            for (int b0 = 0; b0 < NV; b0 += NT * BATCH) {
                float4 v[BATCH];
#pragma unroll
                for (int k = 0; k < BATCH; ++k) {
                    const int e = b0 + tid + k * NT;
                    v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (e < NV) {
                        const int c4 = e % C4;
                        const int t = e / C4;
                        const int col = t % HC;
                        const int row = t / HC;
                        const int gy = p0 + row, gx = q0 + col;
                        if (gy < a.in_h && gx < a.in_w)
                            v[k] = __ldg(reinterpret_cast<const float4*>(a.x + ((long long)gy * a.in_w + gx) * C) + c4);
                    }
                }
#pragma unroll
                for (int k = 0; k < BATCH; ++k) {
                    const int e = b0 + tid + k * NT;
                    if (e < NV) {
                        const int c4 = e % C4;
                        const int t = e / C4;
                        reinterpret_cast<float4*>(xs + t * CP)[c4] = v[k];
                    }
                }
            }
        } else {
            constexpr int NV = HR * HC * C;
#pragma unroll 1
            for (int b0 = 0; b0 < NV; b0 += NT * BATCH) {
                float v[BATCH];
#pragma unroll
                for (int k = 0; k < BATCH; ++k) {
                    const int e = b0 + tid + k * NT;
                    v[k] = 0.f;
                    if (e < NV) {
                        const int c = e % C;
                        const int t = e / C;
                        const int col = t % HC;
                        const int row = t / HC;
                        const int gy = p0 + row, gx = q0 + col;
                        if (gy < a.in_h && gx < a.in_w) v[k] = __ldg(a.x + ((long long)gy * a.in_w + gx) * C + c);
                    }
                }
#pragma unroll
                for (int k = 0; k < BATCH; ++k) {
                    const int e = b0 + tid + k * NT;
                    if (e < NV) xs[(e / C) * CP + e % C] = v[k];
                }
            }
        }
        if constexpr (CPAD > C) {
            for (int e = tid; e < HR * HC * (CPAD - C); e += NT) {
                const int t = e / (CPAD - C);
                xs[t * CP + C + e % (CPAD - C)] = 0.f;
            }
        }
        // ---- bank slice [FH][FW][CPAD][BNP]: w[f0 + f][i][j][c], zero for c >= C or f0 + f >= nf.
        // Filters fastest across the threads: a warp's scalar stores of one
        // component cover BN consecutive words per 4-channel group
        if constexpr (C % 4 == 0) {
            constexpr int C4 = C / 4;
            constexpr int NV = BN * FH * FW * C4;
#pragma unroll 1
            for (int b0 = 0; b0 < NV; b0 += NT * BATCH) {
                float4 v[BATCH];
#pragma unroll
                for (int k = 0; k < BATCH; ++k) {
                    const int e = b0 + tid + k * NT;
                    v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (e < NV) {
                        const int f = e % BN;
                        const int r = e / BN;   // (i*FW + j)*C4 + c4
                        if (f0 + f < a.nf)
                            v[k] = __ldg(reinterpret_cast<const float4*>(a.w + (long long)(f0 + f) * (FH * FW * C)) + r);
                    }
                }
#pragma unroll
                for (int k = 0; k < BATCH; ++k) {
                    const int e = b0 + tid + k * NT;
                    if (e < NV) {
                        const int f = e % BN;
                        const int r = e / BN;
                        const int tap = r / C4;
                        const int c = (r - tap * C4) * 4;
                        float* dst = ws + (tap * CPAD + c) * BNP + f;
                        dst[0] = v[k].x;
                        dst[BNP] = v[k].y;
                        dst[2 * BNP] = v[k].z;
                        dst[3 * BNP] = v[k].w;
                    }
                }
            }
        } else {
            for (int e = tid; e < BN * FH * FW * C; e += NT) {
                const int f = e % BN;
                const int r = e / BN;   // (i*FW + j)*C + c
                const int tap = r / C;
                const int c = r - tap * C;
                ws[(tap * CPAD + c) * BNP + f] = (f0 + f < a.nf) ? __ldg(a.w + (long long)(f0 + f) * (FH * FW * C) + r) : 0.f;
            }
        }
        if constexpr (CPAD > C) {
            for (int e = tid; e < FH * FW * (CPAD - C) * BN; e += NT) {
                const int f = e % BN;
                const int t = e / BN;
                const int tap = t / (CPAD - C);
                const int c = C + t % (CPAD - C);
                ws[(tap * CPAD + c) * BNP + f] = 0.f;
            }
        }
    }

    static __device__ __forceinline__ void run(const FbcDirectArgs& a, float* smem, int tile_x, int tile_y,
                                               int tile_f) {
        const int tid = threadIdx.x;
        const int lane = tid & 31;
        const int warp = tid >> 5;
        const int s = SHI ? lane / LQ : lane % KS;
        const int qs = SHI ? lane % LQ : lane / KS;
        const int wq = warp % WQ;
        const int wr = (warp / WQ) % WR;
        const int wf = warp / (WQ * WR);
        const int q0 = tile_x * BW;
        const int p0 = tile_y * BH;
        const int f0 = tile_f * BN;
        float* xs = smem;
        float* ws = smem + XS;

        float2 acc[TR][TF / 2];   // filters (2k, 2k+1) of row r
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int f = 0; f < TF / 2; ++f) acc[r][f] = make_float2(0.f, 0.f);

        stage(a, xs, ws, p0, q0, f0);
        __syncthreads();

        const float* xb = xs + ((wr * TR) * HC + wq * LQ + qs) * CP + s;
        const float* wb = ws + s * BNP + wf * TF;
#pragma unroll
        for (int t = 0; t < CPL; ++t) {
#pragma unroll 1
            for (int j = 0; j < FW; ++j) {
                float xv[TR + FH - 1];
#pragma unroll
                for (int k = 0; k < TR + FH - 1; ++k) xv[k] = xb[(k * HC + j) * CP + KS * t];
#pragma unroll
                for (int i = 0; i < FH; ++i) {
                    const float4* wp = reinterpret_cast<const float4*>(wb + ((i * FW + j) * CPAD + KS * t) * BNP);
                    float2 wv[TF / 2];
#pragma unroll
                    for (int f4 = 0; f4 < TF / 4; ++f4) {
                        const float4 t4 = wp[f4];
                        wv[2 * f4 + 0] = make_float2(t4.x, t4.y);
                        wv[2 * f4 + 1] = make_float2(t4.z, t4.w);
                    }
#pragma unroll
                    for (int r = 0; r < TR; ++r) {
                        if constexpr (PK) {
                            const float2 xx = make_float2(xv[r + i], xv[r + i]);
#pragma unroll
                            for (int f = 0; f < TF / 2; ++f) acc[r][f] = __ffma2_rn(xx, wv[f], acc[r][f]);
                        } else {
#pragma unroll
                            for (int f = 0; f < TF / 2; ++f) {
                                acc[r][f].x = fmaf(xv[r + i], wv[f].x, acc[r][f].x);
                                acc[r][f].y = fmaf(xv[r + i], wv[f].y, acc[r][f].y);
                            }
                        }
                    }
                }
            }
        }

        // ---- reduce-scatter over the KS lanes of the group (fixed tree)
        float2 v[NPAIR];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int f = 0; f < TF / 2; ++f) v[r * (TF / 2) + f] = acc[r][f];
        reduce_step<KS / 2, NPAIR>(v, s);

        // ---- epilogue: lane s owns pairs s*NOWN .. s*NOWN + NOWN - 1 of its group's block
        const int q = q0 + wq * LQ + qs;
        if (q >= a.out_w) return;
        constexpr int VW = (NOWN % 2 == 0 && (TF / 2) % 2 == 0) ? 2 : 1;   // pairs per store
#pragma unroll
        for (int k = 0; k < NOWN; k += VW) {
            const int o = s * NOWN + k;
            const int r = o / (TF / 2);
            const int n = f0 + wf * TF + 2 * (o % (TF / 2));
            const int p = p0 + wr * TR + r;
            if (p >= a.out_h) continue;
            float e[2 * VW];
#pragma unroll
            for (int u = 0; u < VW; ++u) {
                e[2 * u] = v[k + u].x;
                e[2 * u + 1] = v[k + u].y;
            }
#pragma unroll
            for (int u = 0; u < 2 * VW; ++u) {
                if constexpr (EPI == 2) e[u] = fbc_user_epi(e[u], n + u, a.lo, a.hi);
                if (EPI == 1) e[u] = fminf(fmaxf(e[u], a.lo), a.hi);
            }
            float* yp = a.y + ((long long)p * a.out_w + q) * a.nf + n;
            if (VW == 2 && (a.nf & 3) == 0 && n + 4 <= a.nf) {
                *reinterpret_cast<float4*>(yp) = make_float4(e[0], e[1], e[2 % (2 * VW)], e[3 % (2 * VW)]);
            } else if (VW == 1 && (a.nf & 1) == 0 && n + 2 <= a.nf) {
                *reinterpret_cast<float2*>(yp) = make_float2(e[0], e[1]);
            } else {
#pragma unroll
                for (int u = 0; u < 2 * VW; ++u)
                    if (n + u < a.nf) yp[u] = e[u];
            }
        }
    }

    // One step of the reduce-scatter over bit M of s, LEN pairs: the lane whose
    // bit M is set keeps the upper half, its partner the lower; each adds the
    // partner's copy of the half it keeps.  Then the next bit, on half as many
    // pairs.  The partner differs in lane bit M (s in the low lane bits) or
    // M * LQ (s in the high bits).
    template <int M, int LEN>
    static __device__ __forceinline__ void reduce_step(float2 (&v)[NPAIR], int s) {
        if constexpr (M >= 1) {
            constexpr int LM = SHI ? M * LQ : M;
            const bool hi = (s & M) != 0;
#pragma unroll
            for (int k = 0; k < LEN / 2; ++k) {
                const float2 send = hi ? v[k] : v[k + LEN / 2];
                const float2 mine = hi ? v[k + LEN / 2] : v[k];
                const float gx = __shfl_xor_sync(0xffffffffu, send.x, LM);
                const float gy = __shfl_xor_sync(0xffffffffu, send.y, LM);
                v[k] = make_float2(mine.x + gx, mine.y + gy);
            }
            reduce_step<M / 2, LEN / 2>(v, s);
        }
    }
};

// ---- dL/dw partial sums -----------------------------------------------------
// Grid: x = chunk of output rows, y = filter row i, z = block of NBLK = TN*NG
// filters.  Thread (ng, c) = (tid / C, tid % C) accumulates
// dw[n0 + ng*TN .. +TN][i][0..FW)[c] over its chunk.  For each output row p the
// CTA walks the row in blocks of QB columns: it stages g~[p][q0..q0+QB)[n-block]
// and the input row segment x[p+i][q0..q0+QB+FW-1)[0..C) in shared memory with
// coalesced loads (zero beyond the row end), then every thread slides an FW-wide
// register window x[p+i][q+j][c] along q (one shared load per column, rotated
// by a compile-time index) and adds TN x FW outer-product terms.  Sums run one
// output row at a time into a row partial that is then added to the chunk total
// (two-level summation); the chunk totals go to part[chunk] for a fixed-order
// pairwise reduction by a second kernel.
struct FbcDwArgs {
    const float* __restrict__ x;   // [H][W][C]
    const float* __restrict__ g;   // [Ho][Wo][N]
    const float* __restrict__ m;   // forward output y for the clamp mask, or unused
    float* __restrict__ part;      // [S][N][FH][FW][C]
    int H, W, Ho, Wo, N;
    int rows_per_chunk;
    float lo, hi;
};

// 16-byte asynchronous copy global -> shared (cp.async, L2 only); bytes = 0
// fills the destination with zeros and reads nothing.
__device__ __forceinline__ void fbc_cp_async16(float* dst, const float* src, int bytes) {
    unsigned d;
    asm("{\n .reg .u64 t;\n cvta.to.shared.u64 t, %1;\n cvt.u32.u64 %0, t;\n}\n" : "=r"(d) : "l"(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void fbc_cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void fbc_cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ---- K-split dL/dx tile with channel chunks in a cp.async ring --------------
// dL/dx of the differentiation workload (Sec. 6.2's correlation run over the
// zero-padded upstream gradient with the flipped bank) has a long reduction
// (K = FH*FW*N = 7*7*64) but a small output (256 x 256 x 16): one output column
// per lane with a 28-value register block is 8 warps per SM, too few to hide
// the latencies of the inner loop, and the register prefetch of the next chunk
// that the lane-per-column tile uses keeps it at that.  Here, as in the K-split
// forward tile, the KS lanes of a lane group (qs = lane / KS, s = lane % KS)
// share a TR x TF output block and split the channels: lane s sums channels
// c0 + s + KS*t of every chunk, and a fixed reduce-scatter over the lane bits
// of s combines the partial blocks at the end (deterministic).  Both operands
// keep their global layouts in shared memory, so every staged element is a
// 16-byte cp.async copy and chunks stream through an NS-stage ring while an
// earlier one is summed, with no registers spent on staging:
//   halo  [HR][HC][CP]: gradient pixels with channels c0 .. c0+CC-1, zero
//         outside the gradient (the padding) -- the copy's zero fill;
//   bank  [FH][FW][CC][BNP]: row (i, j, cl) holds the flipped bank's output
//         channels d0 .. d0+BN-1 for gradient channel n = c0 + cl, which are the
//         contiguous run w[n][FH-1-i][FW-1-j][d0 ..] of the bank itself: the flip
//         turns the bank's layout into the one the tile reads.
// The pixel pitch CP = CC + ((KS - CC) mod 32) makes the LQ x KS lanes of a
// warp read 32 distinct banks; BNP / 4 odd puts the KS channel rows of a float4
// filter read into distinct bank quads.  A block of NPAIR accumulator pairs is
// reduced as NPR = NPAIR rounded up to a multiple of KS pairs (the extra pairs
// are zero and not stored).  Requires C % 4 == 0, nf % 4 == 0, CC % KS == 0,
// CC % 4 == 0; no clamp mask (callers check).
template <int FH, int FW, int C, int TR, int TF, int KS, int WQ, int WR, int WF, int CC, int NS, int PK>
struct FbcDirectKSC {
    static constexpr int LQ = 32 / KS;
    static constexpr int BW = LQ * WQ;
    static constexpr int BH = TR * WR;
    static constexpr int BN = TF * WF;
    static constexpr int NT = 32 * WQ * WR * WF;
    static constexpr int HR = BH + FH - 1;
    static constexpr int HC = BW + FW - 1;
    static constexpr int CPL = CC / KS;                            // channels per lane and chunk
    static constexpr int CP = CC + (((KS - CC) % 32) + 32) % 32;   // CP = KS (mod 32)
    static constexpr int BNP = ((BN / 4) % 2 == 1) ? BN : BN + 4;
    static constexpr int XS = HR * HC * CP;
    static constexpr int WS = FH * FW * CC * BNP;
    static constexpr int STAGE = XS + WS;                          // floats per ring stage
    static constexpr int SMEM_BYTES = NS * STAGE * 4;
    static constexpr int NCH = (C + CC - 1) / CC;
    static constexpr int NPAIR = TR * TF / 2;
    static constexpr int NPR = (NPAIR + KS - 1) / KS * KS;
    static constexpr int NOWN = NPR / KS;
    static_assert(KS == 4 || KS == 8 || KS == 16 || KS == 32, "KS must be 4, 8, 16 or 32");
    static_assert(TF % 4 == 0 && CC % 4 == 0 && CC % KS == 0 && C % 4 == 0, "16-byte staging");
    static_assert(NS == 2 || NS == 3, "two or three ring stages");

    // Issue the copies of chunk kc into ring stage sb (one commit group per chunk).
    static __device__ __forceinline__ void issue(const FbcDirectArgs& a, float* sb, int kc, int p0, int q0,
                                                 int f0) {
        constexpr int C4 = CC / 4;
        constexpr int B4 = BN / 4;
        constexpr int NX = HR * HC * C4;
        constexpr int NV = NX + FH * FW * CC * B4;
        const int c0 = kc * CC;
        float* xs = sb;
        float* ws = sb + XS;
#pragma unroll 4
        for (int e = threadIdx.x; e < NV; e += NT) {
            if (e < NX) {
                const int c4 = e % C4;
                const int t = e / C4;
                const int gy = p0 - a.pad_y + t / HC, gx = q0 - a.pad_x + t % HC;
                const int c = c0 + 4 * c4;
                const bool ok = gy >= 0 && gy < a.in_h && gx >= 0 && gx < a.in_w && c < C;
                fbc_cp_async16(xs + t * CP + 4 * c4, ok ? a.x + ((long long)gy * a.in_w + gx) * C + c : a.x,
                               ok ? 16 : 0);
            } else {
                const int r = e - NX;
                const int f4 = r % B4;
                const int row = r / B4;   // (i*FW + j)*CC + cl
                const int tap = row / CC;
                const int cl = row - tap * CC;
                const int i = tap / FW, j = tap - (tap / FW) * FW;
                const int n = c0 + cl, d = f0 + 4 * f4;
                const bool ok = n < C && d < a.nf;
                fbc_cp_async16(ws + row * BNP + 4 * f4,
                               ok ? a.w + (((long long)n * FH + (FH - 1 - i)) * FW + (FW - 1 - j)) * a.nf + d : a.w,
                               ok ? 16 : 0);
            }
        }
    }

    static __device__ __forceinline__ void run(const FbcDirectArgs& a, float* smem, int tile_x, int tile_y,
                                               int tile_f) {
        const int lane = threadIdx.x & 31;
        const int warp = threadIdx.x >> 5;
        const int s = lane % KS;
        const int qs = lane / KS;
        const int wq = warp % WQ;
        const int wr = (warp / WQ) % WR;
        const int wf = warp / (WQ * WR);
        const int q0 = tile_x * BW;
        const int p0 = tile_y * BH;
        const int f0 = tile_f * BN;

        float2 acc[TR][TF / 2];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int f = 0; f < TF / 2; ++f) acc[r][f] = make_float2(0.f, 0.f);

#pragma unroll
        for (int k = 0; k < NS - 1; ++k) {
            if (k < NCH) issue(a, smem + k * STAGE, k, p0, q0, f0);
            fbc_cp_async_commit();
        }
#pragma unroll 1
        for (int kc = 0; kc < NCH; ++kc) {
            fbc_cp_async_wait<NS - 2>();   // this thread's copies of chunk kc have landed
            __syncthreads();               // everyone's have, and chunk kc-1 is no longer read
            const int kn = kc + NS - 1;    // refill the stage chunk kc-1 used
            if (kn < NCH) issue(a, smem + (kn % NS) * STAGE, kn, p0, q0, f0);
            fbc_cp_async_commit();
            const float* xs = smem + (kc % NS) * STAGE;
            const float* xb = xs + ((wr * TR) * HC + wq * LQ + qs) * CP + s;
            const float* wb = xs + XS + s * BNP + wf * TF;
#pragma unroll
            for (int t = 0; t < CPL; ++t) {
#pragma unroll 1
                for (int j = 0; j < FW; ++j) {
                    float xv[TR + FH - 1];
#pragma unroll
                    for (int k = 0; k < TR + FH - 1; ++k) xv[k] = xb[(k * HC + j) * CP + KS * t];
#pragma unroll
                    for (int i = 0; i < FH; ++i) {
                        const float4* wp = reinterpret_cast<const float4*>(wb + ((i * FW + j) * CC + KS * t) * BNP);
                        float2 wv[TF / 2];
#pragma unroll
                        for (int f4 = 0; f4 < TF / 4; ++f4) {
                            const float4 t4 = wp[f4];
                            wv[2 * f4 + 0] = make_float2(t4.x, t4.y);
                            wv[2 * f4 + 1] = make_float2(t4.z, t4.w);
                        }
#pragma unroll
                        for (int r = 0; r < TR; ++r) {
                            if constexpr (PK) {
                                const float2 xx = make_float2(xv[r + i], xv[r + i]);
#pragma unroll
                                for (int f = 0; f < TF / 2; ++f) acc[r][f] = __ffma2_rn(xx, wv[f], acc[r][f]);
                            } else {
#pragma unroll
                                for (int f = 0; f < TF / 2; ++f) {
                                    acc[r][f].x = fmaf(xv[r + i], wv[f].x, acc[r][f].x);
                                    acc[r][f].y = fmaf(xv[r + i], wv[f].y, acc[r][f].y);
                                }
                            }
                        }
                    }
                }
            }
        }
        fbc_cp_async_wait<0>();   // only empty groups remain; nothing is left in flight at exit

        float2 v[NPR];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int f = 0; f < TF / 2; ++f) v[r * (TF / 2) + f] = acc[r][f];
#pragma unroll
        for (int k = NPAIR; k < NPR; ++k) v[k] = make_float2(0.f, 0.f);
        reduce_step<KS / 2, NPR>(v, s);

        const int q = q0 + wq * LQ + qs;
        if (q >= a.out_w) return;
#pragma unroll
        for (int k = 0; k < NOWN; ++k) {
            const int o = s * NOWN + k;
            if (o >= NPAIR) continue;
            const int r = o / (TF / 2);
            const int n = f0 + wf * TF + 2 * (o % (TF / 2));
            const int p = p0 + wr * TR + r;
            if (p >= a.out_h || n >= a.nf) continue;
            // nf % 4 == 0 and n even: both values of the pair are in range
            *reinterpret_cast<float2*>(a.y + ((long long)p * a.out_w + q) * a.nf + n) = v[k];
        }
    }

    template <int M, int LEN>
    static __device__ __forceinline__ void reduce_step(float2 (&v)[NPR], int s) {
        if constexpr (M >= 1) {
            const bool hi = (s & M) != 0;
#pragma unroll
            for (int k = 0; k < LEN / 2; ++k) {
                const float2 send = hi ? v[k] : v[k + LEN / 2];
                const float2 mine = hi ? v[k + LEN / 2] : v[k];
                const float gx = __shfl_xor_sync(0xffffffffu, send.x, M);
                const float gy = __shfl_xor_sync(0xffffffffu, send.y, M);
                v[k] = make_float2(mine.x + gx, mine.y + gy);
            }
            reduce_step<M / 2, LEN / 2>(v, s);
        }
    }
};

// Shared memory holds two (g block, x segment) buffers: with 16-byte rows of g
// and x (N % 4 == 0, C % 4 == 0) and no clamp mask, the blocks of a chunk stream
// through them with cp.async, the next block's copies in flight while the current
// one is summed (the same arithmetic in the same order as the synchronous path,
// which the other cases take).
template <int FH, int FW, int C, int TN, int NG, int QB, int MASK, int PK = 0>
struct FbcDw {
    static constexpr int NT = C * NG;
    static constexpr int NBLK = TN * NG;
    static constexpr int GS = QB * NBLK;
    static constexpr int XS = (QB + FW - 1) * C;
    // PK = 2 keeps each thread's chunk totals in shared memory ([TN/2][FW][NT]
    // float2, thread-private slots, consecutive threads in consecutive words):
    // the 2 x TN x FW accumulators of the packed form otherwise need about 120
    // registers, which leaves 2 CTAs per SM instead of 3.
    static constexpr int TSZ = (PK == 2) ? TN * FW * NT : 0;
    static constexpr int SMEM_BYTES = (2 * (GS + XS) + TSZ) * 4;

    // Issue the copies of block (p, q0) into buffer (gs, xs): g[p][q0..q0+QB)[n0..n0+NBLK)
    // and x[p+i][q0..q0+QB+FW-1)[0..C), zero-filled past the row ends.
    static __device__ __forceinline__ void issue(const FbcDwArgs& a, float* gs, float* xs, int p, int q0, int i,
                                                 int n0) {
        const int tid = threadIdx.x;
        const int nq = min(QB, a.Wo - q0);
        const long long grow = (long long)p * a.Wo;
        const long long xrow = (long long)(p + i) * a.W;
        for (int e4 = tid; e4 < GS / 4; e4 += NT) {
            const int qq = e4 / (NBLK / 4);
            const int n = n0 + (e4 - qq * (NBLK / 4)) * 4;
            const bool ok = qq < nq && n < a.N;
            fbc_cp_async16(gs + e4 * 4, ok ? a.g + (grow + q0 + qq) * a.N + n : a.g, ok ? 16 : 0);
        }
        for (int e4 = tid; e4 < XS / 4; e4 += NT) {
            const int k = (e4 * 4) / C;
            const bool ok = k < nq + FW - 1 && q0 + k < a.W;
            fbc_cp_async16(xs + e4 * 4, ok ? a.x + (xrow + q0) * C + e4 * 4 : a.x, ok ? 16 : 0);
        }
    }

    // TN x FW outer-product terms of one staged block into ra (the synchronous
    // path's inner loop).
    static __device__ __forceinline__ void sum_block(const float* gs, const float* xs, int ng, int c,
                                                     float (&ra)[TN][FW]) {
        if (ng * TN >= NBLK) return;
        float win[FW];
#pragma unroll
        for (int k = 0; k < FW - 1; ++k) win[k] = xs[k * C + c];
        const float* gp = gs + ng * TN;
        // whole periods of FW columns (the window's rotation phase returns to 0
        // after each), then the QB % FW remaining columns with compile-time
        // indices: no per-column bound test
        constexpr int QF = QB - QB % FW;
#pragma unroll 1
        for (int qb = 0; qb < QF; qb += FW) {
#pragma unroll
            for (int s = 0; s < FW; ++s) column(gp, xs, c, qb + s, s, win, ra);
        }
#pragma unroll
        for (int s = 0; s < QB - QF; ++s) column(gp, xs, c, QF + s, s, win, ra);
    }

    // One output column qq of a staged block: the window's next x value enters
    // slot (s + FW - 1) % FW, then TN x FW multiply-adds.
    static __device__ __forceinline__ void column(const float* gp, const float* xs, int c, int qq, int s,
                                                  float (&win)[FW], float (&ra)[TN][FW]) {
        win[(s + FW - 1) % FW] = xs[(qq + FW - 1) * C + c];
        float gv[TN];
        if constexpr ((TN & 3) == 0) {
            // 16-byte broadcast loads (gp is 16-byte aligned: TN, NBLK % 4 == 0)
#pragma unroll
            for (int t4 = 0; t4 < TN; t4 += 4) {
                const float4 g4 = *reinterpret_cast<const float4*>(gp + qq * NBLK + t4);
                gv[t4] = g4.x; gv[t4 + 1] = g4.y; gv[t4 + 2] = g4.z; gv[t4 + 3] = g4.w;
            }
        } else {
#pragma unroll
            for (int t = 0; t < TN; ++t) gv[t] = gp[qq * NBLK + t];
        }
#pragma unroll
        for (int t = 0; t < TN; ++t)
#pragma unroll
            for (int k = 0; k < FW; ++k) ra[t][k] = fmaf(gv[t], win[(s + k) % FW], ra[t][k]);
    }

    // PK = 1: the same TN x FW terms as packed pairs over adjacent filters
    // (fma.rn.f32x2 on (g[t], g[t+1]) x (x, x)): each lane rounds like fmaf in
    // the same order, so the sums are bit-identical and half as many
    // instructions are issued.
    static __device__ __forceinline__ void sum_block_pk(const float* gs, const float* xs, int ng, int c,
                                                        float2 (&ra)[TN / 2][FW]) {
        if (ng * TN >= NBLK) return;
        float2 win[FW];
#pragma unroll
        for (int k = 0; k < FW - 1; ++k) {
            const float v = xs[k * C + c];
            win[k] = make_float2(v, v);
        }
        const float* gp = gs + ng * TN;
        constexpr int QF = QB - QB % FW;
#pragma unroll 1
        for (int qb = 0; qb < QF; qb += FW) {
#pragma unroll
            for (int s = 0; s < FW; ++s) column_pk(gp, xs, c, qb + s, s, win, ra);
        }
#pragma unroll
        for (int s = 0; s < QB - QF; ++s) column_pk(gp, xs, c, QF + s, s, win, ra);
    }

    static __device__ __forceinline__ void column_pk(const float* gp, const float* xs, int c, int qq, int s,
                                                     float2 (&win)[FW], float2 (&ra)[TN / 2][FW]) {
        const float v = xs[(qq + FW - 1) * C + c];
        win[(s + FW - 1) % FW] = make_float2(v, v);
        float2 gv[TN / 2];
#pragma unroll
        for (int t4 = 0; t4 < TN; t4 += 4) {
            const float4 g4 = *reinterpret_cast<const float4*>(gp + qq * NBLK + t4);
            gv[t4 / 2] = make_float2(g4.x, g4.y);
            gv[t4 / 2 + 1] = make_float2(g4.z, g4.w);
        }
#pragma unroll
        for (int u = 0; u < TN / 2; ++u)
#pragma unroll
            for (int k = 0; k < FW; ++k) ra[u][k] = __ffma2_rn(gv[u], win[(s + k) % FW], ra[u][k]);
    }

    // Top of pipeline step b: block b has landed (this thread's copies: the only
    // group in flight), then one barrier -- every thread's copies have landed and
    // every thread is done with block b - 1 -- after which block b + 1 is issued
    // into the buffer block b - 1 used, to land while block b is summed.
    static __device__ __forceinline__ void next_block(const FbcDwArgs& a, float* smem, int b, int nb, int pb,
                                                      int qblocks, int i, int n0) {
        fbc_cp_async_wait<0>();
        __syncthreads();
        if (b + 1 < nb) {
            const int p1 = pb + (b + 1) / qblocks, q1 = ((b + 1) % qblocks) * QB;
            float* nbuf = smem + ((b + 1) & 1) * (GS + XS);
            issue(a, nbuf, nbuf + GS, p1, q1, i, n0);
        }
        fbc_cp_async_commit();
    }

    static __device__ __forceinline__ void run_async_pk(const FbcDwArgs& a, float* smem, int chunk, int i,
                                                        int nblk) {
        const int tid = threadIdx.x;
        const int ng = tid / C;
        const int c = tid - ng * C;
        const int n0 = nblk * NBLK;
        const int pb = chunk * a.rows_per_chunk;
        int pe = pb + a.rows_per_chunk;
        if (pe > a.Ho) pe = a.Ho;
        const int qblocks = (a.Wo + QB - 1) / QB;
        const int nb = (pe - pb) * qblocks;
        constexpr int TOT_R = (PK == 2) ? 1 : TN / 2;   // register totals only for PK = 1
        float2 tot[TOT_R][FW], ra[TN / 2][FW];
        float2* tots = reinterpret_cast<float2*>(smem + 2 * (GS + XS));
#pragma unroll
        for (int u = 0; u < TN / 2; ++u)
#pragma unroll
            for (int k = 0; k < FW; ++k) {
                ra[u][k] = make_float2(0.f, 0.f);
                if constexpr (PK == 2)
                    tots[(u * FW + k) * NT + tid] = make_float2(0.f, 0.f);
                else
                    tot[u][k] = make_float2(0.f, 0.f);
            }
        if (nb > 0) issue(a, smem, smem + GS, pb, 0, i, n0);
        fbc_cp_async_commit();
        for (int b = 0; b < nb; ++b) {
            const int buf = b & 1;
            next_block(a, smem, b, nb, pb, qblocks, i, n0);
            const float* cur = smem + buf * (GS + XS);
            sum_block_pk(cur, cur + GS, ng, c, ra);
            if ((b + 1) % qblocks == 0) {
#pragma unroll
                for (int u = 0; u < TN / 2; ++u)
#pragma unroll
                    for (int k = 0; k < FW; ++k) {
                        if constexpr (PK == 2) {
                            float2 t2 = tots[(u * FW + k) * NT + tid];
                            t2.x += ra[u][k].x;
                            t2.y += ra[u][k].y;
                            tots[(u * FW + k) * NT + tid] = t2;
                        } else {
                            tot[u][k].x += ra[u][k].x;
                            tot[u][k].y += ra[u][k].y;
                        }
                        ra[u][k] = make_float2(0.f, 0.f);
                    }
            }
        }
        fbc_cp_async_wait<0>();
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");   // the reduction may start launching
#pragma unroll
        for (int t = 0; t < TN; ++t) {
            const int n = n0 + ng * TN + t;
            if (n >= a.N) continue;
#pragma unroll
            for (int k = 0; k < FW; ++k) {
                float2 t2;
                if constexpr (PK == 2)
                    t2 = tots[((t / 2) * FW + k) * NT + tid];
                else
                    t2 = tot[t / 2][k];
                a.part[((((long long)chunk * a.N + n) * FH + i) * FW + k) * C + c] = (t & 1) ? t2.y : t2.x;
            }
        }
    }

    static __device__ __forceinline__ void run_async(const FbcDwArgs& a, float* smem, int chunk, int i,
                                                     int nblk) {
        const int tid = threadIdx.x;
        const int ng = tid / C;
        const int c = tid - ng * C;
        const int n0 = nblk * NBLK;
        const int pb = chunk * a.rows_per_chunk;
        int pe = pb + a.rows_per_chunk;
        if (pe > a.Ho) pe = a.Ho;
        const int qblocks = (a.Wo + QB - 1) / QB;
        const int nb = (pe - pb) * qblocks;   // blocks (row, column block) of this chunk, in order
        float tot[TN][FW], ra[TN][FW];
#pragma unroll
        for (int t = 0; t < TN; ++t)
#pragma unroll
            for (int k = 0; k < FW; ++k) tot[t][k] = ra[t][k] = 0.f;
        if (nb > 0) issue(a, smem, smem + GS, pb, 0, i, n0);
        fbc_cp_async_commit();
        for (int b = 0; b < nb; ++b) {
            const int buf = b & 1;
            next_block(a, smem, b, nb, pb, qblocks, i, n0);
            const float* cur = smem + buf * (GS + XS);
            sum_block(cur, cur + GS, ng, c, ra);
            if ((b + 1) % qblocks == 0) {
                // the row is complete: two-level summation as in the synchronous path
#pragma unroll
                for (int t = 0; t < TN; ++t)
#pragma unroll
                    for (int k = 0; k < FW; ++k) {
                        tot[t][k] += ra[t][k];
                        ra[t][k] = 0.f;
                    }
            }
        }
        fbc_cp_async_wait<0>();
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");   // the reduction may start launching
#pragma unroll
        for (int t = 0; t < TN; ++t) {
            const int n = n0 + ng * TN + t;
            if (n >= a.N) continue;
#pragma unroll
            for (int k = 0; k < FW; ++k)
                a.part[((((long long)chunk * a.N + n) * FH + i) * FW + k) * C + c] = tot[t][k];
        }
    }

    static __device__ __forceinline__ void run(const FbcDwArgs& a, float* smem, int chunk, int i,
                                               int nblk) {
        if constexpr (!MASK && (C % 4) == 0) {
            if ((a.N & 3) == 0) {
                if constexpr (PK && (TN & 3) == 0)
                    run_async_pk(a, smem, chunk, i, nblk);
                else
                    run_async(a, smem, chunk, i, nblk);
                return;
            }
        }
        const int tid = threadIdx.x;
        const int ng = tid / C;
        const int c = tid - ng * C;
        const int n0 = nblk * NBLK;
        float* gs = smem;
        float* xs = smem + GS;
        const int pb = chunk * a.rows_per_chunk;
        int pe = pb + a.rows_per_chunk;
        if (pe > a.Ho) pe = a.Ho;

        float tot[TN][FW];
#pragma unroll
        for (int t = 0; t < TN; ++t)
#pragma unroll
            for (int k = 0; k < FW; ++k) tot[t][k] = 0.f;

        for (int p = pb; p < pe; ++p) {
            float ra[TN][FW];
#pragma unroll
            for (int t = 0; t < TN; ++t)
#pragma unroll
                for (int k = 0; k < FW; ++k) ra[t][k] = 0.f;
            const long long grow = (long long)p * a.Wo;
            const long long xrow = (long long)(p + i) * a.W;
            for (int q0 = 0; q0 < a.Wo; q0 += QB) {
                const int nq = min(QB, a.Wo - q0);
                // g: 4 consecutive filters per 16-byte load (N % 4 == 0 keeps every
                // row of g 16-byte aligned; NBLK is a multiple of 4)
                if ((a.N & 3) == 0) {
                    for (int e4 = tid; e4 < GS / 4; e4 += NT) {
                        const int qq = e4 / (NBLK / 4);
                        const int nl = (e4 - qq * (NBLK / 4)) * 4;
                        const int n = n0 + nl;
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (qq < nq && n < a.N) {
                            const long long off = (grow + q0 + qq) * a.N + n;
                            v = __ldg(reinterpret_cast<const float4*>(a.g + off));
                            if (MASK) {
                                const float4 mv = __ldg(reinterpret_cast<const float4*>(a.m + off));
                                v.x = (mv.x > a.lo && mv.x < a.hi) ? v.x : 0.f;
                                v.y = (mv.y > a.lo && mv.y < a.hi) ? v.y : 0.f;
                                v.z = (mv.z > a.lo && mv.z < a.hi) ? v.z : 0.f;
                                v.w = (mv.w > a.lo && mv.w < a.hi) ? v.w : 0.f;
                            }
                        }
                        reinterpret_cast<float4*>(gs)[e4] = v;
                    }
                } else {
                    for (int e = tid; e < GS; e += NT) {
                        const int qq = e / NBLK;
                        const int nl = e - qq * NBLK;
                        const int n = n0 + nl;
                        float v = 0.f;
                        if (qq < nq && n < a.N) {
                            const long long off = (grow + q0 + qq) * a.N + n;
                            v = __ldg(a.g + off);
                            if (MASK) {
                                const float mv = __ldg(a.m + off);
                                v = (mv > a.lo && mv < a.hi) ? v : 0.f;
                            }
                        }
                        gs[e] = v;
                    }
                }
                // x: the contiguous run of (QB + FW - 1) pixels x C channels of input row p + i
                if constexpr ((C & 3) == 0) {
                    for (int e4 = tid; e4 < XS / 4; e4 += NT) {
                        const int k = (e4 * 4) / C;
                        const int col = q0 + k;
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (k < nq + FW - 1 && col < a.W)
                            v = __ldg(reinterpret_cast<const float4*>(a.x + (xrow + q0) * C) + e4);
                        reinterpret_cast<float4*>(xs)[e4] = v;
                    }
                } else {
                    for (int e = tid; e < XS; e += NT) {
                        const int k = e / C;
                        const int cc = e - k * C;
                        const int col = q0 + k;
                        xs[e] = (k < nq + FW - 1 && col < a.W) ? __ldg(a.x + (xrow + col) * C + cc) : 0.f;
                    }
                }
                __syncthreads();
                sum_block(gs, xs, ng, c, ra);
                __syncthreads();
            }
#pragma unroll
            for (int t = 0; t < TN; ++t)
#pragma unroll
                for (int k = 0; k < FW; ++k) tot[t][k] += ra[t][k];
        }
        // part[chunk][n][i][j][c]
#pragma unroll
        for (int t = 0; t < TN; ++t) {
            const int n = n0 + ng * TN + t;
            if (n >= a.N) continue;
#pragma unroll
            for (int k = 0; k < FW; ++k)
                a.part[((((long long)chunk * a.N + n) * FH + i) * FW + k) * C + c] = tot[t][k];
        }
    }
};

// ---- batched persistent forward ----------------------------------------------
// One launch serves many images, each with its own shape and bank.  Work items
// (image, tile_x, tile_y, tile_f) are sorted largest-first on the host and
// handed out through an atomic counter; the generated kernel switches on the
// image's variant (filter size, depth, tile) and runs that variant's FbcDirect
// tile.  Per-image pointers are kernel parameters; shapes live in `meta`.
struct FbcBatchPtrs {
    const float* x;
    const float* w;
    float* y;
};

template <int NIMG>
struct FbcBatchArgs {
    const int4* __restrict__ work;   // nwork items
    const int* __restrict__ meta;    // per image: in_h, in_w, out_h, out_w, nf, variant
    int* counter;                    // zeroed before every launch
    int nwork;
    float lo, hi;
    int pad_;
    FbcBatchPtrs img[NIMG];
};

__device__ __forceinline__ bool fbc_batch_next(int* counter, int nwork, int* s_item, int4* wk,
                                               const int4* __restrict__ work) {
    if (threadIdx.x == 0) *s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = *s_item;
    __syncthreads();
    if (item >= nwork) return false;
    *wk = work[item];
    return true;
}
