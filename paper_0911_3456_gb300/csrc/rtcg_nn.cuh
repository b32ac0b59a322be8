// rtcg_nn.cuh -- exact brute-force nearest-neighbour search (the paper's second
// case study, Sec. 6.4): the screening kernel, compiled at plan time by NVRTC
// with the chunk-plane count NC (dimension / 8), the split mode and the
// epilogue warp count EW baked in.  Prefixed with nn_params.h and rtcg_ptx.cuh.
//
// For target t and neighbour n, |t - n|^2 = |t|^2 + |n|^2 - 2 t.n, and |t|^2 is
// the same for every neighbour of t, so the nearest neighbours of t are those
// with the smallest d'(t, n) = |n|^2 - 2 t.n.  The dot products of a tile of 128
// targets and 256 neighbours are one 128x256xdim GEMM on the tensor cores
// (tcgen05.mma, BF16 in, FP32 accumulate in TMEM; split BF16 by default, three
// products per K step like the correlation kernel), and the epilogue keeps, per
// target, the FBC_NN_KEEP smallest keys (d' as order-preserving bits, neighbour index)
// over the tiles of a work item (only keys below the row's threshold, when the
// plan screens a sample of the neighbours first).  A work item is one target tile against one
// chunk of neighbour tiles; items run chunk-major, so the target tiles that share
// a chunk run at the same time and read its neighbours from HBM once.  The host
// merges the per-item candidates and re-ranks the best few by their exact FP32
// distance (nn.cu).
//
// Roles (persistent CTA, one per SM, 64 + 32*EW threads): warp 0 bulk-copies the
// item's target tile (one copy per half) and streams its neighbour tiles through
// a ring of `nb` stages, and each tile's 256 |n|^2 into one of two 1 KB slots
// that follow the accumulators; warp 1 issues the MMAs into two alternating
// accumulators; EW epilogue warps read the accumulators (tcgen05.ld 32x32b: one
// target row per thread, 32 neighbours per load, the next load in flight while
// one is processed), form d' and keep the running best keys per target row in
// registers, rejecting a 32-column chunk with one comparison of its minimum.

__device__ __forceinline__ fbc_u64 fbc_nn_key(float d, unsigned j) {
    // order-preserving map of the float onto unsigned bits, index in the low word:
    // the smallest key is the smallest distance, then the lowest index
    unsigned u = __float_as_uint(d);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((fbc_u64)u << 32) | j;
}

// Running FBC_NN_KEEP smallest (distance, index) of one target row, sorted; the
// columns of a thread arrive in increasing index order, so strict '<' keeps the
// lowest index on ties.  Almost every candidate fails the first comparison.
// (Four keys per part were measured: no target needed a re-scan on the 1/f patch
// sets, but the insertions made the screening of 4096 x 1M three times slower.)
__device__ __forceinline__ void fbc_nn_keep(float (&bd)[FBC_NN_KEEP], unsigned (&bi)[FBC_NN_KEEP], float d,
                                            unsigned j) {
    if constexpr (FBC_NN_KEEP == 2) {
        if (d < bd[1]) {
            if (d < bd[0]) {
                bd[1] = bd[0];
                bi[1] = bi[0];
                bd[0] = d;
                bi[0] = j;
            } else {
                bd[1] = d;
                bi[1] = j;
            }
        }
        return;
    }
    if (d < bd[FBC_NN_KEEP - 1]) {
#pragma unroll
        for (int k = FBC_NN_KEEP - 1; k > 0; --k) {
            // slot k takes slot k-1's entry if d goes before it, else d if d goes here
            const bool shift = d < bd[k - 1];
            const bool here = !shift && d < bd[k];
            bd[k] = shift ? bd[k - 1] : (here ? d : bd[k]);
            bi[k] = shift ? bi[k - 1] : (here ? j : bi[k]);
        }
        if (d < bd[0]) {
            bd[0] = d;
            bi[0] = j;
        }
    }
}

__device__ __forceinline__ fbc_u64 fbc_shfl_xor_u64(fbc_u64 v, int m) {
    const unsigned lo = __shfl_xor_sync(0xffffffffu, (unsigned)v, m);
    const unsigned hi = __shfl_xor_sync(0xffffffffu, (unsigned)(v >> 32), m);
    return ((fbc_u64)hi << 32) | lo;
}

template <int NC, int SPLIT, int EW>
__device__ __forceinline__ void fbc_nn_body(const FbcNnParams& P) {
    __shared__ int s_abort;
    __shared__ fbc_u32 s_tmem;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const fbc_u32 sbase = fbc_smem_addr(fbc_tc_smem);
    // barrier table: a_full[2] a_empty[2] b_full[nb] b_empty[nb] acc_full[2] acc_empty[2] drain
    const fbc_u32 a_full0 = sbase + P.bar_off;
    const fbc_u32 a_empty0 = a_full0 + 16u;
    const fbc_u32 b_full0 = a_empty0 + 16u;
    const fbc_u32 b_empty0 = b_full0 + 8u * P.nb;
    const fbc_u32 acc_full0 = b_empty0 + 8u * P.nb;
    const fbc_u32 acc_empty0 = acc_full0 + 16u;
    const fbc_u32 drain_bar = acc_empty0 + 16u;
    const fbc_u32 nrm_full0 = drain_bar + 8u;     // |n|^2 slots, paired with the accumulators
    const fbc_u32 nrm_empty0 = nrm_full0 + 16u;
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            fbc_mbar_init(a_full0 + 8u * s, 1);
            fbc_mbar_init(a_empty0 + 8u * s, 1);
            fbc_mbar_init(acc_full0 + 8u * s, 1);
            fbc_mbar_init(acc_empty0 + 8u * s, EW);
        }
        for (int s = 0; s < P.nb; ++s) {
            fbc_mbar_init(b_full0 + 8u * s, 1);
            fbc_mbar_init(b_empty0 + 8u * s, 1);
        }
        fbc_mbar_init(drain_bar, 1);
        for (int s = 0; s < 2; ++s) {
            fbc_mbar_init(nrm_full0 + 8u * s, 1);
            fbc_mbar_init(nrm_empty0 + 8u * s, EW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(fbc_smem_addr(&s_tmem)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fbc_tc_fence_before();
    __syncthreads();
    fbc_tc_fence_after();
    const fbc_u32 tmem = s_tmem;
    volatile int* abort_flag = &s_abort;
    const int items = P.chunks * P.t_tiles;
    constexpr fbc_u32 halves = SPLIT ? 2u : 1u;
    const fbc_u32 a_slot = halves * P.a_bytes, b_stage = halves * P.b_bytes;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            fbc_u32 a_it = 0, b_it = 0;
            int as = 0, bs = 0;
            fbc_u32 aph = 0, bph = 0;
            bool ok = true;
            fbc_u32 n_it = 0;   // neighbour tiles so far: |n|^2 slot n_it & 1
            for (int k = blockIdx.x; k < items && ok; k += gridDim.x) {
                const int c = k / P.t_tiles, t = k - c * P.t_tiles;
                if (!(ok = fbc_wait(a_empty0 + 8u * as, aph ^ 1, P, abort_flag, 4))) break;
                const fbc_u32 afull = a_full0 + 8u * as;
                fbc_mbar_expect_tx(afull, a_slot);
                const fbc_u32 adst = sbase + P.a_off + as * a_slot;
                fbc_bulk_g2s(adst, P.thi + (long long)t * P.a_bytes, P.a_bytes, afull);
                if (SPLIT) fbc_bulk_g2s(adst + P.a_bytes, P.tlo + (long long)t * P.a_bytes, P.a_bytes, afull);
                ++a_it;
                if (++as == P.na) { as = 0; aph ^= 1; }
                const int j1 = min(P.n_tiles, P.tile0 + (c + 1) * P.chunk_tiles);
                for (int jt = P.tile0 + c * P.chunk_tiles; jt < j1 && ok; ++jt) {
                    if (!(ok = fbc_wait(b_empty0 + 8u * bs, bph ^ 1, P, abort_flag, 4))) break;
                    const fbc_u32 bfull = b_full0 + 8u * bs;
                    fbc_mbar_expect_tx(bfull, b_stage);
                    const fbc_u32 bdst = sbase + P.b_off + bs * b_stage;
                    fbc_bulk_g2s(bdst, P.nhi + (long long)jt * P.b_bytes, P.b_bytes, bfull);
                    if (SPLIT) fbc_bulk_g2s(bdst + P.b_bytes, P.nlo + (long long)jt * P.b_bytes, P.b_bytes, bfull);
                    ++b_it;
                    if (++bs == P.nb) { bs = 0; bph ^= 1; }
                    // the tile's |n|^2 for the epilogue (slot freed when it has read them)
                    const fbc_u32 ns = n_it & 1u;
                    if (!(ok = fbc_wait(nrm_empty0 + 8u * ns, ((n_it >> 1) & 1u) ^ 1u, P, abort_flag, 4))) break;
                    const fbc_u32 nfull = nrm_full0 + 8u * ns;
                    fbc_mbar_expect_tx(nfull, FBC_NN_TILE_N * 4u);
                    fbc_bulk_g2s(sbase + P.nrm_off + ns * (FBC_NN_TILE_N * 4u), P.n2 + (long long)jt * FBC_NN_TILE_N,
                                 FBC_NN_TILE_N * 4u, nfull);
                    ++n_it;
                }
            }
            if (!ok) {
                const fbc_u32 a0 = a_it > (fbc_u32)P.na ? a_it - P.na : 0u;
                for (fbc_u32 q = a0; q < a_it; ++q) fbc_wait_drain(a_full0 + 8u * (q % P.na), (q / P.na) & 1, P);
                const fbc_u32 b0 = b_it > (fbc_u32)P.nb ? b_it - P.nb : 0u;
                for (fbc_u32 q = b0; q < b_it; ++q) fbc_wait_drain(b_full0 + 8u * (q % P.nb), (q / P.nb) & 1, P);
                const fbc_u32 n0 = n_it > 2u ? n_it - 2u : 0u;
                for (fbc_u32 q = n0; q < n_it; ++q) fbc_wait_drain(nrm_full0 + 8u * (q & 1u), (q >> 1) & 1u, P);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const fbc_u32 idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((fbc_u32)(FBC_NN_TILE_N >> 3) << 17) |
                                  ((fbc_u32)(FBC_NN_TILE_T >> 4) << 24);
            constexpr fbc_u32 aplane = FBC_NN_TILE_T * 16, bplane = FBC_NN_TILE_N * 16;
            const fbc_u64 adesc0 = fbc_smem_desc(sbase + P.a_off, aplane, 128);
            const fbc_u64 bdesc0 = fbc_smem_desc(sbase + P.b_off, bplane, 128);
            constexpr fbc_u64 ak = (2 * aplane) >> 4, bk = (2 * bplane) >> 4;
            const fbc_u64 alo = P.a_bytes >> 4, blo = P.b_bytes >> 4;
            int as = 0, bs = 0;
            fbc_u32 aph = 0, bph = 0, acc_it = 0;
            bool ok = true, issued = false;
            for (int k = blockIdx.x; k < items && ok; k += gridDim.x) {
                const int c = k / P.t_tiles;
                if (!(ok = fbc_wait(a_full0 + 8u * as, aph, P, abort_flag, 1))) break;
                const fbc_u64 ad = adesc0 + (fbc_u64)((as * a_slot) >> 4);
                const int j1 = min(P.n_tiles, P.tile0 + (c + 1) * P.chunk_tiles);
                for (int jt = P.tile0 + c * P.chunk_tiles; jt < j1 && ok; ++jt) {
                    const int acc = acc_it & 1;
                    if (!(ok = fbc_wait(acc_empty0 + 8u * acc, ((acc_it >> 1) & 1) ^ 1, P, abort_flag, 3))) break;
                    if (!(ok = fbc_wait(b_full0 + 8u * bs, bph, P, abort_flag, 2))) break;
                    fbc_tc_fence_after();
                    const fbc_u32 d_tmem = tmem + (fbc_u32)(acc * 256);
                    const fbc_u64 bd = bdesc0 + (fbc_u64)((bs * b_stage) >> 4);
#pragma unroll
                    for (int kk = 0; kk < NC / 2; ++kk) {
                        const fbc_u64 a = ad + kk * ak, b = bd + kk * bk;
                        if (SPLIT) {
                            fbc_umma(d_tmem, a, b + blo, idesc, kk > 0 ? 1u : 0u);
                            fbc_umma(d_tmem, a + alo, b, idesc, 1u);
                            fbc_umma(d_tmem, a, b, idesc, 1u);
                        } else {
                            fbc_umma(d_tmem, a, b, idesc, kk > 0 ? 1u : 0u);
                        }
                    }
                    issued = true;
                    fbc_umma_commit(b_empty0 + 8u * bs);
                    fbc_umma_commit(acc_full0 + 8u * acc);
                    ++acc_it;
                    if (++bs == P.nb) { bs = 0; bph ^= 1; }
                }
                if (!ok) break;
                fbc_umma_commit(a_empty0 + 8u * as);
                if (++as == P.na) { as = 0; aph ^= 1; }
            }
            if (!ok && issued) {
                fbc_umma_commit(drain_bar);
                fbc_wait_drain(drain_bar, 0, P);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        // tcgen05.ld 32x32b: lane l holds 32 consecutive columns of TMEM lane
        // lq*32 + l, i.e. one target row; warp part (ew / 4) takes the 32-column
        // chunks part, part + EW/4, ... of every tile, in increasing column order.
        static_assert((FBC_NN_TILE_N / 32) % (EW / 4) == 0, "chunks per epilogue warp");
        constexpr int NCH = FBC_NN_TILE_N / 32 / (EW / 4);   // chunks per warp and tile
        const int ew = warp - 2;
        const int lq = warp & 3;
        const int part = ew >> 2;
        const int rows_total = P.t_tiles * FBC_NN_TILE_T;
        fbc_u32 acc_it = 0;
        bool ok = true;
        for (int k = blockIdx.x; k < items && ok; k += gridDim.x) {
            const int c = k / P.t_tiles, t = k - c * P.t_tiles;
            // keys at or above the row's threshold (from a screening of a sample of
            // the neighbours) cannot enter the certificate window: none is kept,
            // so the insertions are rare from the first tile on
            const int row = t * FBC_NN_TILE_T + lq * 32 + lane;
            const float thr0 = P.thr ? P.thr[row] : __int_as_float(0x7f800000);
            float bd[FBC_NN_KEEP];
            unsigned bi[FBC_NN_KEEP];
#pragma unroll
            for (int k = 0; k < FBC_NN_KEEP; ++k) {
                bd[k] = thr0;
                bi[k] = 0xffffffffu;
            }
            const int j1 = min(P.n_tiles, P.tile0 + (c + 1) * P.chunk_tiles);
            for (int jt = P.tile0 + c * P.chunk_tiles; jt < j1; ++jt) {
                const int acc = acc_it & 1;
                const fbc_u32 par = (acc_it >> 1) & 1;
                if (!(ok = fbc_wait(acc_full0 + 8u * acc, par, P, abort_flag, 3))) break;
                if (!(ok = fbc_wait(nrm_full0 + 8u * acc, par, P, abort_flag, 3))) break;
                fbc_tc_fence_after();
                const fbc_u32 trow = tmem + ((fbc_u32)(lq * 32) << 16) + (fbc_u32)(acc * 256);
                const fbc_u32 nrm = sbase + P.nrm_off + (fbc_u32)acc * (FBC_NN_TILE_N * 4u);
                fbc_u32 r[2][32];
                fbc_tmem_ld32x32b_x32_async(trow + (fbc_u32)(part * 32), r[0]);
#pragma unroll
                for (int i = 0; i < NCH; ++i) {
                    const int cc = part + i * (EW / 4);
                    fbc_tmem_ld_wait();
                    fbc_reg_fence(r[i & 1]);
                    if (i + 1 < NCH)   // the next chunk's load runs while this one is processed
                        fbc_tmem_ld32x32b_x32_async(trow + (fbc_u32)((cc + EW / 4) * 32), r[(i + 1) & 1]);
                    float d[32];
                    const float2 neg2 = make_float2(-2.f, -2.f);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const uint4 nv = fbc_ld_shared_v4(nrm + (fbc_u32)(cc * 32 + 4 * q) * 4u);
                        const float2 p0 = __ffma2_rn(neg2, make_float2(__uint_as_float(r[i & 1][4 * q + 0]),
                                                                       __uint_as_float(r[i & 1][4 * q + 1])),
                                                     make_float2(__uint_as_float(nv.x), __uint_as_float(nv.y)));
                        const float2 p1 = __ffma2_rn(neg2, make_float2(__uint_as_float(r[i & 1][4 * q + 2]),
                                                                       __uint_as_float(r[i & 1][4 * q + 3])),
                                                     make_float2(__uint_as_float(nv.z), __uint_as_float(nv.w)));
                        d[4 * q + 0] = p0.x;
                        d[4 * q + 1] = p0.y;
                        d[4 * q + 2] = p1.x;
                        d[4 * q + 3] = p1.y;
                    }
                    // minimum of the chunk as a balanced tree; almost every chunk fails
                    // the comparison with the row's last kept key
                    float m[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) m[j] = fminf(d[2 * j], d[2 * j + 1]);
#pragma unroll
                    for (int w2 = 8; w2 >= 1; w2 >>= 1)
#pragma unroll
                        for (int j = 0; j < w2; ++j) m[j] = fminf(m[j], m[j + w2]);
                    if (m[0] < bd[FBC_NN_KEEP - 1]) {
                        const unsigned n0 = (unsigned)(jt * FBC_NN_TILE_N + cc * 32);
#pragma unroll
                        for (int j = 0; j < 32; ++j) fbc_nn_keep(bd, bi, d[j], n0 + (unsigned)j);
                    }
                }
                fbc_tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    fbc_mbar_arrive(acc_empty0 + 8u * acc);
                    fbc_mbar_arrive(nrm_empty0 + 8u * acc);
                }
                ++acc_it;
            }
            if (!ok) break;
            fbc_u64* dst =
                P.part + (((long long)(P.chunk_base + c) * (EW / 4) + part) * rows_total + row) * FBC_NN_KEEP;
#pragma unroll
            for (int k = 0; k < FBC_NN_KEEP; ++k) dst[k] = bi[k] == 0xffffffffu ? ~0ull : fbc_nn_key(bd[k], bi[k]);
        }
    }
    __syncwarp();
    fbc_tc_fence_before();
    __syncthreads();
    fbc_tc_fence_after();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}
