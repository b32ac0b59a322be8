// rtcg_tc.cuh -- the tensor-core correlation kernel, compiled at plan time by
// NVRTC for sm_103a with the chunk-plane count NC, the split mode, the filter
// width FW, the taps per B stage BT, the epilogue warp count EW, the fused
// conversion switch FUSE (and its converter warps CW), the snippet switch USER,
// the epilogue store path TS (with SB staging slots), the resident-bank
// switch RES, the CTA-pair switch PAIR and the sliding-window switch SW baked in.  Embedded as a string into libfbcorr and prefixed with
// tc_params.h and rtcg_ptx.cuh; self-contained (no system headers).
//
// The correlation of Sec. 6.2 as an implicit GEMM: for every filter tap (i, j)
//   Y[m, n] += sum_d X[m + i*W + j, d] * Wt[n, i, j, d]
// where m = p*W + q runs over output pixels laid out with the INPUT width W
// (columns q >= W' are computed and discarded).  With that layout the A operand
// of every tap is a contiguous run of 128 input pixels, so one shared-memory
// slab of 128+FW-1 pixels per filter row i serves all FW taps of that row:
// tap j is the same slab started j pixels later.
//
// Why run-time generation: one thread issues every tcgen05.mma of a CTA, and a
// 128x256x16 MMA lasts 128 tensor-core cycles, about three times what issuing
// one costs.  Loop control, ring-index and descriptor arithmetic between MMAs
// (runtime tap counts, stage boundaries) left the tensor core idle for a third
// of the time; with FW and BT compile-time the MMA sequence of a filter row is
// straight-line code (the paper's loop unrolling by RTCG, Sec. 4.2 and 6.2).
//
// Roles per CTA (persistent, one per SM):
//   warp 0      producer: cp.async.bulk (1D TMA) of B slices of BT consecutive
//               taps (and, unfused, of pre-split A slabs) into rings,
//               mbarrier complete_tx; it first waits (griddepcontrol.wait) for
//               the operand split the kernel is launched as a dependent of;
//   warp 1      allocates 512 TMEM columns, issues tcgen05.mma (M=128, N<=256,
//               K=16, kind::f16 BF16, FP32 accumulate) into one of two
//               accumulators; tcgen05.commit frees ring slots and hands
//               finished accumulators to the epilogue (PAIR: the even CTA's
//               warp 1 issues M=256 cta_group::2 MMAs for both CTAs, the odd
//               CTA's relays its filled rows);
//   warps 2..   EW epilogue warps (two per TMEM lane quarter when EW = 8),
//               overlapping the MMAs of the next tile; clamp or snippet, then
//               TS = 0: tcgen05.ld 16x256b and streaming stores straight from
//               registers (four lanes write 32 contiguous bytes of one pixel);
//               TS = 1: tcgen05.ld 32x32b into a swizzled shared-memory slot,
//               read back transposed, 16-byte stores of four full lines;
//               TS = 32: the same swizzled 32-pixel x 32-filter blocks leave
//               as tiled bulk stores through the tensor map of y;
//   last CW     (FUSE) converter warps: FP32 x rows -> BF16 hi (and lo) chunk
//               planes of an A slot; FUSE = 1 reads the rows from global memory
//               into registers two rows ahead, FUSE = 2 from a ring of raw rows
//               that the producer fills with one bulk copy per row.
// The bulk-copy unit costs about 150 cycles per copy whatever its size up to
// 16 KB (and moves at most ~110 B per cycle per SM), so the copy count per tile
// matters: B goes in stages of BT taps (one copy per half), and FUSE = 2 brings
// a slab row in one copy where the pre-split planes (FUSE = 0) need NC.
// Operands use the no-swizzle K-major canonical layout: a core matrix is 8 rows
// x 16 bytes, rows contiguous; LBO = byte stride between K-adjacent core
// matrices (one chunk plane), SBO = 128 bytes between 8-row groups.
//
// Split BF16: v = hi + lo, hi = bf16_rn(v), lo = bf16_rn(v - hi); each K step
// issues hi*lo + lo*hi, then hi*hi, into the same FP32 accumulator (the lo*lo
// term, ~2^-16 relative, is dropped).
//
// Resident bank (RES = 1): every 128-row tile otherwise streams the whole bank
// slice of its filter tile through the B ring (400 KB for 256 filters of
// 5x5x32 in BF16), and in plain BF16 the refills, not the tensor core, set the
// pace.  With RES the B ring holds every tap of one filter tile (nb = fh *
// stages per filter row), the producer loads it once, and the CTA walks pixel
// tiles under it: CTA b keeps filter tile b % ntn and takes the pixel tiles
// b / ntn, b / ntn + gridDim.x / ntn, ... (the grid is a multiple of ntn).
//
// CTA pairs (PAIR = 1, launched as clusters of two): with one CTA per tile, a
// 128-row tile of plain BF16 needs 256 B of bank per 256 tensor-core cycles of
// each SM from L2, and the bank refills, not the tensor core, set the pace.  A
// pair shares one M = 256 tile (its two 128-pixel tiles) under cta_group::2
// MMAs: each CTA stages its own A rows and HALF of the bank slice (filters
// 0..127 in the even CTA, 128..255 in the odd one, from the half-width planes),
// so every SM moves half the bank bytes per tile.  The even CTA's MMA thread
// issues for both; the odd CTA's MMA warp relays each filter row it has filled
// (A slot and B stages) to the even CTA's pa_full barriers with one remote
// arrival per row; the MMA commits
// arrive on the ring and accumulator barriers of both CTAs; the odd CTA's
// epilogue warps release an accumulator with remote arrivals on the even CTA's
// acc_empty.  Each CTA stores its own 128 accumulator rows.
//
// Sliding window (SW = 1; one filter tile, W a multiple of 128, single CTAs):
// the slab of filter row i of the tile at output row p, columns c .. c+127, is
// input row p + i, which is also the slab of filter row i - 1 of the tile one
// output row down.  A CTA takes a run of consecutive output rows of one
// 128-pixel column block, and its A ring holds slabs, not (tile, filter row)
// pairs: tile k of the run reads slabs k .. k + fh - 1, so the run of n tiles
// brings in and converts n + fh - 1 slab rows instead of n * fh.  Slab j sits in
// slot j % na (na >= fh), is waited for by every tile that reads it (its slot's
// barrier cannot move on before the slab is released) and is released by its
// last reader: tile j as its filter row 0, or the run's last tile.
//
// Tail halves: tiles t >= nfull, the last partial round of a single 256-wide
// filter tile, run as two 128-column work items each (instruction N = 128, B
// from half-width planes), so that round keeps twice as many SMs busy for half
// as long.  A pair does the same with its pairs of tiles w >= nfull: M = 256,
// N = 128, each CTA staging a quarter of the bank (64 filters) from the
// quarter-width planes.
//
// Every mbarrier wait is bounded in time (%globaltimer); on expiry the kernel
// records an error code in host-mapped memory, stops every role, waits (again
// bounded) for its own copies and MMAs in flight, frees TMEM and returns.

// The PTX wrappers (rtcg_ptx.cuh) precede this file in the generated source.

// Snippet epilogue (USER = 1): defined by the generated source after this file.
__device__ float fbc_user_epi(float y, int n, float lo, float hi);

// All MMAs of one filter tap: K = 16 per instruction over the NC/2 pairs of
// chunk planes; split mode adds hi*lo and lo*hi before hi*hi.
template <int NC, int SPLIT, int CG>
__device__ __forceinline__ void fbc_issue_tap(fbc_u32 d_tmem, fbc_u64 ad, fbc_u64 bd, fbc_u64 ak, fbc_u64 bk,
                                              fbc_u64 alo, fbc_u64 blo, fbc_u32 idesc, fbc_u32& accumulate) {
#pragma unroll
    for (int kk = 0; kk < NC / 2; ++kk) {
        const fbc_u64 a = ad + kk * ak;
        const fbc_u64 b = bd + kk * bk;
        if (SPLIT) {
            fbc_umma<CG>(d_tmem, a, b + blo, idesc, accumulate);
            fbc_umma<CG>(d_tmem, a + alo, b, idesc, 1);
            fbc_umma<CG>(d_tmem, a, b, idesc, 1);
        } else {
            fbc_umma<CG>(d_tmem, a, b, idesc, accumulate);
        }
        accumulate = 1;
    }
}

// ---------------------------------------------------------------- the kernel body
template <int NC, int SPLIT, int FW, int BT, int EW, int FUSE, int CW, int USER, int TS, int SB, int RES,
          int PAIR, int SW>
__device__ __forceinline__ void fbc_tc_corr_body(const FbcTcParams& P) {
    static_assert(!(PAIR && RES), "a CTA pair streams the bank");
    static_assert(!(SW && (PAIR || RES)), "the sliding window runs single CTAs over a streamed bank");
    constexpr int CG = PAIR ? 2 : 1;                 // cta_group of every tcgen05 instruction
    constexpr int NST = (FW + BT - 1) / BT;          // B stages per filter row
    constexpr int L = FBC_TC_TILE_M + FW - 1;        // slab pixels per filter row
    __shared__ int s_abort;
    __shared__ fbc_u32 s_tmem;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const fbc_u32 sbase = fbc_smem_addr(fbc_tc_smem);
    // barrier table: a_full[na] a_empty[na] b_full[nb] b_empty[nb] acc_full[2] acc_empty[2]
    // drain raw_full[nr] raw_empty[nr], and for a pair pa_full[na] (the odd CTA's
    // filter rows, A slot and B stages, relayed to the even CTA)
    const fbc_u32 a_full0 = sbase + P.bar_off;
    const fbc_u32 a_empty0 = a_full0 + 8u * P.na;
    const fbc_u32 b_full0 = a_empty0 + 8u * P.na;
    const fbc_u32 b_empty0 = b_full0 + 8u * P.nb;
    const fbc_u32 acc_full0 = b_empty0 + 8u * P.nb;
    const fbc_u32 acc_empty0 = acc_full0 + 16u;
    const fbc_u32 drain_bar = acc_empty0 + 16u;
    const fbc_u32 raw_full0 = drain_bar + 8u;
    const fbc_u32 raw_empty0 = raw_full0 + 8u * P.nr;
    const fbc_u32 pa_full0 = raw_empty0 + 8u * P.nr;
    // PAIR: this CTA's rank in the pair; rank 0 issues the MMAs of both
    const fbc_u32 rank = PAIR ? fbc_cluster_rank() : 0u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < P.na; ++s) {
            fbc_mbar_init(a_full0 + 8u * s, FUSE ? CW : 1);
            fbc_mbar_init(a_empty0 + 8u * s, 1);
        }
        for (int s = 0; s < P.nb; ++s) {
            fbc_mbar_init(b_full0 + 8u * s, 1);
            fbc_mbar_init(b_empty0 + 8u * s, 1);
        }
        for (int s = 0; s < 2; ++s) {
            fbc_mbar_init(acc_full0 + 8u * s, 1);
            fbc_mbar_init(acc_empty0 + 8u * s, PAIR ? 2 * EW : EW);   // pair: both CTAs' epilogue warps
        }
        if (PAIR)
            for (int s = 0; s < P.na; ++s) fbc_mbar_init(pa_full0 + 8u * s, 1);
        fbc_mbar_init(drain_bar, 1);
        for (int s = 0; s < P.nr; ++s) {
            fbc_mbar_init(raw_full0 + 8u * s, 1);
            fbc_mbar_init(raw_empty0 + 8u * s, CW > 0 ? CW : 1);   // nr = 0 unless FUSE = 2
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 1) {
        // a pair allocates collectively: one warp of each CTA, the same columns in both
        if constexpr (PAIR) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             fbc_smem_addr(&s_tmem)),
                         "r"(FBC_TC_TMEM_COLS));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             fbc_smem_addr(&s_tmem)),
                         "r"(FBC_TC_TMEM_COLS));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        }
    }
    fbc_tc_fence_before();
    // a pair: the peer's barriers are initialised before any remote arrival
    if constexpr (PAIR)
        fbc_cluster_sync();
    else
        __syncthreads();
    fbc_tc_fence_after();
    const fbc_u32 tmem = s_tmem;
    volatile int* abort_flag = &s_abort;
    // Schedule: tile t is pixel tile t % mtiles of filter tile t / mtiles; CTA b
    // takes the work items b, b + gridDim.x, ...
    // Tail halves (one filter tile of 256): the tiles from nfull on, the
    // last partial round, run as two work items each, one per 128-column half of
    // the filter tile, so that round occupies twice as many SMs for half as long;
    // a half takes its B operand from the half-width planes whi2 / wlo2.
    // RES: the CTA's filter tile is blockIdx.x % ntn and its pixel tiles are
    // unit, unit + nunits, ... with unit = blockIdx.x / ntn
    // PAIR (one filter tile of 256): pair u = blockIdx.x / 2 takes the pixel-tile
    // pairs u, u + gridDim.x / 2, ...; pair w is tiles 2w (even CTA) and 2w + 1
    // (odd CTA; tile mtiles, past the image when mtiles is odd, stores nothing)
    // SW: column block blockIdx.x % sw_delta, output rows [sw_r0, sw_r1) of the
    // gridDim.x / sw_delta equal runs of that block
    const int nsched = P.mtiles * P.ntn;
    const int res_fi = RES ? (int)blockIdx.x % P.ntn : 0;
    const int unit = RES ? (int)blockIdx.x / P.ntn : PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
    const int nunits = RES ? (int)gridDim.x / P.ntn : PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
    const int npairs = (P.mtiles + 1) >> 1;
    const int nwork = RES ? P.mtiles : PAIR ? P.nfull + 2 * (npairs - P.nfull) : P.nfull + 2 * (nsched - P.nfull);
    const int sw_runs = SW ? (int)gridDim.x / P.sw_delta : 1;
    const int sw_u = SW ? (int)blockIdx.x / P.sw_delta : 0;
    const int sw_t0 = SW ? (int)((long long)sw_u * P.Ho / sw_runs) * P.sw_delta + (int)blockIdx.x % P.sw_delta : 0;
    const int sw_n = SW ? (int)((long long)(sw_u + 1) * P.Ho / sw_runs - (long long)sw_u * P.Ho / sw_runs) : 0;
    const int my_tiles = SW ? (sw_u < sw_runs ? sw_n : 0)
                            : unit < nwork ? (nwork - 1 - unit) / nunits + 1 : 0;   // work items
    struct Item {
        int tile;    // pixel tile t % mtiles of filter tile t / mtiles
        int nt;      // filter columns of this item (the MMA's N)
        int bn;      // filter rows of B this CTA stages (a pair: nt / 2)
        int n0;      // first filter
        long long wbase;   // byte offset of the item's planes in whi / wlo (half: whi2 / wlo2; quarter: whi4 / wlo4)
        bool half;   // B from the half-width planes
        bool quarter;   // B from the quarter-width planes (a pair's tail half)
    };
    auto item_of = [&](int k) -> Item {
        const int w = unit + k * nunits;
        Item it;
        it.quarter = false;
        if (SW) {
            it.half = false;
            it.tile = sw_t0 + k * P.sw_delta;
            it.nt = P.nt;
            it.bn = P.nt;
            it.n0 = 0;
            it.wbase = 0;
            return it;
        }
        if (PAIR) {
            it.half = true;
            if (w < P.nfull) {
                it.tile = 2 * w + (int)rank;
                it.nt = P.nt;
                it.bn = P.nt >> 1;
                it.n0 = 0;
                it.wbase = (long long)rank * P.fh * FW * NC * it.bn * 16;
            } else {
                // tail half h of pair pw: filters h * 128 .., this CTA's quarter 2h + rank
                const int h = (w - P.nfull) & 1;
                it.quarter = true;
                it.tile = 2 * (P.nfull + ((w - P.nfull) >> 1)) + (int)rank;
                it.nt = P.nt >> 1;
                it.bn = P.nt >> 2;
                it.n0 = h * it.nt;
                it.wbase = (long long)(2 * h + (int)rank) * P.fh * FW * NC * it.bn * 16;
            }
            return it;
        }
        it.half = !RES && w >= P.nfull;
        if (RES) {
            it.tile = res_fi * P.mtiles + w;
        } else if (!it.half) {
            it.tile = w;
        } else {
            it.tile = P.nfull + ((w - P.nfull) >> 1);
        }
        const int nti = it.tile / P.mtiles;
        const int h = (w - P.nfull) & 1;
        it.nt = it.half ? P.nt >> 1 : P.nt;
        it.bn = it.nt;
        it.n0 = it.half ? h * it.nt : nti * P.nt;
        it.wbase = (long long)(it.half ? h : nti) * P.fh * FW * NC * it.nt * 16;
        return it;
    };
    auto tile_of = [&](int k) -> int { return item_of(k).tile; };
    const int R = my_tiles * P.fh;                    // filter rows this CTA runs, in order
    // slab rows this CTA brings in: one per filter row, or (SW) the run's
    // distinct input rows; filter row r reads slab slab_of(r)
    const int RA = SW ? (my_tiles > 0 ? my_tiles + P.fh - 1 : 0) : R;
    auto slab_of = [&](int r) -> int { return SW ? r / P.fh + r % P.fh : r; };
    const fbc_u32 plane = (fbc_u32)P.lp * 16u;        // bytes per A chunk plane (shared)
    const fbc_u32 a_half = NC * plane;                // offset of the lo planes in an A slot
    // first input pixel of slab row r
    auto row_p0 = [&](int r) -> long long {
        if (SW) return (long long)sw_t0 * FBC_TC_TILE_M + (long long)r * P.W;
        const int tile = tile_of(r / P.fh);
        return (long long)(tile % P.mtiles) * FBC_TC_TILE_M + (long long)(r % P.fh) * P.W;
    };
    // pixels of slab row r that lie inside x (the rest reads as zero)
    auto row_valid = [&](long long p0) -> int {
        const long long v = P.npix - p0;
        return (int)(v < 0 ? 0 : (v > L ? L : v));
    };

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            // launched as a dependent of the operand split: its planes (B, and the
            // pre-split x of FUSE = 0) are complete and visible after this wait
            asm volatile("griddepcontrol.wait;" ::: "memory");
            fbc_u32 a_it = 0, b_it = 0, r_it = 0;
            int as = 0, bs = 0, rs = 0;
            fbc_u32 aph = 0, bph = 0, rph = 0;
            bool ok = true;
            const fbc_u32 a_copy = (fbc_u32)L * 16u;
            int next_a = 0;
            for (int r = 0; r < R && ok; ++r) {
                // the A side of rows up to r + look goes out before the B stages of
                // row r, so it is in flight while the MMAs of earlier rows run
                while (FUSE != 1 && ok && next_a < RA && next_a <= slab_of(r) + P.alook) {
                    const long long p0 = row_p0(next_a);
                    if (FUSE == 2) {
                        // one copy of the raw FP32 slab row (16-byte multiples: D % 4 == 0)
                        if (!(ok = fbc_wait(raw_empty0 + 8u * rs, rph ^ 1, P, abort_flag, FBC_TC_ERR_WAIT_EMPTY))) break;
                        const fbc_u32 rfull = raw_full0 + 8u * rs;
                        const fbc_u32 bytes = (fbc_u32)row_valid(p0) * (fbc_u32)P.D * 4u;
                        fbc_mbar_expect_tx(rfull, bytes);
                        if (bytes) fbc_bulk_g2s(sbase + P.raw_off + rs * P.raw_slot, P.xraw + p0 * P.D, bytes, rfull);
                        ++r_it;
                        if (++rs == P.nr) { rs = 0; rph ^= 1; }
                    } else {
                        if (!(ok = fbc_wait(a_empty0 + 8u * as, aph ^ 1, P, abort_flag, FBC_TC_ERR_WAIT_EMPTY))) break;
                        const fbc_u32 afull = a_full0 + 8u * as;
                        fbc_mbar_expect_tx(afull, P.a_tx);
                        const fbc_u32 dst = sbase + P.a_off + as * P.a_slot;
#pragma unroll
                        for (int c = 0; c < NC; ++c) {
                            const long long src = (c * P.npix_pad + p0) * 16;
                            fbc_bulk_g2s(dst + c * plane, P.xhi + src, a_copy, afull);
                            if (SPLIT) fbc_bulk_g2s(dst + a_half + c * plane, P.xlo + src, a_copy, afull);
                        }
                        ++a_it;
                        if (++as == P.na) { as = 0; aph ^= 1; }
                    }
                    ++next_a;
                }
                if (!ok) break;
                // RES: the B stages of the first item's filter rows fill the ring once
                if (RES && r >= P.fh) continue;
                const Item it = item_of(r / P.fh);
                const long long tap_bytes = (long long)NC * it.bn * 16;   // = the item's b_half
                const long long woff = it.wbase + (long long)((r % P.fh) * FW) * tap_bytes;
                const fbc_u8* wtap_hi = (it.quarter ? P.whi4 : it.half ? P.whi2 : P.whi) + woff;
                const fbc_u8* wtap_lo = (it.quarter ? P.wlo4 : it.half ? P.wlo2 : P.wlo) + woff;
                const fbc_u32 b_half = (fbc_u32)tap_bytes;
#pragma unroll
                for (int s = 0; s < NST; ++s) {
                    // taps s*BT .. s*BT+tcnt-1 of this filter row are contiguous in the
                    // operand layout: one copy per half for the whole stage
                    const int tcnt = (s + 1) * BT <= FW ? BT : FW - s * BT;
                    if (!(ok = fbc_wait(b_empty0 + 8u * bs, bph ^ 1, P, abort_flag, FBC_TC_ERR_WAIT_EMPTY))) break;
                    const fbc_u32 bfull = b_full0 + 8u * bs;
                    const fbc_u32 bytes = (fbc_u32)tcnt * b_half;
                    fbc_mbar_expect_tx(bfull, SPLIT ? 2u * bytes : bytes);
                    if ((int)b_it != P.drop_b) {
                        const fbc_u32 bdst = sbase + P.b_off + bs * P.b_stage;
                        fbc_bulk_g2s(bdst, wtap_hi + s * BT * tap_bytes, bytes, bfull);
                        if (SPLIT)
                            fbc_bulk_g2s(bdst + (fbc_u32)BT * b_half, wtap_lo + s * BT * tap_bytes, bytes, bfull);
                    }
                    ++b_it;
                    if (++bs == P.nb) { bs = 0; bph ^= 1; }
                }
            }
            if (!ok) {
                // wait (bounded) for the copies still in flight into each ring slot
                const fbc_u32 a0 = a_it > (fbc_u32)P.na ? a_it - P.na : 0;
                for (fbc_u32 k = a0; k < a_it; ++k) fbc_wait_drain(a_full0 + 8u * (k % P.na), (k / P.na) & 1, P);
                const fbc_u32 b0 = b_it > (fbc_u32)P.nb ? b_it - P.nb : 0;
                for (fbc_u32 k = b0; k < b_it; ++k) fbc_wait_drain(b_full0 + 8u * (k % P.nb), (k / P.nb) & 1, P);
                const fbc_u32 r0 = r_it > (fbc_u32)P.nr ? r_it - P.nr : 0;
                for (fbc_u32 k = r0; k < r_it; ++k) fbc_wait_drain(raw_full0 + 8u * (k % P.nr), (k / P.nr) & 1, P);
            }
        }
    } else if (warp == 1) {
        if (PAIR && rank != 0) {
            // -------------------------------------------------------- relay (odd CTA of a pair)
            // once this CTA's A slot and all B stages of a filter row are filled,
            // one arrival on the even CTA's pa_full of that slot (rows in the
            // order its MMA thread consumes them; the ring holds a whole row)
            if (lane == 0) {
                int as = 0, bs = 0;
                fbc_u32 aph = 0, bph = 0;
                bool ok = true;
                for (int k = 0; k < my_tiles && ok; ++k)
                    for (int i = 0; i < P.fh && ok; ++i) {
                        if (!(ok = fbc_wait(a_full0 + 8u * as, aph, P, abort_flag, FBC_TC_ERR_WAIT_A))) break;
                        for (int s = 0; s < NST && ok; ++s) {
                            ok = fbc_wait(b_full0 + 8u * bs, bph, P, abort_flag, FBC_TC_ERR_WAIT_B);
                            if (++bs == P.nb) { bs = 0; bph ^= 1; }
                        }
                        if (!ok) break;
                        fbc_mbar_arrive_remote(fbc_mapa(pa_full0 + 8u * as, 0u));
                        if (++as == P.na) { as = 0; aph ^= 1; }
                    }
            }
        } else if (lane == 0) {
            // ------------------------------------------------------------ MMA issuer
            const fbc_u32 idesc0 = (1u << 4)                                 // D: FP32
                                   | (1u << 7) | (1u << 10)                  // A, B: BF16
                                   | ((fbc_u32)((PAIR ? 2 : 1) * FBC_TC_TILE_M >> 4) << 24);  // M; N per item
            // descriptor arithmetic: the start address sits in the low 14 bits as
            // (addr >> 4); every shared address is < 2^18, so adding (offset >> 4)
            // to the descriptor never carries out of that field
            const fbc_u64 adesc0 = fbc_smem_desc(sbase + P.a_off, plane, 128);
            const fbc_u64 a_step = P.a_slot >> 4;
            const fbc_u64 ak = (2 * plane) >> 4;
            const fbc_u64 alo = a_half >> 4;
            int as = 0, bs = 0;
            fbc_u32 aph = 0, bph = 0, acc_it = 0;
            fbc_u64 adesc = adesc0;
            bool ok = true;
            bool issued = false;
            for (int k = 0; k < my_tiles && ok; ++k) {
                const int acc = acc_it & 1;
                if (!(ok = fbc_wait(acc_empty0 + 8u * acc, ((acc_it >> 1) & 1) ^ 1, P, abort_flag,
                                        FBC_TC_ERR_WAIT_ACC)))
                    break;
                fbc_tc_fence_after();
                const fbc_u32 d_tmem = tmem + (fbc_u32)(acc * FBC_TC_ACC_COLS);
                // B operand geometry of this work item (a tail half has 128 columns;
                // a pair's N = 256 takes 128 B rows from each CTA)
                const Item itk = item_of(k);
                const int nt_k = itk.nt;
                const fbc_u32 idesc = idesc0 | ((fbc_u32)(nt_k >> 3) << 17);
                const fbc_u32 bplane_i = (fbc_u32)itk.bn * 16u;
                const fbc_u32 bhalf_i = NC * bplane_i;
                const fbc_u64 bk = (2 * bplane_i) >> 4, blo = ((fbc_u64)BT * bhalf_i) >> 4, btap = bhalf_i >> 4;
                fbc_u32 accumulate = 0;
                for (int i = 0; i < P.fh && ok; ++i) {
                    if (SW) {
                        // slab k + i: its slot and the parity of its fill
                        const int j = k + i;
                        as = j % P.na;
                        aph = (fbc_u32)(j / P.na) & 1u;
                        adesc = adesc0 + (fbc_u64)as * a_step;
                    }
                    if (!(ok = fbc_wait(a_full0 + 8u * as, aph, P, abort_flag, FBC_TC_ERR_WAIT_A))) break;
                    if (PAIR && !(ok = fbc_wait(pa_full0 + 8u * as, aph, P, abort_flag, FBC_TC_ERR_WAIT_A))) break;
#pragma unroll
                    for (int s = 0; s < NST; ++s) {
                        // RES: stage (filter row i, s) stays in slot i * NST + s; its
                        // copy is waited for by the first work item only
                        const int slot = RES ? i * NST + s : bs;
                        if (!RES || k == 0)
                            if (!(ok = fbc_wait(b_full0 + 8u * slot, RES ? 0u : bph, P, abort_flag,
                                                    FBC_TC_ERR_WAIT_B)))
                                break;
                        const fbc_u64 bdesc =
                            fbc_smem_desc(sbase + P.b_off + (fbc_u32)slot * P.b_stage, bplane_i, 128);
#pragma unroll
                        for (int t = 0; t < BT; ++t)
                            if (s * BT + t < FW)
                                fbc_issue_tap<NC, SPLIT, CG>(d_tmem, adesc + (fbc_u64)(s * BT + t),
                                                             bdesc + (fbc_u64)t * btap, ak, bk, alo, blo, idesc,
                                                             accumulate);
                        issued = true;
                        if constexpr (!RES) {
                            fbc_umma_commit<CG>(b_empty0 + 8u * bs);
                            if (PAIR) fbc_umma_commit<CG>(fbc_mapa(b_empty0 + 8u * bs, 1u));
                            if (++bs == P.nb) { bs = 0; bph ^= 1; }
                        }
                    }
                    if (!ok) break;
                    if (SW) {
                        // the slab's last reader releases it
                        if (i == 0 || k == my_tiles - 1) fbc_umma_commit<CG>(a_empty0 + 8u * as);
                        continue;
                    }
                    fbc_umma_commit<CG>(a_empty0 + 8u * as);
                    if (PAIR) fbc_umma_commit<CG>(fbc_mapa(a_empty0 + 8u * as, 1u));
                    if (++as == P.na) { as = 0; aph ^= 1; adesc = adesc0; } else { adesc += a_step; }
                }
                if (!ok) break;
                fbc_umma_commit<CG>(acc_full0 + 8u * acc);
                if (PAIR) fbc_umma_commit<CG>(fbc_mapa(acc_full0 + 8u * acc, 1u));
                ++acc_it;
            }
            if (!ok && issued) {
                fbc_umma_commit<CG>(drain_bar);
                fbc_wait_drain(drain_bar, 0, P);
            }
        }
    } else if (warp < 2 + EW) {
        // ------------------------------------------------------------ epilogue
        // tcgen05.ld 16x256b: four consecutive lanes hold 8 contiguous columns of
        // one output pixel, so every 8-byte store of a warp completes one 32-byte
        // sector of each of 8 pixels; no shared-memory transpose.
        const int ew = warp - 2;
        const int lq = warp & 3;         // the TMEM lane quarter this warp may access
        const int part = ew >> 2;        // EW = 8: even / odd 64-column chunks of the quarter
        const bool vec2 = (P.N & 1) == 0;
        // TS: staging slots of this warp (1024-byte aligned for the 128-byte swizzle)
        const fbc_u32 st_base = ((sbase + P.st_off + 1023u) & ~1023u) + (fbc_u32)(ew * SB * FBC_TC_ST_BOX);
        int st_slot = 0;
        fbc_u32 acc_it = 0;
        // the accumulator is free again: this CTA's arrival, or for the odd CTA of
        // a pair a remote arrival on the even CTA's barrier (count 2 EW there)
        const fbc_u32 acc_release0 = (PAIR && rank != 0) ? fbc_mapa(acc_empty0, 0u) : acc_empty0;
        auto release_acc = [&](int acc) {
            if (PAIR && rank != 0)
                fbc_mbar_arrive_remote(acc_release0 + 8u * acc);
            else
                fbc_mbar_arrive(acc_empty0 + 8u * acc);
        };
        for (int k = 0; k < my_tiles; ++k) {
            const Item itm = item_of(k);
            // a pair's odd CTA may hold tile mtiles (past the image): no wrap-around
            const int mt = PAIR ? itm.tile : itm.tile % P.mtiles;
            const int nt_i = itm.nt;     // filter columns of this work item, from column 0 of the accumulator
            const int nb0 = itm.n0;      // its first filter
            const int acc = acc_it & 1;
            if (!fbc_wait(acc_full0 + 8u * acc, (acc_it >> 1) & 1, P, abort_flag, FBC_TC_ERR_WAIT_ACC)) break;
            fbc_tc_fence_after();
            // columns past this tile's last filter hold no result: stop at the tile end as well as N
            const int nend = min(P.N, nb0 + nt_i);
            if constexpr (TS == 1) {
                // tcgen05.ld 32x32b (lane l: 32 consecutive columns of pixel m0 + l)
                // into this warp's swizzled staging slot, read back transposed so
                // that eight lanes hold the 128 contiguous bytes of one pixel's
                // chunk: every 16-byte store instruction writes four full lines.
                const int m0 = mt * FBC_TC_TILE_M + lq * 32;
                long long orow[8];    // output offsets of pixels m0 + 4i + lane / 8 (-1: outside)
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int m = m0 + 4 * i + (lane >> 3);
                    const int p = m / P.W;
                    const int q = m - p * P.W;
                    orow[i] = (p < P.Ho && q < P.Wo) ? ((long long)p * P.Wo + q) * P.N : -1;
                }
                const fbc_u32 wbuf = st_base + (fbc_u32)lane * 128u;
                const fbc_u32 sw = (fbc_u32)(lane & 7);
                const int ch = lane & 7;     // 16-byte chunk this lane reads back and stores
                const bool vec4 = (P.N & 3) == 0 && (reinterpret_cast<unsigned long long>(P.y) & 15) == 0;
                const fbc_u32 trow = tmem + ((fbc_u32)(lq * 32) << 16) + (fbc_u32)(acc * FBC_TC_ACC_COLS);
#pragma unroll 1
                for (int cc = part; cc < (nt_i + 31) >> 5; cc += EW / 4) {
                    fbc_u32 r[32];
                    fbc_tmem_ld32x32b_x32_async(trow + (fbc_u32)(cc * 32), r);
                    fbc_tmem_ld_wait();
                    fbc_reg_fence(r);
                    const int n0 = nb0 + cc * 32;
                    if (n0 >= nend) continue;   // warp-uniform
                    if constexpr (USER != 0) {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            r[j] = __float_as_uint(fbc_user_epi(__uint_as_float(r[j]), n0 + j, P.lo, P.hi));
                    } else if (P.epi == 1) {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            r[j] = __float_as_uint(fminf(fmaxf(__uint_as_float(r[j]), P.lo), P.hi));
                    }
                    __syncwarp();   // the previous chunk's read-back is done
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        fbc_st_shared_v4(wbuf + ((((fbc_u32)c) ^ sw) << 4), r[4 * c], r[4 * c + 1], r[4 * c + 2],
                                         r[4 * c + 3]);
                    __syncwarp();
                    const int n = n0 + 4 * ch;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int row = 4 * i + (lane >> 3);
                        const uint4 v = fbc_ld_shared_v4(st_base + (fbc_u32)row * 128u +
                                                         ((((fbc_u32)ch) ^ (fbc_u32)(row & 7)) << 4));
                        if (orow[i] < 0 || n >= nend) continue;
                        float* dst = P.y + orow[i] + n;
                        if (vec4 && n + 4 <= nend) {
                            fbc_st_cs_v4(dst, v);
                        } else {
                            dst[0] = __uint_as_float(v.x);
                            if (n + 1 < nend) dst[1] = __uint_as_float(v.y);
                            if (n + 2 < nend) dst[2] = __uint_as_float(v.z);
                            if (n + 3 < nend) dst[3] = __uint_as_float(v.w);
                        }
                    }
                }
                fbc_tc_fence_before();
                __syncwarp();
                if (lane == 0) release_acc(acc);
                ++acc_it;
                continue;
            }
            if constexpr (TS > 1) {
                if (P.tma_y) {
                    // tcgen05.ld 32x32b: lane l holds 32 consecutive columns of the
                    // accumulator row of pixel m0 + l.  W % 32 == 0, so the warp's 32
                    // pixels lie in one output row; columns ending past the last
                    // filter, and pixels q >= W', fall outside the tensor map and are
                    // not written.  Each 32x32 block is written into a staging slot
                    // in the 128-byte swizzled layout (16-byte chunk c of row l at
                    // chunk c ^ (l % 8): conflict-free) and leaves as one tiled store.
                    const int m0 = mt * FBC_TC_TILE_M + lq * 32;
                    const int p = m0 / P.W;
                    const int q0 = m0 - p * P.W;
                    const bool inside = p < P.Ho && q0 < P.Wo;
                    const fbc_u32 sw = (fbc_u32)(lane & 7);
                    const fbc_u32 trow = tmem + ((fbc_u32)(lq * 32) << 16) + (fbc_u32)(acc * FBC_TC_ACC_COLS);
#pragma unroll 1
                    for (int cc = part; cc < (nt_i >> 5); cc += EW / 4) {
                        fbc_u32 r[32];
                        fbc_tmem_ld32x32b_x32_async(trow + (fbc_u32)(cc * 32), r);
                        fbc_tmem_ld_wait();
                        fbc_reg_fence(r);
                        const int n0 = nb0 + cc * 32;
                        if (!inside || n0 >= P.N) continue;   // warp-uniform
                        if constexpr (USER != 0) {
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                r[j] = __float_as_uint(fbc_user_epi(__uint_as_float(r[j]), n0 + j, P.lo, P.hi));
                        } else if (P.epi == 1) {
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                r[j] = __float_as_uint(fminf(fmaxf(__uint_as_float(r[j]), P.lo), P.hi));
                        }
                        const fbc_u32 buf = st_base + (fbc_u32)(st_slot * FBC_TC_ST_BOX) + (fbc_u32)lane * 128u;
                        if (lane == 0) fbc_bulk_wait_read<SB - 1>();   // the slot's previous store has read it
                        __syncwarp();
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            fbc_st_shared_v4(buf + ((((fbc_u32)c) ^ sw) << 4), r[4 * c], r[4 * c + 1], r[4 * c + 2],
                                             r[4 * c + 3]);
                        fbc_fence_proxy_async_smem();
                        __syncwarp();
                        if (lane == 0) {
                            fbc_tma_store_3d(P.ymap, st_base + (fbc_u32)(st_slot * FBC_TC_ST_BOX), n0, q0, p);
                            fbc_bulk_commit();
                        }
                        if (++st_slot == SB) st_slot = 0;
                    }
                    fbc_tc_fence_before();
                    __syncwarp();
                    if (lane == 0) release_acc(acc);
                    ++acc_it;
                    continue;
                }
            }
            // 16x256b loads of 64 columns (nt is a multiple of 16)
            const int ncol = (nt_i + 63) / 64;
            // output offsets of pixels lane/4 + 8e of the two 16-lane halves h: ob[2h + e]
            long long ob[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = mt * FBC_TC_TILE_M + lq * 32 + e * 8 + (lane >> 2);
                const int p = m / P.W;
                const int q = m - p * P.W;
                ob[e] = (p < P.Ho && q < P.Wo) ? ((long long)p * P.Wo + q) * P.N : -1;
            }
#pragma unroll 1
            for (int cc = part; cc < ncol; cc += EW / 4) {
                // both 16-lane halves of the quarter in flight before one wait
                fbc_u32 r[2][32];
                const fbc_u32 taddr = tmem + ((fbc_u32)(lq * 32) << 16) + (fbc_u32)(acc * FBC_TC_ACC_COLS + cc * 64);
                fbc_tmem_ld16x256b_x8_async(taddr, r[0]);
                fbc_tmem_ld16x256b_x8_async(taddr + (16u << 16), r[1]);
                fbc_tmem_ld_wait();
                fbc_reg_fence(r[0]);
                fbc_reg_fence(r[1]);
                const int n0 = nb0 + cc * 64 + 2 * (lane & 3);
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int g8 = 0; g8 < 8; ++g8) {
                        const int n = n0 + g8 * 8;
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            float a = __uint_as_float(r[h][4 * g8 + 2 * e]);
                            float b = __uint_as_float(r[h][4 * g8 + 2 * e + 1]);
                            if constexpr (USER != 0) {
                                a = fbc_user_epi(a, n, P.lo, P.hi);
                                b = fbc_user_epi(b, n + 1, P.lo, P.hi);
                            } else if (P.epi == 1) {
                                a = fminf(fmaxf(a, P.lo), P.hi);
                                b = fminf(fmaxf(b, P.lo), P.hi);
                            }
                            const long long o = ob[2 * h + e];
                            if (o < 0 || n >= nend) continue;
                            float* dst = P.y + o + n;
                            if (vec2 && n + 2 <= nend) {
                                fbc_st_cs_f2(dst, a, b);
                            } else {
                                dst[0] = a;
                                if (n + 1 < nend) dst[1] = b;
                            }
                        }
                    }
            }
            fbc_tc_fence_before();
            __syncwarp();
            if (lane == 0) release_acc(acc);
            ++acc_it;
        }
        // tiled stores still in flight read this CTA's shared memory: finish them
        if constexpr (TS > 1)
            if (lane == 0) fbc_bulk_wait_all();
    } else if constexpr (FUSE != 0) {
        // ------------------------------------------------------------ converters
        // FP32 slab row -> BF16 hi (and lo) chunk planes of an A slot, by CW warps.
        // Thread ct owns the 32-byte chunks item = ct + k*32*CW (pixel item / NC,
        // plane item % NC)
        // of every row: FUSE = 1 loads them from x in global memory (a warp reads
        // 1 KB contiguously) two rows ahead of the conversion, FUSE = 2 reads them
        // from the raw-row slot the producer filled.  Generic-proxy shared-memory
        // writes are made visible to the tensor core's async proxy by
        // fence.proxy.async before the arrival on a_full.
        constexpr int NCT = (CW > 0 ? CW : 1) * 32;   // CW = 0 only without conversion (branch discarded)
        constexpr int NITEMS = L * NC;
        constexpr int KI = (NITEMS + NCT - 1) / NCT;   // chunks per thread and row
        static_assert(FUSE != 1 || KI <= FBC_TC_CONV_ITEMS, "slab row too large for the converter registers");
        const int ct = threadIdx.x - (2 + EW) * 32;
        int as = 0, rs = 0;
        fbc_u32 aph = 0, rph = 0;
        if constexpr (FUSE == 1) {
            // two register buffers, even and odd rows: row r + 2 is loaded into the
            // buffer of row r as soon as row r is converted, so a load has about two
            // rows of MMAs to arrive (one row of plain-BF16 MMAs is shorter than a
            // load under load); the same 2 x KI x 32 bytes as a row held while the
            // next one loads
            auto load_row = [&](int r, float4 (&buf)[KI][2]) {
                const long long p0 = row_p0(r);
#pragma unroll
                for (int k = 0; k < KI; ++k) {
                    const int item = ct + k * NCT;
                    const int px = item / NC;
                    const int c = item - px * NC;
                    float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
                    if (item < NITEMS && p0 + px < P.npix) {
                        // D % 4 == 0: each half of the chunk is wholly inside or outside D
                        const float* src = P.xraw + (p0 + px) * P.D + c * 8;
                        if (c * 8 < P.D) v0 = __ldg(reinterpret_cast<const float4*>(src));
                        if (c * 8 + 4 < P.D) v1 = __ldg(reinterpret_cast<const float4*>(src + 4));
                    }
                    buf[k][0] = v0;
                    buf[k][1] = v1;
                }
            };
            auto convert_row = [&](const float4 (&buf)[KI][2]) -> bool {
                if (!fbc_wait(a_empty0 + 8u * as, aph ^ 1, P, abort_flag, FBC_TC_ERR_WAIT_EMPTY)) return false;
                fbc_u8* dst = fbc_tc_smem + P.a_off + as * P.a_slot;
#pragma unroll
                for (int k = 0; k < KI; ++k) {
                    const int item = ct + k * NCT;
                    if (item < NITEMS) {
                        const int px = item / NC;
                        const int c = item - px * NC;
                        const float v[8] = {buf[k][0].x, buf[k][0].y, buf[k][0].z, buf[k][0].w,
                                            buf[k][1].x, buf[k][1].y, buf[k][1].z, buf[k][1].w};
                        fbc_split8<SPLIT>(v, reinterpret_cast<uint4*>(dst + c * plane + px * 16),
                                          reinterpret_cast<uint4*>(dst + a_half + c * plane + px * 16));
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) fbc_mbar_arrive(a_full0 + 8u * as);
                if (++as == P.na) { as = 0; aph ^= 1; }
                return true;
            };
            float4 even[KI][2], odd[KI][2];
            if (RA > 0) load_row(0, even);
            if (RA > 1) load_row(1, odd);
            for (int r = 0; r < RA; r += 2) {
                if (!convert_row(even)) break;
                if (r + 2 < RA) load_row(r + 2, even);
                if (r + 1 >= RA || !convert_row(odd)) break;
                if (r + 3 < RA) load_row(r + 3, odd);
            }
        } else {
            for (int r = 0; r < RA; ++r) {
                if (!fbc_wait(raw_full0 + 8u * rs, rph, P, abort_flag, FBC_TC_ERR_WAIT_A)) break;
                if (!fbc_wait(a_empty0 + 8u * as, aph ^ 1, P, abort_flag, FBC_TC_ERR_WAIT_EMPTY)) break;
                const int valid = row_valid(row_p0(r));
                const float* raw = reinterpret_cast<const float*>(fbc_tc_smem + P.raw_off + rs * P.raw_slot);
                fbc_u8* dst = fbc_tc_smem + P.a_off + as * P.a_slot;
#pragma unroll
                for (int k = 0; k < KI; ++k) {
                    const int item = ct + k * NCT;
                    if (item < NITEMS) {
                        const int px = item / NC;
                        const int c = item - px * NC;
                        float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
                        if (px < valid) {
                            // the two 16-byte halves in an order that spreads the eight
                            // threads of a phase over distinct bank groups (D = 16, 32, 64)
                            const float* src = raw + px * P.D + c * 8;
                            const bool swap = NC == 4 ? (px & 1) : NC == 2 ? ((px >> 1) & 1) : NC == 8 ? ((c >> 2) & 1) : 0;
                            if (swap) {
                                if (c * 8 + 4 < P.D) v1 = *reinterpret_cast<const float4*>(src + 4);
                                if (c * 8 < P.D) v0 = *reinterpret_cast<const float4*>(src);
                            } else {
                                if (c * 8 < P.D) v0 = *reinterpret_cast<const float4*>(src);
                                if (c * 8 + 4 < P.D) v1 = *reinterpret_cast<const float4*>(src + 4);
                            }
                        }
                        const float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                        fbc_split8<SPLIT>(v, reinterpret_cast<uint4*>(dst + c * plane + px * 16),
                                          reinterpret_cast<uint4*>(dst + a_half + c * plane + px * 16));
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    fbc_mbar_arrive(a_full0 + 8u * as);
                    fbc_mbar_arrive(raw_empty0 + 8u * rs);
                }
                if (++as == P.na) { as = 0; aph ^= 1; }
                if (++rs == P.nr) { rs = 0; rph ^= 1; }
            }
        }
    }
    __syncwarp();
    fbc_tc_fence_before();
    // a pair: neither CTA leaves (or frees TMEM) while the other may still reach
    // its shared memory or TMEM, or arrive on its barriers
    if constexpr (PAIR)
        fbc_cluster_sync();
    else
        __syncthreads();
    fbc_tc_fence_after();
    if (warp == 1) {
        if constexpr (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(FBC_TC_TMEM_COLS));
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(FBC_TC_TMEM_COLS));
    }
}
