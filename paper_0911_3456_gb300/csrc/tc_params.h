// tc_params.h -- the launch parameters and fixed geometry of the tensor-core
// correlation kernel, shared verbatim by the host (tc_kernel.cu) and by the
// NVRTC source (rtcg_tc.cuh), which gets this text prepended.  Plain types only,
// no includes: NVRTC compiles it without system headers.
#ifndef FBC_TC_PARAMS_H
#define FBC_TC_PARAMS_H

#define FBC_TC_TILE_M 128       // output pixels per tile (MMA M)
#define FBC_TC_ACC_COLS 256     // TMEM columns per accumulator (MMA N <= 256)
#define FBC_TC_TMEM_COLS 512    // two accumulators
#define FBC_TC_CONV_ITEMS 5     // 32-byte x chunks per converter thread and slab row
#define FBC_TC_ST_BOX 4096      // bytes of one staged store box: 32 pixels x 32 FP32 columns

// Error codes written to the host-mapped error word when a bounded wait expires.
#define FBC_TC_ERR_WAIT_A 1
#define FBC_TC_ERR_WAIT_B 2
#define FBC_TC_ERR_WAIT_ACC 3
#define FBC_TC_ERR_WAIT_EMPTY 4

struct FbcTcParams {
    // CUtensorMap of y as {N, Wo, Ho} FP32, 128-byte swizzle, box {32, 32, 1}:
    // the target of the tiled-store epilogue (TS = 32 and tma_y != 0)
    alignas(64) unsigned long long ymap[16];
    const unsigned char* xhi;   // [nc][npix_pad][16 B] pre-split x planes (unfused)
    const unsigned char* xlo;
    const unsigned char* whi;   // [ntn][fh*fw][nc][nt][16 B]
    const unsigned char* wlo;
    const unsigned char* whi2;  // tail halves (nt = 256, ntn = 1): [2][fh*fw][nc][128][16 B]
    const unsigned char* wlo2;
    const unsigned char* whi4;  // a pair's tail halves: quarter-width planes [4][fh*fw][nc][64][16 B]
    const unsigned char* wlo4;
    float* y;                   // [Ho][Wo][N]
    int* err;                   // host-mapped error word
    const float* xraw;          // x itself [H*W][D] (fused: read by the converter warps)
    long long npix_pad;
    long long npix;             // H*W
    unsigned long long wait_ns; // bound of every mbarrier wait
    int W, Ho, Wo, N, D;
    int fh, nt, ntn, mtiles;
    int nfull;                  // tiles (a pair: pairs of tiles) run whole; the rest run as two
                                // halves of the filter tile
    int lp;                     // pixels per chunk plane of an A slot
    int na, nb;                 // A slots, B stages
    int alook;                  // rows by which the A side (slabs or raw rows) runs ahead of the B stages
    int nr;                     // raw-row slots (FUSE = 2)
    int epi;                    // 0: none, 1: clamp to [lo, hi]
    float lo, hi;
    int drop_b;                 // fault injection: B load index whose copy is skipped (-1: none)
    unsigned int a_slot, b_stage;   // bytes per A slot / B stage (hi [+ lo])
    unsigned int a_tx;              // bytes copied per A slot (unfused)
    unsigned int a_off, b_off, bar_off;
    unsigned int raw_off, raw_slot;   // raw-row ring (FUSE = 2): offset, bytes per slot
    unsigned int st_off;              // store staging (TS > 0): offset, 1024-byte aligned at run time
    int tma_y;                        // 1: ymap describes y, epilogue stores go through it
    int sw_delta;                     // sliding window (SW = 1): pixel tiles per input row, W / 128
};

#endif
