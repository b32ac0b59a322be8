// nn_params.h -- launch parameters of the nearest-neighbour distance kernel,
// shared verbatim by the host (nn.cu) and the NVRTC source (rtcg_nn.cuh).
// Plain types only, no includes.
#ifndef FBC_NN_PARAMS_H
#define FBC_NN_PARAMS_H

#define FBC_NN_TILE_T 128     // targets per tile (MMA M)
#define FBC_NN_TILE_N 256     // neighbours per tile (MMA N)
#define FBC_NN_KEEP 2         // smallest keys kept per target and screening part

struct FbcNnParams {
    const unsigned char* thi;     // targets, tile-major [t_tiles][nc][128][16 B] BF16 hi
    const unsigned char* tlo;     //   and lo
    const unsigned char* nhi;     // neighbours, tile-major [n_tiles][nc][256][16 B] BF16 hi
    const unsigned char* nlo;     //   and lo
    const float* n2;              // |n_j|^2 (FP32), +inf for the padding neighbours
    unsigned long long* part;     // [chunks][parts][t_tiles*128][FBC_NN_KEEP] smallest keys per target
    const float* thr;             // per target row: keys at or above it are not kept (null: none)
    int* err;                     // host-mapped error word
    unsigned long long wait_ns;   // bound of every mbarrier wait
    int t_tiles, n_tiles;         // 128-target tiles; neighbour tiles [tile0, n_tiles) screened
    int chunk_tiles, chunks;      // neighbour tiles per work item; items = chunks * t_tiles
    int tile0;                    // first neighbour tile of chunk 0
    int chunk_base;               // chunk c writes its parts as chunk chunk_base + c of `part`
    int nb;                       // B stages (neighbour tiles in flight)
    int na;                       // A slots (target tiles): 1 or 2
    unsigned int a_bytes, b_bytes;          // bytes of one half (hi or lo) of an A tile / B tile
    unsigned int a_off, b_off, bar_off;     // shared-memory layout
    unsigned int nrm_off;                   // two 1 KB slots of |n|^2 of a neighbour tile
};

#endif
