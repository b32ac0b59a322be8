// tc_kernel.cu -- host side of the tensor-core (tcgen05) correlation path:
// plan geometry, shared-memory layout, the candidate configurations the
// auto-tuner measures, run-time generation of the kernel source (rtcg_tc.cuh
// specialised per plan) and the BF16 split pre-pass, which is compiled here.
//
// Per forward call: (1) fbc_tc_split writes w -- and, unless the kernel
// converts x itself, x -- as BF16 hi (and lo) chunk planes in the workspace;
// (2) the NVRTC-generated fbc_tc kernel runs the implicit GEMM on the tensor
// cores (one persistent CTA per SM).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <sstream>

#include "internal.h"
#include "tc_params.h"

namespace fbc {

namespace {

constexpr int kTileM = FBC_TC_TILE_M;
constexpr size_t kSmemMax = 227 * 1024 - 1024;   // leave room for static shared memory

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


// ---------------------------------------------------------------- split pre-pass
// Blocks [0, xblocks) convert x, the rest convert w, into the BF16 chunk-plane
// layouts read by the fbc_tc kernel (zero padding for channels >= D, pixels >= H*W,
// filters >= N).  hi = bf16_rn(v); lo = bf16_rn(v - hi) (v - hi is exact in FP32).
struct SplitParams {
    const float* x;
    const float* w;
    uint8_t* xhi;
    uint8_t* xlo;
    uint8_t* whi;
    uint8_t* wlo;
    uint8_t* whi2;   // half-width planes of the tail halves (halves != 0)
    uint8_t* wlo2;
    uint8_t* whi4;   // quarter-width planes of a pair's tail halves (quarters != 0)
    uint8_t* wlo4;
    long long npix, npix_pad;
    int D, nc, N, fh, fw, nt, ntn, split, halves, quarters;
    long long xblocks;
};


__global__ void __launch_bounds__(256) fbc_tc_split(const __grid_constant__ SplitParams S) {
    // the correlation kernel that follows may start now: it waits (griddepcontrol.wait)
    // for this grid's completion before its producer reads any operand plane
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
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
        // one thread per (filter, tap, chunk plane), filters fastest: it reads
        // the 8 channels of its chunk and writes one 16-byte chunk to the planes
        // [ntn][taps][nc][nt] (and the half- and quarter-width copies), contiguous
        // across the warp in every plane
        const long long t = ((long long)blockIdx.x - S.xblocks) * 256 + threadIdx.x;
        const int taps = S.fh * S.fw;
        const long long total = (long long)S.ntn * taps * S.nc * S.nt;
        if (t >= total) return;
        const int nl = (int)(t % S.nt);
        const long long uc = t / S.nt;   // u * nc + c
        const int c = (int)(uc % S.nc);
        const long long u = uc / S.nc;
        const int tap = (int)(u % taps);
        const int nti = (int)(u / taps);
        const int n = nti * S.nt + nl;
        const int i = tap / S.fw, j = tap % S.fw;
        const float* src = S.w + (((long long)n * S.fh + i) * S.fw + j) * S.D;
        const bool inside = n < S.N;
        const bool vec = inside && (S.D & 3) == 0;
        float v[8];
        if (vec && c * 8 + 8 <= S.D) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(src + c * 8));
            const float4 b = __ldg(reinterpret_cast<const float4*>(src + c * 8 + 4));
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int d = c * 8 + k;
                v[k] = (inside && d < S.D) ? __ldg(src + d) : 0.f;
            }
        }
        split8(v, reinterpret_cast<uint4*>(S.whi) + t, reinterpret_cast<uint4*>(S.wlo) + t, S.split);
        if (S.halves) {
            // the same chunk in the half-width planes [2][taps][nc][nt/2] (one filter tile)
            const int hn = S.nt >> 1;
            const int h = nl / hn;
            const long long idx2 = (((long long)h * taps + tap) * S.nc + c) * hn + (nl - h * hn);
            split8(v, reinterpret_cast<uint4*>(S.whi2) + idx2, reinterpret_cast<uint4*>(S.wlo2) + idx2, S.split);
        }
        if (S.quarters) {
            // and in the quarter-width planes [4][taps][nc][nt/4] (a pair's tail halves)
            const int qn = S.nt >> 2;
            const int q = nl / qn;
            const long long idx4 = (((long long)q * taps + tap) * S.nc + c) * qn + (nl - q * qn);
            split8(v, reinterpret_cast<uint4*>(S.whi4) + idx4, reinterpret_cast<uint4*>(S.wlo4) + idx4, S.split);
        }
    }
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct TcConfig {
    int na = 2, nb = 5, ntmax = 256;   // A slots, B stages, widest filter tile
    int bt = 1;                        // filter taps per B stage
    int ew = 4;                        // epilogue warps (4 or 8)
    int fuse = 0;                      // x conversion: 0 pre-pass, 1 converters from global, 2 from a raw ring
    int nr = 0;                        // raw-row slots (fuse = 2)
    int cw = 0;                        // converter warps (fuse = 1, 2): 4 or 8
    int ts = 0;                        // epilogue stores: 0 direct, 32 tiled (32-pixel boxes)
    int sb = 0;                        // staging slots per epilogue warp (ts = 32): 1..3
    int rs = 0;                        // 1: the B ring holds the CTA's whole filter tile (resident bank)
    int cg = 0;                        // 2: CTA pairs (clusters of two, cta_group::2 MMAs, M = 256)
    int sw = 0;                        // 1: sliding window (runs of output rows share their slab rows)
};

struct TcPlan {
    FbcTcParams kp{};     // pointers filled per call
    SplitParams sp{};
    TcConfig cfg;
    size_t smem = 0;
    size_t ws_bytes = 0;  // the largest any candidate configuration needs
    size_t off_xhi = 0, off_xlo = 0, off_whi = 0, off_wlo = 0, off_whi2 = 0, off_wlo2 = 0, off_whi4 = 0, off_wlo4 = 0;
    size_t ws_end = 0;    // workspace bytes this configuration uses
    int grid = 0;
    int split_blocks = 0;
    int H = 0, W = 0, D = 0, N = 0, fh = 0, fw = 0, nc = 0, split = 0, epi = 0;
    float lo = 0.f, hi = 0.f;
    std::string snippet;   // user epilogue expression ("" for none)
    int sm_count = 1;
    unsigned long long wait_ns = 0;
    int drop_b = -1;
    std::map<std::string, Kernel> kernels;   // generated kernels of this plan, by name
    // tensor map of the last output pointer (tiled-store epilogue)
    const float* map_y = nullptr;
    bool map_ok = false;
    alignas(64) unsigned long long map[16] = {};
};

namespace {

int tc_threads(const TcConfig& c) { return 64 + 32 * c.ew + 32 * c.cw; }

std::string tc_kernel_name(int nc, int split, int fw, const TcConfig& c, const std::string& snippet) {
    char b[96];
    snprintf(b, sizeof b, "fbc_tc_c%d_s%d_f%d_b%d_e%d_z%d_w%d", nc, split, fw, c.bt, c.ew, c.fuse, c.cw);
    std::string name = b;
    if (c.ts) name += "_t" + std::to_string(c.ts) + "s" + std::to_string(c.sb);
    if (c.rs) name += "_r";
    if (c.cg) name += "_p";
    if (c.sw) name += "_sw";
    return snippet.empty() ? name : name + "_u" + snippet_tag(snippet);
}

// The NVRTC source of one kernel: parameter block, kernel templates, and an
// extern "C" entry point with this configuration's template arguments.
std::string tc_kernel_source(int nc, int split, int fw, const TcConfig& c, const std::string& snippet) {
    std::ostringstream o;
    o << rtcg_tc_params_source() << "\n" << rtcg_ptx_source() << "\n" << rtcg_tc_source() << "\n"
      << snippet_definition(snippet);
    o << "static_assert(sizeof(FbcTcParams) == " << sizeof(FbcTcParams)
      << ", \"host and device disagree on the parameter block\");\n";
    o << "extern \"C\" __global__ void " << (c.cg ? "__cluster_dims__(2, 1, 1) " : "") << "__launch_bounds__("
      << tc_threads(c) << ", 1) "
      << tc_kernel_name(nc, split, fw, c, snippet) << "(const __grid_constant__ FbcTcParams P) {\n"
      << "  fbc_tc_corr_body<" << nc << "," << split << "," << fw << "," << c.bt << "," << c.ew << ","
      << c.fuse << "," << c.cw << "," << (snippet.empty() ? 0 : 1) << "," << c.ts << "," << (c.ts ? c.sb : 1)
      << "," << c.rs << "," << (c.cg ? 1 : 0) << "," << c.sw << ">(P);\n}\n";
    return o.str();
}

// Filter-tile width for a widest tile of `ntmax` columns: equal tiles, multiples of 16.
void filter_tiles(int N, int ntmax, int* nt, int* ntn) {
    const int npad = (N + 15) / 16 * 16;
    *ntn = (npad + ntmax - 1) / ntmax;
    *nt = ((npad + *ntn - 1) / *ntn + 15) / 16 * 16;
}

bool fuse_ok(int fuse, int cw, int D, int nc, int fw) {
    // x is read as float4 (and copied in 16-byte units); fuse = 1 holds a slab row
    // in at most FBC_TC_CONV_ITEMS 32-byte chunks per converter thread
    if (fuse == 0) return cw == 0;
    if ((D % 4) != 0 || (cw != 4 && cw != 8)) return false;
    return fuse == 2 || (nc <= 4 && (kTileM + fw - 1) * nc <= FBC_TC_CONV_ITEMS * cw * 32);
}

// Tiled stores of 32 pixels x 32 filters: every 32-pixel group of a tile in one
// output row (W % 32 == 0), a row stride of y in 16-byte units (N % 4 == 0), and
// 32-column chunks that never cross into the next filter tile (nt % 32 == 0).
bool ts_ok(int ts, int sb, int W, int N, int nt) {
    if (ts == 0) return sb == 0;
    if (ts == 1) return sb == 1;   // staged transpose: any shape
    return ts == 32 && sb >= 1 && sb <= 3 && W % 32 == 0 && N % 4 == 0 && nt % 32 == 0;
}

// Pixels per A chunk plane: at least the slab (128 + fw - 1), padded so that the
// converters' 16-byte writes are spread over the eight 16-byte bank groups.  A
// converter thread writes the chunk (pixel item / nc, plane item % nc) at
// plane * lp * 16 + pixel * 16; eight consecutive items form one shared-memory
// phase, so the padding e (lp = base + e) is the one that minimises the
// largest number of those eight writes landing in one bank group.
int a_plane_pixels(int slab, int nc) {
    const int base = (slab + 7) / 8 * 8;
    int best_e = 0, best = 1 << 30;
    for (int e = 0; e < 8; ++e) {
        int worst = 0;
        for (int p0 = 0; p0 < 8 * nc; p0 += 8) {   // the phase pattern repeats after 8 nc items
            int hits[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int i = p0; i < p0 + 8; ++i) {
                const int px = i / nc, c = i % nc;
                ++hits[((c * (base + e)) + px) & 7];
            }
            for (int h : hits) worst = std::max(worst, h);
        }
        if (worst < best) { best = worst; best_e = e; }
    }
    return base + best_e;
}

// Lay out shared memory, pipeline depths and the workspace for one configuration.
bool tc_layout(TcPlan* p, const TcConfig& c, bool commit) {
    const int nc = p->nc;
    const int Ho = p->H - p->fh + 1, Wo = p->W - p->fw + 1;
    int nt, ntn;
    filter_tiles(p->N, c.ntmax, &nt, &ntn);
    const long long mvirt = (long long)Ho * p->W;
    const int mtiles = (int)((mvirt + kTileM - 1) / kTileM);
    // the padding spreads the converters' writes over the bank groups; slabs the
    // pre-pass planes fill by bulk copies (fuse = 0) need none
    const int lp = c.fuse ? a_plane_pixels(kTileM + p->fw - 1, nc) : (kTileM + p->fw - 1 + 7) / 8 * 8;
    const int halves = p->split ? 2 : 1;
    const uint32_t a_slot = (uint32_t)align_up((size_t)nc * lp * 16 * halves, 128);
    if (c.bt < 1 || c.bt > p->fw || (c.ew != 4 && c.ew != 8)) return false;
    if (c.fuse < 0 || c.fuse > 2 || !fuse_ok(c.fuse, c.cw, p->D, nc, p->fw)) return false;
    if ((c.fuse == 2) != (c.nr > 0) || c.nr > 4) return false;
    // CTA pairs: one filter tile of 256 (each CTA stages half of it from the
    // half-width planes), streamed (not resident), at least one pair of SMs
    if (c.cg != 0 && (c.cg != 2 || ntn != 1 || nt != 256 || c.rs != 0 || p->sm_count < 2)) return false;
    // a pair relays whole filter rows: the B ring holds at least one row's stages
    if (c.cg && c.nb < (p->fw + c.bt - 1) / c.bt) return false;
    const int bn = c.cg ? nt / 2 : nt;   // B rows this CTA stages
    const uint32_t b_stage = (uint32_t)align_up((size_t)c.bt * nc * bn * 16 * halves, 128);
    const uint32_t raw_slot = (uint32_t)align_up((size_t)(kTileM + p->fw - 1) * p->D * 4, 128);
    if (c.na < 2 || c.nb < 2 || (c.fuse == 2 && c.nr < 2)) return false;
    if (!ts_ok(c.ts, c.sb, p->W, p->N, nt)) return false;
    // resident bank: the ring holds every stage of the filter tile, each CTA
    // keeps one filter tile, and there are at least as many SMs as filter tiles
    if (c.rs != 0 && (c.rs != 1 || c.nb != p->fh * ((p->fw + c.bt - 1) / c.bt) || ntn > std::max(1, p->sm_count)))
        return false;
    // sliding window: one filter tile, whole 128-pixel column blocks per input
    // row, single CTAs over a streamed bank, the A ring holding fh slabs, and a
    // run of at least one output row for every CTA
    const int sw_delta = p->W / kTileM;
    if (c.sw != 0 && (c.sw != 1 || c.cg || c.rs || ntn != 1 || p->W % kTileM != 0 || c.na < p->fh ||
                      p->sm_count < sw_delta))
        return false;
    // the barrier table: a_full / a_empty per A slot, b_full / b_empty per B stage,
    // two accumulator pairs, the drain barrier, raw_full / raw_empty per raw slot,
    // and for a pair pa_full per A slot
    if (8 * (2 * c.na + 2 * c.nb + 5 + 2 * c.nr + (c.cg ? c.na : 0)) > 512) return false;
    // staging: a 1024-byte aligned run of ew * sb boxes placed after the barriers
    const size_t staging = c.ts ? (size_t)c.ew * c.sb * FBC_TC_ST_BOX + 1024 : 0;
    const size_t need = (size_t)c.na * a_slot + (size_t)c.nb * b_stage + (size_t)c.nr * raw_slot + 512 + staging;
    if (need > kSmemMax) return false;
    if (!commit) return true;
    p->cfg = c;
    FbcTcParams& k = p->kp;
    k = FbcTcParams{};
    k.npix_pad = (long long)align_up((size_t)p->H * p->W + kTileM + p->fw + 8, 8);
    k.npix = (long long)p->H * p->W;
    k.W = p->W; k.Ho = Ho; k.Wo = Wo; k.N = p->N; k.D = p->D;
    k.fh = p->fh; k.nt = nt; k.ntn = ntn; k.mtiles = mtiles;
    // tail halves: when the last round of whole tiles would leave at least half
    // of the CTAs idle, its tiles run as two 128-column halves each
    const int grid_full = std::min(mtiles * ntn, std::max(1, p->sm_count));
    const int rem = (mtiles * ntn) % grid_full;
    const bool tail_halves = !c.rs && !c.cg && !c.sw && ntn == 1 && nt == 256 && rem > 0 && 2 * rem <= grid_full &&
                             env_str("FBCORR_TAIL_HALVES", "1") != "0";
    const bool half_planes = tail_halves || c.cg;   // B from the half-width planes
    k.nfull = tail_halves ? mtiles * ntn - rem : mtiles * ntn;
    // a pair's tail halves: the same rule over pairs of tiles and pairs of SMs;
    // nfull then counts pairs run whole
    const int npairs = (mtiles + 1) / 2;
    const int grid_pairs = std::min(npairs, std::max(1, p->sm_count / 2));
    const int prem = npairs % grid_pairs;
    const bool pair_tail = c.cg && prem > 0 && 2 * prem <= grid_pairs && env_str("FBCORR_TAIL_HALVES", "1") != "0";
    if (c.cg) k.nfull = pair_tail ? npairs - prem : npairs;
    k.lp = lp; k.na = c.na; k.nb = c.nb;
    k.a_slot = a_slot; k.b_stage = b_stage;
    k.a_tx = (uint32_t)(nc * (kTileM + p->fw - 1) * 16 * halves);
    k.a_off = 0;
    k.b_off = (uint32_t)(c.na * a_slot);
    // A-side look-ahead: pre-split slabs need a free A slot beyond the one the
    // MMAs of the previous row still read (three slots); raw rows run nr - 1 ahead
    k.alook = c.fuse == 2 ? c.nr - 1 : (c.na >= 3 ? 1 : 0);
    k.nr = c.nr;
    k.raw_off = (uint32_t)(k.b_off + c.nb * b_stage);
    k.raw_slot = c.nr ? raw_slot : 0;
    k.bar_off = (uint32_t)(k.raw_off + (size_t)c.nr * raw_slot);
    k.epi = p->epi; k.lo = p->lo; k.hi = p->hi;
    k.wait_ns = p->wait_ns;
    k.drop_b = p->drop_b;
    k.st_off = k.bar_off + 512;
    k.sw_delta = c.sw ? sw_delta : 0;
    p->smem = k.st_off + staging;
    // a pair's CTAs must sit on two SMs, one CTA per SM: with room for two CTAs
    // in one SM's shared memory two CTAs of different pairs could share an SM,
    // and pairs waiting for each other's TMEM could deadlock
    if (c.cg) p->smem = std::max(p->smem, kSmemMax / 2 + 4096);
    p->map_y = nullptr;   // re-encode for the next call

    const size_t xplanes = (size_t)nc * k.npix_pad * 16;
    const size_t wplanes = (size_t)ntn * p->fh * p->fw * nc * nt * 16;
    size_t off = 0;
    p->off_xhi = off; off = align_up(off + xplanes, 256);
    p->off_xlo = off; if (p->split) off = align_up(off + xplanes, 256);
    p->off_whi = off; off = align_up(off + wplanes, 256);
    p->off_wlo = off; if (p->split) off = align_up(off + wplanes, 256);
    p->off_whi2 = off; if (half_planes) off = align_up(off + wplanes, 256);
    p->off_wlo2 = off; if (half_planes && p->split) off = align_up(off + wplanes, 256);
    p->off_whi4 = off; if (pair_tail) off = align_up(off + wplanes, 256);
    p->off_wlo4 = off; if (pair_tail && p->split) off = align_up(off + wplanes, 256);
    p->ws_end = off;

    SplitParams& sp = p->sp;
    sp = SplitParams{};
    sp.npix = k.npix;
    sp.npix_pad = k.npix_pad;
    sp.D = p->D; sp.nc = nc; sp.N = p->N; sp.fh = p->fh; sp.fw = p->fw; sp.nt = nt; sp.ntn = ntn;
    sp.split = p->split;
    sp.halves = half_planes ? 1 : 0;
    sp.quarters = pair_tail ? 1 : 0;
    sp.xblocks = (k.npix_pad + 255) / 256;
    const long long wblocks = ((long long)ntn * p->fh * p->fw * nc * nt + 255) / 256;
    if (c.fuse) sp.xblocks = 0;   // x is converted inside the correlation kernel
    p->split_blocks = (int)(sp.xblocks + wblocks);
    // one CTA per SM (the 512 TMEM columns); resident bank: a multiple of the
    // filter-tile count, each group of ntn CTAs sharing the pixel tiles
    if (c.sw)   // runs of output rows: the same number of runs in every column block
        p->grid = sw_delta * std::min(Ho, p->sm_count / sw_delta);
    else if (c.rs)
        p->grid = ntn * std::min(mtiles, std::max(1, p->sm_count / ntn));
    else if (c.cg)   // pairs of tiles, one pair of CTAs per pair of SMs
        p->grid = 2 * std::min((mtiles + 1) / 2, std::max(1, p->sm_count / 2));
    else
        p->grid = std::min(mtiles * ntn, std::max(1, p->sm_count));
    return true;
}

size_t tc_ws_need(TcPlan* p, const TcConfig& c) {
    TcPlan tmp;
    tmp.H = p->H; tmp.W = p->W; tmp.D = p->D; tmp.N = p->N; tmp.fh = p->fh; tmp.fw = p->fw;
    tmp.nc = p->nc; tmp.split = p->split; tmp.sm_count = p->sm_count;
    tmp.epi = p->epi;
    if (!tc_layout(&tmp, c, true)) return 0;
    return tmp.ws_end;
}

std::vector<TcConfig> tc_candidate_configs(TcPlan* p, bool pairs) {
    // widest filter tile first; within it raw-ring conversion, register
    // conversion, pre-pass; taps per stage from the most (fewest copies and
    // barrier handoffs) down, each with the deepest B ring that fits.  Every
    // configuration is also offered with the tiled-store (ts = 32) epilogue, and
    // with eight epilogue warps with the staged (ts = 1) one, again with the
    // deepest ring beside their staging slots.
    std::vector<TcConfig> out;
    auto deepest = [&](TcConfig c) -> int {
        int best = 0;
        for (int nb = 2; nb <= 12; ++nb) {
            c.nb = nb;
            if (tc_layout(p, c, false)) best = nb;
        }
        return best;
    };
    const int widths[] = {256, 128};
    for (int ntmax : widths) {
        if (ntmax == 128 && p->N <= 128) continue;
        for (int fuse = 2; fuse >= 0; --fuse)
            for (int cw : fuse ? std::vector<int>{8, 4} : std::vector<int>{0}) {
                if (!fuse_ok(fuse, cw, p->D, p->nc, p->fw)) continue;
                for (int nr : fuse == 2 ? std::vector<int>{3, 2} : std::vector<int>{0})
                    for (int bt = std::min(p->fw, 5); bt >= 1; --bt)
                        for (int ew : {8, 4})
                            for (int na = 2; na <= 3; ++na) {
                                TcConfig c{na, 0, ntmax, bt, ew, fuse, nr, cw};
                                if ((c.nb = deepest(c))) out.push_back(c);
                                for (int ts : {1, 32}) {
                                    if (ew != 8 && ts == 1) continue;
                                    TcConfig t = c;
                                    t.ts = ts;
                                    t.sb = 1;
                                    if ((t.nb = deepest(t))) out.push_back(t);
                                }
                            }
            }
    }
    // CTA pairs (cg = 2): the same family over one 256-wide filter tile, each
    // CTA's B stages half as large (deeper rings in the same shared memory)
    if (pairs)
        for (int fuse = 2; fuse >= 0; --fuse)
            for (int cw : fuse ? std::vector<int>{8, 4} : std::vector<int>{0}) {
                if (!fuse_ok(fuse, cw, p->D, p->nc, p->fw)) continue;
                for (int nr : fuse == 2 ? std::vector<int>{3, 2} : std::vector<int>{0})
                    for (int bt = std::min(p->fw, 5); bt >= 1; --bt)
                        for (int ew : {8, 4})
                            for (int na = 2; na <= 3; ++na)
                                for (int ts : {0, 1, 32}) {
                                    if (ew != 8 && ts == 1) continue;
                                    TcConfig c{na, 0, 256, bt, ew, fuse, nr, cw};
                                    c.ts = ts;
                                    c.sb = ts ? 1 : 0;
                                    c.cg = 2;
                                    if ((c.nb = deepest(c))) out.push_back(c);
                                }
            }
    // sliding window (sw = 1): one 256-wide filter tile over runs of output rows,
    // the A ring fh or fh + 1 slabs deep, raw-ring or register conversion by 8
    // warps, tiled stores where they apply (direct stores otherwise)
    {
        const int ts = ts_ok(32, 1, p->W, p->N, 256) ? 32 : 0;
        for (int fuse = 2; fuse >= 1; --fuse) {
            if (!fuse_ok(fuse, 8, p->D, p->nc, p->fw)) continue;
            for (int bt : {5, 3, 2, 1}) {
                if (bt > p->fw) continue;
                for (int ew : {4, 8})
                    for (int na = p->fh; na <= p->fh + 1; ++na) {
                        TcConfig c{na, 0, 256, bt, ew, fuse, fuse == 2 ? 3 : 0, 8};
                        c.ts = ts;
                        c.sb = ts ? 1 : 0;
                        c.sw = 1;
                        if ((c.nb = deepest(c))) out.push_back(c);
                    }
            }
        }
    }
    // resident bank (rs = 1): the ring holds all fh * ceil(fw / bt) stages of a
    // filter tile, loaded once per CTA; offered wherever a filter tile fits in
    // shared memory beside the A slots (plain BF16 of the headline shape: 128
    // filters of 5x5x32 = 200 KB)
    for (int ntmax : widths)
        for (int fuse = 2; fuse >= 0; --fuse)
            for (int cw : fuse ? std::vector<int>{8, 4} : std::vector<int>{0}) {
                if (!fuse_ok(fuse, cw, p->D, p->nc, p->fw)) continue;
                for (int nr : fuse == 2 ? std::vector<int>{3, 2} : std::vector<int>{0})
                    for (int bt = std::min(p->fw, 5); bt >= 1; --bt)
                        for (int ew : {8, 4})
                            for (int na = 2; na <= 3; ++na)
                                for (int ts : {0, 1, 32}) {
                                    if (ew != 8 && ts == 1) continue;
                                    TcConfig c{na, 0, ntmax, bt, ew, fuse, nr, cw};
                                    c.ts = ts;
                                    c.sb = ts ? 1 : 0;
                                    c.rs = 1;
                                    c.nb = p->fh * ((p->fw + bt - 1) / bt);
                                    if (tc_layout(p, c, false)) out.push_back(c);
                                }
            }
    return out;
}

// CTA-pair configurations among the tuning candidates (FBCORR_TC_PAIR=0 leaves
// them out; a pair spec can still be set explicitly).
bool pairs_offered() { return env_str("FBCORR_TC_PAIR", "1") != "0"; }

std::string format_spec(const TcConfig& c) {
    char b[128];
    snprintf(b, sizeof b, "tcgen05:na=%d,nb=%d,nt=%d,bt=%d,ew=%d,fz=%d,nr=%d,cw=%d", c.na, c.nb, c.ntmax,
             c.bt, c.ew, c.fuse, c.nr, c.cw);
    std::string out = b;
    if (c.ts) out += ",ts=" + std::to_string(c.ts) + ",sb=" + std::to_string(c.sb);
    if (c.rs) out += ",rs=1";
    if (c.cg) out += ",cg=2";
    if (c.sw) out += ",sw=1";
    return out;
}

bool parse_tc_spec(const std::string& s, TcConfig* c) {
    TcConfig t;
    int used = 0;
    const int n = sscanf(s.c_str(), "tcgen05:na=%d,nb=%d,nt=%d,bt=%d,ew=%d,fz=%d,nr=%d,cw=%d%n", &t.na, &t.nb,
                         &t.ntmax, &t.bt, &t.ew, &t.fuse, &t.nr, &t.cw, &used);
    if (n != 8) return false;
    // optional suffixes, in this order: staged / tiled stores, resident bank, CTA pairs
    int used2 = 0;
    if (sscanf(s.c_str() + used, ",ts=%d,sb=%d%n", &t.ts, &t.sb, &used2) == 2) {
        if ((t.ts != 32 && t.ts != 1) || t.sb < 1 || t.sb > 3 || (t.ts == 1 && t.sb != 1)) return false;
        used += used2;
    }
    if (s.compare(used, 5, ",rs=1") == 0) {
        t.rs = 1;
        used += 5;
    }
    if (s.compare(used, 5, ",cg=2") == 0) {
        t.cg = 2;
        used += 5;
    }
    if (s.compare(used, 5, ",sw=1") == 0) {
        t.sw = 1;
        used += 5;
    }
    if (t.rs && t.cg) return false;
    if (t.sw && (t.rs || t.cg)) return false;
    if (used != (int)s.size()) return false;
    if ((t.fuse == 0) != (t.cw == 0) || (t.cw != 0 && t.cw != 4 && t.cw != 8)) return false;
    if (t.fuse < 0 || t.fuse > 2 || (t.ew != 4 && t.ew != 8)) return false;
    if ((t.fuse == 2) != (t.nr > 0) || t.nr < 0 || t.nr > 4) return false;
    if (t.ntmax != 256 && t.ntmax != 128 && t.ntmax != 64) return false;
    *c = t;
    return true;
}

// The generated kernel of configuration `c` (compiled or taken from the caches).
fbcorr_status_t tc_kernel(TcPlan* p, const TcConfig& c, Kernel* out) {
    const std::string name = tc_kernel_name(p->nc, p->split, p->fw, c, p->snippet);
    auto it = p->kernels.find(name);
    if (it != p->kernels.end()) {
        *out = it->second;
        return FBCORR_OK;
    }
    Kernel k;
    FBC_TRY(rtcg_kernel(tc_kernel_source(p->nc, p->split, p->fw, c, p->snippet), name, kSmemMax, tc_threads(c), &k));
    p->kernels[name] = k;
    *out = k;
    return FBCORR_OK;
}

}  // namespace

std::string tc_spec(const TcPlan* p) { return format_spec(p->cfg); }

std::vector<std::string> tc_candidates(TcPlan* p) {
    std::vector<std::string> out;
    for (const auto& c : tc_candidate_configs(p, pairs_offered())) out.push_back(format_spec(c));
    return out;
}

fbcorr_status_t tc_precompile(TcPlan* p, const std::vector<std::string>& specs) {
    std::vector<std::string> srcs;
    std::map<std::string, bool> seen;
    for (const auto& s : specs) {
        TcConfig c;
        if (!parse_tc_spec(s, &c)) continue;
        const std::string name = tc_kernel_name(p->nc, p->split, p->fw, c, p->snippet);
        if (seen[name]) continue;
        seen[name] = true;
        srcs.push_back(tc_kernel_source(p->nc, p->split, p->fw, c, p->snippet));
    }
    return rtcg_precompile(srcs);
}

fbcorr_status_t tc_set_spec(TcPlan* p, const std::string& spec) {
    TcConfig c;
    if (!parse_tc_spec(spec, &c)) return set_error(FBCORR_ERR_INVALID_ARG, "unknown tcgen05 spec '%s'", spec.c_str());
    if (!tc_layout(p, c, false) || tc_ws_need(p, c) > p->ws_bytes)
        return set_error(FBCORR_ERR_UNSUPPORTED, "tcgen05 spec '%s' does not fit this shape", spec.c_str());
    Kernel k;
    FBC_TRY(tc_kernel(p, c, &k));
    tc_layout(p, c, true);
    return FBCORR_OK;
}

fbcorr_status_t tc_plan_create(TcPlan** out, int H, int W, int D, int N, int fh, int fw, int split,
                               int epi, float lo, float hi, const std::string& snippet, const DeviceInfo& dev) {
    *out = nullptr;
    if ((D + 15) / 16 * 16 / 8 > 8)
        return set_error(FBCORR_ERR_UNSUPPORTED,
                         "tensor-core modes support depth D <= 64 (got %d); use FBCORR_F32", D);
    TcPlan* p = new (std::nothrow) TcPlan();
    if (!p) return set_error(FBCORR_ERR_OOM, "host allocation failed");
    p->H = H; p->W = W; p->D = D; p->N = N; p->fh = fh; p->fw = fw;
    p->nc = (D + 15) / 16 * 16 / 8;
    p->split = split; p->epi = epi; p->lo = lo; p->hi = hi;
    p->snippet = snippet;
    p->sm_count = dev.sm_count;
    const long long wait_ms = atoll(env_str("FBCORR_WAIT_MS", "4000").c_str());
    p->wait_ns = (unsigned long long)std::max(1LL, wait_ms) * 1000000ull;
    p->drop_b = fault_injected("tcdrop") ? 0 : -1;   // the first B stage: every CTA has one
    // the workspace covers every configuration, CTA pairs included
    const std::vector<TcConfig> cands = tc_candidate_configs(p, true);
    if (cands.empty()) {
        delete p;
        return set_error(FBCORR_ERR_UNSUPPORTED, "shape needs more shared memory than one SM has");
    }
    for (const auto& c : cands) p->ws_bytes = std::max(p->ws_bytes, tc_ws_need(p, c));
    // default: the first candidate (widest filter tile, raw-ring conversion where
    // possible, most taps per stage, two A slots, deepest B ring)
    const fbcorr_status_t s = tc_set_spec(p, format_spec(cands.front()));
    if (s != FBCORR_OK) {
        delete p;
        return s;
    }
    logf("tc plan: nc=%d nt=%d ntn=%d mtiles=%d lp=%d na=%d nb=%d smem=%zu ws=%zu grid=%d", p->nc,
         p->kp.nt, p->kp.ntn, p->kp.mtiles, p->kp.lp, p->kp.na, p->kp.nb, p->smem, p->ws_bytes, p->grid);
    *out = p;
    return FBCORR_OK;
}

void tc_plan_destroy(TcPlan* p) { delete p; }

size_t tc_workspace_bytes(const TcPlan* p) { return p->ws_bytes; }

int tc_launches(const TcPlan*) { return 2; }

std::string tc_describe(const TcPlan* p) {
    std::ostringstream o;
    o << "{\"precision\":\"" << (p->split ? "bf16x3" : "bf16") << "\",\"mma\":\""
      << (p->cfg.cg ? "256x" : "128x") << p->kp.nt << "x16" << (p->cfg.cg ? " (CTA pair)" : "")
      << "\",\"filter_tiles\":" << p->kp.ntn << ",\"tiles\":" << p->kp.mtiles * p->kp.ntn
      << ",\"tail_half_tiles\":"
      << (p->cfg.cg ? 2 * ((p->kp.mtiles + 1) / 2 - p->kp.nfull)
                    : p->kp.mtiles * p->kp.ntn - std::min(p->kp.nfull, p->kp.mtiles * p->kp.ntn))
      << ",\"smem\":" << p->smem << ",\"grid\":" << p->grid << ",\"threads\":" << tc_threads(p->cfg)
      << ",\"kernel\":\"" << tc_kernel_name(p->nc, p->split, p->fw, p->cfg, p->snippet) << "\"";
    auto it = p->kernels.find(tc_kernel_name(p->nc, p->split, p->fw, p->cfg, p->snippet));
    if (it != p->kernels.end()) o << ",\"source_hash\":\"" << hex64(it->second.src_hash) << "\"";
    o << "}";
    return o.str();
}

fbcorr_status_t tc_forward(TcPlan* p, const float* x, const float* w, float* y, void* ws,
                           int* err_word, cudaStream_t s, cudaEvent_t ev_start, cudaEvent_t ev_stop) {
    Kernel k;
    FBC_TRY(tc_kernel(p, p->cfg, &k));
    k.smem = p->smem;
    uint8_t* base = static_cast<uint8_t*>(ws);
    SplitParams sp = p->sp;
    sp.x = x;
    sp.w = w;
    sp.xhi = base + p->off_xhi;
    sp.xlo = base + p->off_xlo;
    sp.whi = base + p->off_whi;
    sp.wlo = base + p->off_wlo;
    sp.whi2 = base + p->off_whi2;
    sp.wlo2 = base + p->off_wlo2;
    sp.whi4 = base + p->off_whi4;
    sp.wlo4 = base + p->off_wlo4;
    // timing events bracket both launches of the step: an event between them
    // would hold the correlation kernel back until the split has finished
    if (ev_start) FBC_CUDA(cudaEventRecord(ev_start, s));
    fbc_tc_split<<<p->split_blocks, 256, 0, s>>>(sp);
    FBC_CUDA(cudaGetLastError());
    FbcTcParams kp = p->kp;
    kp.xhi = sp.xhi;
    kp.xlo = sp.xlo;
    kp.whi = sp.whi;
    kp.wlo = sp.wlo;
    kp.whi2 = sp.whi2;
    kp.wlo2 = sp.wlo2;
    kp.whi4 = sp.whi4;
    kp.wlo4 = sp.wlo4;
    kp.y = y;
    kp.err = err_word;
    kp.xraw = x;
    kp.tma_y = 0;
    if (p->cfg.ts > 1) {
        // y as {N, W', H'}: pixels q >= W' and filters n >= N of a box are clipped;
        // a y that is not 16-byte aligned keeps the direct stores
        if (p->map_y != y) {
            const unsigned long long dims[3] = {(unsigned long long)p->N, (unsigned long long)p->kp.Wo,
                                                (unsigned long long)p->kp.Ho};
            const unsigned long long strides[2] = {(unsigned long long)p->N * 4,
                                                   (unsigned long long)p->N * p->kp.Wo * 4};
            const unsigned box[3] = {32, (unsigned)p->cfg.ts, 1};
            p->map_ok = (reinterpret_cast<uintptr_t>(y) & 15) == 0 &&
                        encode_f32_store_map(p->map, y, dims, strides, box);
            p->map_y = y;
        }
        if (p->map_ok) {
            memcpy(kp.ymap, p->map, sizeof kp.ymap);
            kp.tma_y = 1;
        }
    }
    void* args[] = {&kp};
    // dependent launch: the prologue (barriers, TMEM, converters' first rows)
    // overlaps the operand split
    FBC_TRY(launch_dependent(k, dim3(p->grid), args, s));
    if (ev_stop) FBC_CUDA(cudaEventRecord(ev_stop, s));
    return FBCORR_OK;
}

fbcorr_status_t tc_rtcg_check(int D, int fw, const std::string& spec, std::string* log) {
    TcConfig c;
    if (!parse_tc_spec(spec, &c)) return set_error(FBCORR_ERR_INVALID_ARG, "unknown tcgen05 spec '%s'", spec.c_str());
    const int nc = (D + 15) / 16 * 16 / 8;
    if (nc > 8) return set_error(FBCORR_ERR_UNSUPPORTED, "tensor-core modes support depth D <= 64");
    if (!fuse_ok(c.fuse, c.cw, D, nc, fw))
        return set_error(FBCORR_ERR_UNSUPPORTED, "fused conversion does not fit this shape");
    if (c.bt < 1 || c.bt > fw) return set_error(FBCORR_ERR_UNSUPPORTED, "taps per stage out of range");
    for (int split = 0; split <= 1; ++split)
        FBC_TRY(rtcg_compile_only(tc_kernel_source(nc, split, fw, c, ""), log));
    return FBCORR_OK;
}

fbcorr_status_t tc_snippet_check(int D, int fw, int split, const std::string& snippet, std::string* log) {
    const int nc = (D + 15) / 16 * 16 / 8;
    if (nc > 8) return set_error(FBCORR_ERR_UNSUPPORTED, "tensor-core modes support depth D <= 64");
    TcConfig c;   // the pre-pass configuration: valid for every shape
    c.na = 2; c.nb = 2; c.ntmax = 256; c.bt = 1; c.ew = 4; c.fuse = 0; c.nr = 0; c.cw = 0;
    return rtcg_compile_only(tc_kernel_source(nc, split, fw, c, snippet), log);
}

}  // namespace fbc
