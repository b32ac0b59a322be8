// variants.cu -- the space of generated kernel variants and the source text
// handed to NVRTC for each of them.
//
// The paper's auto-tuner searches "unique combinations of loop unrolling
// depth, register spilling, block/grid dimensions, thread work size, shared
// memory padding" (Sec. 6.2).  On sm_103a the corresponding knobs of the
// direct FP32 kernel are the thread work size TR x TF (output rows x output
// channels per thread, i.e. the register block), the CTA shape WR x WF warps,
// and -- fixed per plan -- the filter size and depth that NVRTC unrolls.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <sstream>

#include "internal.h"

namespace fbc {

#include "_embedded_src.inc"   // the texts of the NVRTC kernel sources

const char* rtcg_header_source() { return kRtcgDirectSrc; }
const char* rtcg_tc_params_source() { return kRtcgTcParamsSrc; }
const char* rtcg_ptx_source() { return kRtcgPtxSrc; }
const char* rtcg_tc_source() { return kRtcgTcSrc; }
const char* rtcg_nn_params_source() { return kRtcgNnParamsSrc; }
const char* rtcg_nn_source() { return kRtcgNnSrc; }

size_t direct_smem_bytes(const DirectTile& t, int fh, int fw, int c) {
    if (t.ks_chunked()) {
        // FbcDirectKSC: a ring of (halo [HR][HC][CP] + bank [fh][fw][cc][BNP]) stages
        const long cp = t.cc + (((t.ks - t.cc) % 32) + 32) % 32;
        const long bn = t.bn();
        const long bnp = ((bn / 4) % 2 == 1) ? bn : bn + 4;
        const long hr = t.bh() + fh - 1, hc = t.bw() + fw - 1;
        return (size_t)(t.pf ? 3 : 2) * (size_t)(hr * hc * cp + (long)fh * fw * t.cc * bnp) * 4;
    }
    if (t.ks > 1) {
        // FbcDirectKS: halo [HR][HC][CP] + bank [fh][fw][CPAD][BNP]
        const long cpad = (c + t.ks - 1) / t.ks * t.ks;
        const long cp = cpad + (((t.ks - cpad) % 32) + 32) % 32;
        const long bn = t.bn();
        const long bnp = ((bn / 4) % 2 == 1) ? bn : bn + 4;
        const long hr = t.bh() + fh - 1, hc = t.bw() + fw - 1;
        return (size_t)(hr * hc * cp + (long)fh * fw * cpad * bnp) * 4;
    }
    const long cc = t.chunk(c);
    const long bh = t.tr * t.wr, bn = t.tf * t.wf;
    const long hr = bh + fh - 1, hc = 32 + fw - 1;
    const long colp = (hc % 2 == 1) ? hc : hc + 1;
    const long bnp = bn + 4;
    const long xs = ((hr * cc * colp + 3) / 4) * 4;
    const long ws = (long)fh * fw * cc * bnp;
    return (size_t)(xs + ws) * 4;
}

std::string direct_tile_spec(const DirectTile& t) {
    char b[128];
    snprintf(b, sizeof b, "direct:tr=%d,tf=%d,wr=%d,wf=%d,cc=%d%s%s", t.tr, t.tf, t.wr, t.wf, t.cc,
             t.pk ? ",pk=1" : "", t.pf ? ",pf=1" : "");
    std::string out = b;
    if (t.ks > 1) out += ",ks=" + std::to_string(t.ks) + ",wq=" + std::to_string(t.wq);
    if (t.sh) out += ",sh=1";
    if (t.mb) out += ",mb=" + std::to_string(t.mb);
    return out;
}

static bool ks_tile_ok(const DirectTile& t) {
    if (t.ks == 1) return t.wq == 1 && t.sh == 0;
    if (t.ks_chunked())   // chunks of cc channels, cc / ks of them per lane
        return (t.ks == 4 || t.ks == 8 || t.ks == 16) && t.sh == 0 && t.cc % t.ks == 0 && t.cc % 4 == 0 &&
               t.cc / t.ks <= 4 && t.wq >= 1 && t.wq <= 32;
    if (t.pf) return false;   // the K-split tile stages the whole depth once
    if (t.sh != 0 && t.sh != 1) return false;
    if (t.ks != 4 && t.ks != 8 && t.ks != 16 && t.ks != 32) return false;
    // whole depth in one stage; the register block splits evenly over the ks lanes
    return t.cc == 0 && t.wq >= 1 && t.wq <= 32 && (t.tr * t.tf / 2) % t.ks == 0;
}

bool parse_direct_spec(const std::string& s, DirectTile* t) {
    // "direct:tr=R,tf=F,wr=WR,wf=WF" then optionally ",cc=CC", ",pk=P", ",pf=F",
    // ",ks=K,wq=Q", ",sh=S" and ",mb=M", in that order; anything else left over
    // rejects the spec
    DirectTile d;
    d.cc = 0;
    d.pk = 0;
    int used = -1;
    if (sscanf(s.c_str(), "direct:tr=%d,tf=%d,wr=%d,wf=%d%n", &d.tr, &d.tf, &d.wr, &d.wf, &used) != 4 ||
        used < 0)
        return false;
    const char* rest = s.c_str() + used;
    int u = -1;
    if (strncmp(rest, ",cc=", 4) == 0) {
        if (sscanf(rest, ",cc=%d%n", &d.cc, &u) != 1 || u < 0) return false;
        rest += u;
    }
    u = -1;
    if (strncmp(rest, ",pk=", 4) == 0) {
        if (sscanf(rest, ",pk=%d%n", &d.pk, &u) != 1 || u < 0) return false;
        rest += u;
    }
    u = -1;
    if (strncmp(rest, ",pf=", 4) == 0) {
        if (sscanf(rest, ",pf=%d%n", &d.pf, &u) != 1 || u < 0 || (d.pf != 0 && d.pf != 1)) return false;
        rest += u;
    }
    u = -1;
    if (strncmp(rest, ",ks=", 4) == 0) {
        if (sscanf(rest, ",ks=%d,wq=%d%n", &d.ks, &d.wq, &u) != 2 || u < 0) return false;
        rest += u;
    }
    u = -1;
    if (strncmp(rest, ",sh=", 4) == 0) {
        if (sscanf(rest, ",sh=%d%n", &d.sh, &u) != 1 || u < 0) return false;
        rest += u;
    }
    u = -1;
    if (strncmp(rest, ",mb=", 4) == 0) {
        if (sscanf(rest, ",mb=%d%n", &d.mb, &u) != 1 || u < 0 || d.mb < 2 || d.mb > 4) return false;
        rest += u;
    }
    if (*rest != '\0') return false;
    if (!ks_tile_ok(d)) return false;
    if (d.tr < 1 || d.tr > 16 || (d.tf != 4 && d.tf != 8 && d.tf != 12 && d.tf != 16) ||
        d.wr < 1 || d.wf < 1 || d.threads() > 1024 || d.cc < 0 || d.cc > 4096 || d.pk < 0 || d.pk > 1)
        return false;
    *t = d;
    return true;
}

std::string snippet_definition(const std::string& expr) {
    if (expr.empty()) return "";
    return "__device__ float fbc_user_epi(float y, int n, float lo, float hi) {\n"
           "  (void)y; (void)n; (void)lo; (void)hi;\n  return (float)(" + expr + ");\n}\n";
}

std::string snippet_tag(const std::string& expr) {
    uint32_t h = 2166136261u;   // FNV-1a
    for (unsigned char c : expr) {
        h ^= c;
        h *= 16777619u;
    }
    char b[16];
    snprintf(b, sizeof b, "%08x", h);
    return b;
}

std::string direct_kernel_source(const DirectProblem& pr, const DirectTile& t,
                                 const std::string& kname) {
    std::ostringstream o;
    o << rtcg_header_source() << "\n";
    if (pr.epi == 2) o << snippet_definition(pr.snippet);
    if (t.ks_chunked()) {
        // the chunked K-split tile (dL/dx only: callers check flip == 1, mask == 0)
        o << "typedef FbcDirectKSC<" << pr.fh << "," << pr.fw << "," << pr.c << "," << t.tr << "," << t.tf << ","
          << t.ks << "," << t.wq << "," << t.wr << "," << t.wf << "," << t.cc << "," << (t.pf ? 3 : 2) << ","
          << t.pk << "> FbcThis;\n";
    } else if (t.ks > 1) {
        // the K-split tile (forward only: callers check flip == 0 and mask == 0)
        o << "typedef FbcDirectKS<" << pr.fh << "," << pr.fw << "," << pr.c << "," << t.tr << "," << t.tf << ","
          << t.ks << "," << t.wq << "," << t.wr << "," << t.wf << "," << pr.epi << "," << t.pk << "," << t.sh
          << "> FbcThis;\n";
    } else {
        o << "typedef FbcDirect<" << pr.fh << "," << pr.fw << "," << pr.c << "," << t.tr << ","
          << t.tf << "," << t.wr << "," << t.wf << "," << pr.flip << "," << pr.epi << "," << pr.mask
          << "," << t.chunk(pr.c) << "," << t.pk << "," << t.pf << "> FbcThis;\n";
    }
    o << "static_assert(FbcThis::SMEM_BYTES == " << direct_smem_bytes(t, pr.fh, pr.fw, pr.c)
      << ", \"host and device disagree on the shared-memory size\");\n";
    o << "extern \"C\" __global__ void __launch_bounds__(" << t.threads();
    if (t.mb) o << ", " << t.mb;
    o << ") " << kname << "(FbcDirectArgs a) {\n"
      << "  extern __shared__ __align__(16) float fbc_smem[];\n"
      // launched as a programmatic dependent: nothing the previous kernel of
      // the stream may still read or write is touched before its grid has
      // completed, and the next kernel may begin launching at once
      << "  asm volatile(\"griddepcontrol.wait;\" ::: \"memory\");\n"
      << "  asm volatile(\"griddepcontrol.launch_dependents;\" ::: \"memory\");\n"
      << "  FbcThis::run(a, fbc_smem, blockIdx.x, blockIdx.y, blockIdx.z);\n"
      << "}\n";
    return o.str();
}

size_t dw_smem_bytes(int fw, int c, int tn, int ng, int qb, int pk) {
    // two (g, x) buffers, plus the chunk totals of every thread for pk = 2
    return (2 * (size_t)(qb * tn * ng + (qb + fw - 1) * c) + (pk == 2 ? (size_t)tn * fw * c * ng : 0)) * 4;
}

std::string dw_kernel_source(int fh, int fw, int c, int tn, int ng, int qb, int mask, int pk,
                             const std::string& kname, int min_blocks) {
    std::ostringstream o;
    o << rtcg_header_source() << "\n";
    o << "typedef FbcDw<" << fh << "," << fw << "," << c << "," << tn << "," << ng << "," << qb << ","
      << mask << "," << pk << "> FbcDwThis;\n";
    o << "static_assert(FbcDwThis::SMEM_BYTES == " << dw_smem_bytes(fw, c, tn, ng, qb, pk)
      << ", \"host and device disagree on the shared-memory size\");\n";
    o << "extern \"C\" __global__ void __launch_bounds__(" << c * ng;
    if (min_blocks > 0) o << ", " << min_blocks;
    o << ") " << kname
      << "(FbcDwArgs a) {\n"
      << "  extern __shared__ __align__(16) float fbc_smem[];\n"
      << "  FbcDwThis::run(a, fbc_smem, blockIdx.x, blockIdx.y, blockIdx.z);\n"
      << "}\n";
    return o.str();
}

namespace {
int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// How evenly `ctas` CTAs spread over the SMs, `res` resident per SM: within one
// round the busiest SM runs ceil(ctas / sms) of them against an average of
// ctas / sms; beyond one round, whole rounds of res * sms CTAs.
double wave_balance(long ctas, int res, int sms) {
    const long slots = (long)res * sms;
    if (ctas <= slots) {
        const long per = (ctas + sms - 1) / sms;
        return ((double)ctas / sms) / (double)per;
    }
    const long waves = (ctas + slots - 1) / slots;
    return (double)ctas / (double)(waves * slots);
}
}  // namespace

// The chunked K-split tile's problem: dL/dx (flipped bank) without a clamp mask
// or epilogue, 16-byte rows of the gradient (c % 4 == 0) and of the bank's
// output-channel runs (nf % 4 == 0).
bool ks_chunked_fits(const DirectProblem& pr) {
    return pr.flip == 1 && pr.mask == 0 && pr.epi == 0 && pr.c % 4 == 0 && pr.nf % 4 == 0;
}

std::vector<DirectTile> direct_candidates(const DirectProblem& pr, size_t smem_limit, int threads,
                                          int max_block) {
    std::vector<DirectTile> out;
    // row blocks of 6 and 7 give grids that fill 152 SMs on 248- and 256-row
    // outputs (e.g. dL/dx of the differentiation workload: 8 x 19 = 152 CTAs)
    const int trs[] = {2, 4, 6, 7, 8};
    const int tfs[] = {4, 8};
    const int wrs[] = {1, 2, 3, 4, 5, 6, 7, 8};   // any count: block heights that fit 152 SMs better
    const int wfs[] = {1, 2, 4, 8};
    const int nf4 = ((pr.nf + 3) / 4) * 4;
    // channel chunks: the whole depth, or 16 / 8 / 4 channels per stage
    std::vector<int> ccs = {0};
    for (int cc : {16, 8, 4})
        if (cc < pr.c) ccs.push_back(cc);
    for (int tr : trs)
        for (int tf : tfs)
            for (int wr : wrs)
                for (int wf : wfs)
                    for (int cc : ccs) {
                        DirectTile t{tr, tf, wr, wf, cc};
                        if (t.threads() > 512) continue;
                        if (threads > 0 && t.threads() != threads) continue;
                        if (tf > nf4) continue;                       // no all-padding channels
                        if (t.bn() > nf4 && wf > 1) continue;
                        if (tr * tf > max_block) continue;            // register block
                        if (tr + pr.fh - 1 > 40) continue;            // input window registers
                        if (t.bh() > ((pr.out_h + 1) / 2) * 2 + 8 && wr > 1) continue;
                        if (direct_smem_bytes(t, pr.fh, pr.fw, pr.c) > smem_limit) continue;
                        out.push_back(t);
                    }
    // K-split tiles (forward only, not in the batched kernel's fixed CTA size):
    // ks lanes per output split the depth, at most a quarter of them on zero
    // padding channels and at most 8 channels per lane (deeper inputs keep the
    // lane-per-column tile busy enough)
    if (threads > 0 && (pr.flip || pr.mask)) return out;
    if (threads == 0 && ks_chunked_fits(pr)) {
        // chunked K-split tiles for dL/dx: chunks of cc = ks or 2 ks channels
        for (int ks : {4, 8})
            for (int cpl : {1, 2})
                for (int tr : {4, 6, 7, 8})
                    for (int tf : {4, 8})
                        for (int wq : {1, 2, 4})
                            for (int wr : {1, 2, 3, 4})
                                for (int wf : {1, 2, 4})
                                    for (int pf : {0, 1}) {
                                        DirectTile t{tr, tf, wr, wf, ks * cpl};
                                        t.ks = ks;
                                        t.wq = wq;
                                        t.pf = pf;
                                        if (t.cc > pr.c || t.threads() > 512 || t.threads() < 128) continue;
                                        if (tf > pr.nf || (t.bn() > pr.nf && wf > 1)) continue;
                                        if (tr * tf > max_block || tr + pr.fh - 1 > 40) continue;
                                        if (t.bw() > ((pr.out_w + 7) / 8) * 8 + 8 && wq > 1) continue;
                                        if (t.bh() > ((pr.out_h + 1) / 2) * 2 + 8 && wr > 1) continue;
                                        if (direct_smem_bytes(t, pr.fh, pr.fw, pr.c) > smem_limit) continue;
                                        out.push_back(t);
                                    }
        return out;
    }
    if (pr.flip || pr.mask) return out;
    // K-split tiles inside the batched kernel: offered to its tuner only with
    // FBCORR_TUNE_KS_BATCH=1 (measured on the 64-image batch: picked for 6 of 37
    // variants by their single-image timings, the batch 7.98 against 7.95 ms;
    // FBCORR_BATCH_KS=1, for tests and profiling, forces them)
    if (threads > 0 && env_str("FBCORR_TUNE_KS_BATCH", "0") != "1" && env_str("FBCORR_BATCH_KS", "0") != "1")
        return out;
    for (int ks : {4, 8, 16, 32}) {
        const int cpad = (pr.c + ks - 1) / ks * ks;
        if (4 * (cpad - pr.c) > cpad || cpad / ks > 8) continue;
        for (int tr : {2, 4, 8, 16})
            for (int tf : {4, 8, 16})
                for (int wq : {1, 2, 3, 4, 8})
                    for (int wr : {1, 2, 3, 4, 6, 8})
                        for (int wf : {1, 2, 4})
                            for (int sh : {0, 1}) {
                                DirectTile t{tr, tf, wr, wf, 0};
                                t.ks = ks;
                                t.wq = wq;
                                t.sh = sh;
                                if ((tr * tf / 2) % ks != 0 || t.threads() > 512 || t.threads() < 64) continue;
                                if (threads > 0 && t.threads() != threads) continue;   // the batch's CTA size
                                if (tf > nf4 || (t.bn() > nf4 && wf > 1)) continue;
                                if (tr * tf > max_block || tr + pr.fh - 1 > 40) continue;
                                if (t.bw() > ((pr.out_w + 7) / 8) * 8 + 8 && wq > 1) continue;
                                if (t.bh() > ((pr.out_h + 1) / 2) * 2 + 8 && wr > 1) continue;
                                if (direct_smem_bytes(t, pr.fh, pr.fw, pr.c) > smem_limit) continue;
                                out.push_back(t);
                            }
    }
    return out;
}

// A small analytic model: tile edge waste x wave quantisation x inner-loop
// issue efficiency (including the per-chunk staging) x latency hiding
// (resident warps).  The auto-tuner replaces it with measurements; it also
// orders the candidates the tuner measures first.
static double direct_score(const DirectProblem& pr, const DirectTile& t, int sm_count) {
    const size_t smem_per_sm = 228 * 1024;
    if (t.ks_chunked()) {
        // chunked K-split tile: tile edges and wave quantisation, the inner loop
        // of the K-split tile, a barrier per chunk, and latency hiding, which
        // wants about 16 warps per SM (the staging is asynchronous)
        const int gx = ceil_div(pr.out_w, t.bw()), gy = ceil_div(pr.out_h, t.bh()), gz = ceil_div(pr.nf, t.bn());
        const double useful = (double)pr.out_w * pr.out_h * pr.nf;
        const double computed = (double)gx * t.bw() * gy * t.bh() * gz * t.bn();
        const int nch = ceil_div(pr.c, t.cc);
        const double e_tile = useful / computed * pr.c / ((double)nch * t.cc);
        const size_t smem = direct_smem_bytes(t, pr.fh, pr.fw, pr.c) + 1024;
        const int regs = t.tr * t.tf + t.tr + pr.fh + t.tf + 40;
        int res = (int)(smem_per_sm / smem);
        res = std::min(res, 2048 / t.threads());
        res = std::min(res, 65536 / (t.threads() * std::min(255, regs)));
        if (res < 1) return -1.0;
        const long ctas = (long)gx * gy * gz;
        const double wave_eff = wave_balance(ctas, res, sm_count);
        const double fma_cyc = t.tr * t.tf * pr.fh / 4.0;
        const double lsu_cyc = (t.tr + pr.fh - 1) + pr.fh * t.tf;
        const double iss_cyc = (t.tr * t.tf * pr.fh / 2.0 + (t.tr + pr.fh - 1) + pr.fh * t.tf / 4.0) / 4.0;
        const double e_inner = fma_cyc / std::max(fma_cyc, std::max(lsu_cyc, iss_cyc));
        const double fma_chunk = (double)t.tr * t.tf * pr.fh * pr.fw * (t.cc / t.ks);
        const double e_issue = e_inner * fma_chunk / (fma_chunk + 300.0 + 4.0 * t.tr * t.tf / nch);
        const int warps = std::min<long>(res, (ctas + sm_count - 1) / sm_count) * t.threads() / 32;
        const double occ = std::min(1.0, warps / 16.0);
        return e_tile * wave_eff * e_issue * (0.4 + 0.6 * occ);
    }
    if (t.ks > 1) {
        // K-split tile: the same factors, with the depth split over ks lanes (a
        // share of them on zero padding), vectorised staging, and the shuffle
        // reduction of the register block at the end
        const int gx = ceil_div(pr.out_w, t.bw()), gy = ceil_div(pr.out_h, t.bh()), gz = ceil_div(pr.nf, t.bn());
        const double useful = (double)pr.out_w * pr.out_h * pr.nf;
        const double computed = (double)gx * t.bw() * gy * t.bh() * gz * t.bn();
        const int cpad = (pr.c + t.ks - 1) / t.ks * t.ks;
        const double e_tile = useful / computed * pr.c / cpad;
        const size_t smem = direct_smem_bytes(t, pr.fh, pr.fw, pr.c) + 1024;
        const int regs = t.tr * t.tf + t.tr + pr.fh + t.tf + 32;
        int res = (int)(smem_per_sm / smem);
        res = std::min(res, 2048 / t.threads());
        res = std::min(res, 65536 / (t.threads() * std::min(255, regs)));
        if (res < 1) return -1.0;
        const long ctas = (long)gx * gy * gz;
        const double wave_eff = wave_balance(ctas, res, sm_count);
        // inner loop per warp and (tap column, channel step), in SM cycles: the
        // FMA pipe (128 lanes), the shared-memory pipe (one wavefront per cycle:
        // one per input load, four per float4 filter load, whose lanes read
        // ks different channels) and instruction issue (4 per cycle)
        const int cpl = cpad / t.ks;
        const double fma_cyc = t.tr * t.tf * pr.fh / 4.0;
        const double lsu_cyc = (t.tr + pr.fh - 1) + pr.fh * t.tf;
        const double iss_cyc = (t.tr * t.tf * pr.fh / 2.0 + (t.tr + pr.fh - 1) + pr.fh * t.tf / 4.0) / 4.0;
        const double e_inner = fma_cyc / std::max(fma_cyc, std::max(lsu_cyc, iss_cyc));
        const double fma_total = (double)t.tr * t.tf * pr.fh * pr.fw * cpl;
        const double staged = ((double)(t.bh() + pr.fh - 1) * (t.bw() + pr.fw - 1) * pr.c +
                               (double)pr.fh * pr.fw * pr.c * t.bn()) / t.threads();
        const double reduce = 4.0 * t.tr * t.tf / 2.0;
        const double e_issue = e_inner * fma_total / (fma_total + 2.5 * staged + reduce + 400.0);
        const int warps = std::min<long>(res, (ctas + sm_count - 1) / sm_count) * t.threads() / 32;
        const double occ = std::min(1.0, warps / 12.0);
        return e_tile * wave_eff * e_issue * (0.5 + 0.5 * occ);
    }
    const int gx = ceil_div(pr.out_w, 32), gy = ceil_div(pr.out_h, t.bh()), gz = ceil_div(pr.nf, t.bn());
    const double useful = (double)pr.out_w * pr.out_h * pr.nf;
    const double computed = (double)gx * 32 * gy * t.bh() * gz * t.bn();
    const double e_tile = useful / computed;
    const size_t smem = direct_smem_bytes(t, pr.fh, pr.fw, pr.c) + 1024;
    const int regs = t.tr * t.tf + t.tr + pr.fh + t.tf + 28;
    int res = (int)(smem_per_sm / smem);
    res = std::min(res, 2048 / t.threads());
    res = std::min(res, 65536 / (t.threads() * std::min(255, regs)));
    if (res < 1) return -1.0;
    const long ctas = (long)gx * gy * gz;
    const double wave_eff = wave_balance(ctas, res, sm_count);
    const double loads = (t.tr + pr.fh - 1) + pr.fh * t.tf / 4.0 + 2.0;
    const double fmas = (double)t.tr * t.tf * pr.fh;
    const int cc = t.chunk(pr.c);
    const double staged = ((double)(t.bh() + pr.fh - 1) * (32 + pr.fw - 1) * cc +
                           (double)pr.fh * pr.fw * cc * t.bn()) / t.threads();
    const double fma_chunk = fmas * pr.fw * cc;
    const double e_issue = fma_chunk / (fma_chunk + loads * pr.fw * cc + 6.0 * staged + 400.0);
    const int warps = std::min<long>(res, (ctas + sm_count - 1) / sm_count) * t.threads() / 32;
    const double occ = std::min(1.0, warps / 12.0);
    return e_tile * wave_eff * e_issue * (0.5 + 0.5 * occ);
}

std::vector<DirectTile> direct_ranked(const DirectProblem& pr, size_t smem_limit, int sm_count,
                                      int threads, int max_block) {
    auto cands = direct_candidates(pr, smem_limit, threads, max_block);
    std::vector<std::pair<double, DirectTile>> scored;
    for (const auto& t : cands) {
        const double sc = direct_score(pr, t, sm_count);
        if (sc > 0) scored.push_back({sc, t});
    }
    std::stable_sort(scored.begin(), scored.end(),
                     [](const std::pair<double, DirectTile>& a, const std::pair<double, DirectTile>& b) {
                         return a.first > b.first;
                     });
    std::vector<DirectTile> out;
    for (auto& st : scored) out.push_back(st.second);
    return out;
}

std::vector<std::string> direct_tuning_specs(const std::vector<DirectTile>& ranked, int topk, int depth) {
    const bool twins = env_str("FBCORR_TUNE_PK", "1") != "0";
    const bool pf = depth > 0 && env_str("FBCORR_TUNE_PF", "1") != "0";
    std::vector<std::string> specs;
    // the first topk lane-per-column tiles and, beside them, the first topk / 2
    // K-split tiles (their model scores are not comparable enough to let one
    // family crowd out the other)
    int tiles = 0, ks_tiles = 0;
    for (const auto& t : ranked) {
        if (t.ks > 1 ? ks_tiles++ >= topk / 2 : tiles++ >= topk) continue;
        DirectTile a = t;
        a.pk = 0;
        specs.push_back(direct_tile_spec(a));
        if (twins) {
            a.pk = 1;
            specs.push_back(direct_tile_spec(a));
        }
        if (pf && a.ks == 1 && a.chunk(depth) < depth) {
            // several channel chunks: the register-prefetch form (packed pairs)
            a.pk = 1;
            a.pf = 1;
            specs.push_back(direct_tile_spec(a));
        }
    }
    return specs;
}

DirectTile direct_heuristic(const DirectProblem& pr, size_t smem_limit, int sm_count, int threads,
                            int max_block) {
    auto r = direct_ranked(pr, smem_limit, sm_count, threads, max_block);
    // the model does not rate the chunked K-split tile against the others (its
    // score is on another scale): only the tuner's measurements choose it;
    // likewise the K-split tile inside the batched kernel
    r.erase(std::remove_if(r.begin(), r.end(),
                           [threads](const DirectTile& c) { return c.ks_chunked() || (threads > 0 && c.ks > 1); }),
            r.end());
    DirectTile t = !r.empty() ? r.front() : (threads == 256 ? DirectTile{4, 4, 2, 4, 4} : DirectTile{4, 4, 1, 1, 4});
    // packed-pair FMAs: the same bits, and faster on most tiles measured on a
    // GB300 (median 0.91-0.93 of the scalar time across the top 48 tiles)
    t.pk = 1;
    return t;
}


// ---- building, launching and timing generated direct kernels -------------------

namespace {
// Host mirror of the NVRTC kernels' by-value argument struct (rtcg_direct.cuh).
struct DirectArgsK {
    const float* x;
    const float* m;
    const float* w;
    float* y;
    int in_h, in_w, out_h, out_w, nf;
    int pad_y, pad_x;
    float lo, hi;
};
}  // namespace

std::string kname_for(const char* base, const DirectProblem& pr, const DirectTile& t) {
    char b[160];
    snprintf(b, sizeof b, "%s_f%dx%d_c%d_t%d_%d_%d_%d_cc%d_fl%d_e%d_m%d%s", base, pr.fh, pr.fw, pr.c,
             t.tr, t.tf, t.wr, t.wf, t.chunk(pr.c), pr.flip, pr.epi, pr.mask, t.pk ? "_pk1" : "");
    std::string name = b;
    if (t.pf) name += "_pf1";
    if (t.ks > 1) name += "_ks" + std::to_string(t.ks) + "q" + std::to_string(t.wq) + (t.sh ? "h" : "");
    if (t.mb) name += "_mb" + std::to_string(t.mb);
    return pr.epi == 2 ? name + "_u" + snippet_tag(pr.snippet) : name;
}

size_t smem_limit(const DeviceInfo& dev) {
    return std::min<size_t>(dev.smem_optin ? dev.smem_optin : 227 * 1024, 200 * 1024);
}

fbcorr_status_t build_direct(const DirectProblem& pr, const DirectTile& t, Kernel* k) {
    if (t.ks_chunked() && !ks_chunked_fits(pr))
        return set_error(FBCORR_ERR_UNSUPPORTED,
                         "chunked K-split tiles compute dL/dx without a clamp mask, with depth and filter count "
                         "multiples of 4");
    if (t.ks > 1 && !t.ks_chunked() && (pr.flip || pr.mask))
        return set_error(FBCORR_ERR_UNSUPPORTED, "K-split tiles compute the forward correlation only");
    const std::string name = kname_for("fbc_direct", pr, t);
    const std::string src = direct_kernel_source(pr, t, name);
    return rtcg_kernel(src, name, direct_smem_bytes(t, pr.fh, pr.fw, pr.c), t.threads(), k);
}

dim3 direct_grid(const DirectProblem& pr, const DirectTile& t) {
    return dim3((unsigned)((pr.out_w + t.bw() - 1) / t.bw()), (unsigned)((pr.out_h + t.bh() - 1) / t.bh()),
                (unsigned)((pr.nf + t.bn() - 1) / t.bn()));
}

fbcorr_status_t run_direct(const Kernel& k, const DirectProblem& pr, const DirectTile& t,
                           const float* x, const float* m, const float* w, float* y, float lo,
                           float hi, cudaStream_t s) {
    DirectArgsK a{x, m, w, y, pr.in_h, pr.in_w, pr.out_h, pr.out_w, pr.nf, pr.pad_y, pr.pad_x, lo, hi};
    void* args[] = {&a};
    return launch_dependent(k, direct_grid(pr, t), args, s);
}

fbcorr_status_t run_default(const DirectProblem& pr, const float* x, const float* m,
                            const float* w, float* y, float lo, float hi, cudaStream_t s) {
    DirectArgsRT a{x, m, w, y, pr.in_h, pr.in_w, pr.c, pr.out_h, pr.out_w, pr.nf, pr.fh, pr.fw,
                   pr.pad_y, pr.pad_x, pr.flip, pr.epi, pr.mask, lo, hi};
    FBC_CUDA(launch_default_direct(a, s));
    return FBCORR_OK;
}


fbcorr_status_t tune_direct_problem(const DeviceInfo& dev, const DirectProblem& pr, cudaStream_t s,
                                    int threads, int max_block, size_t smem_cap, int topk,
                                    bool include_default, const char* what, std::string* best_spec,
                                    float* best_ms_out) {
    // Time the top candidates of one direct-correlation problem (and, when asked,
    // the prebuilt default kernel) on patterned buffers; keep the fastest.
    std::vector<DirectTile> ranked = direct_ranked(pr, smem_cap, dev.sm_count, threads, max_block);
    // the batched kernel (fixed CTA size, two CTAs per SM) takes no prefetch variants
    std::vector<std::string> specs = direct_tuning_specs(ranked, topk, threads > 0 ? 0 : pr.c);
    if (threads == 0 && env_str("FBCORR_TUNE_MB", "1") != "0") {
        // occupancy variants: the packed-pair form of the first candidates bounded
        // to 2 or 3 CTAs per SM (registers, where the shared memory allows it), so
        // that one CTA stages while the others compute
        const size_t n0 = specs.size();
        int added = 0;
        for (size_t i = 0; i < n0 && added < topk / 2; ++i) {
            DirectTile t;
            if (!parse_direct_spec(specs[i], &t) || t.pk != 1) continue;
            const size_t sm = direct_smem_bytes(t, pr.fh, pr.fw, pr.c) + 1024;
            for (int mb = 2; mb <= 3; ++mb)
                if ((size_t)mb * sm <= 228 * 1024 && (size_t)mb * t.threads() <= 2048) {
                    DirectTile u = t;
                    u.mb = mb;
                    specs.push_back(direct_tile_spec(u));
                    ++added;
                }
        }
    }
    if (specs.empty() && !include_default)
        return set_error(FBCORR_ERR_UNSUPPORTED, "no %s candidate fits", what);
    {
        // compile every candidate in parallel before timing them one by one
        std::vector<std::string> srcs;
        for (const auto& sp : specs) {
            DirectTile t;
            if (parse_direct_spec(sp, &t)) srcs.push_back(direct_kernel_source(pr, t, kname_for("fbc_direct", pr, t)));
        }
        rtcg_precompile(srcs);
    }
    if (include_default) specs.push_back("default");
    const size_t xb = (size_t)pr.in_h * pr.in_w * pr.c * 4;
    const size_t wb = (size_t)pr.nf * pr.fh * pr.fw * pr.c * 4;
    const size_t yb = (size_t)pr.out_h * pr.out_w * pr.nf * 4;
    float *x = nullptr, *w = nullptr, *y = nullptr, *m = nullptr;
    if (cudaMalloc(&x, xb) != cudaSuccess || cudaMalloc(&w, wb) != cudaSuccess ||
        cudaMalloc(&y, yb) != cudaSuccess || (pr.mask && cudaMalloc(&m, xb) != cudaSuccess)) {
        cudaFree(x); cudaFree(w); cudaFree(y); cudaFree(m);
        cudaGetLastError();
        return set_error(FBCORR_ERR_OOM, "autotune buffers");
    }
    // patterned, non-zero operands, as for the tensor-core candidates
    launch_fill_pattern(x, xb / 4, 1.0f, 0x1234u, s);
    launch_fill_pattern(w, wb / 4, 0.05f, 0x5678u, s);
    if (m) launch_fill_pattern(m, xb / 4, 1.0f, 0x9abcu, s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    best_spec->clear();
    fbcorr_status_t status = FBCORR_OK;
    std::vector<std::pair<float, std::string>> timed;   // (median single-launch ms, spec)
    for (const auto& sp : specs) {
        Kernel k;
        DirectTile t;
        const bool dflt = sp == "default";
        if (!dflt && (!parse_direct_spec(sp, &t) || build_direct(pr, t, &k) != FBCORR_OK)) continue;
        auto run = [&]() {
            return dflt ? run_default(pr, x, m, w, y, 0.f, 1.f, s)
                        : run_direct(k, pr, t, x, m, w, y, 0.f, 1.f, s);
        };
        std::vector<float> ms_list;
        bool ok = true;
        for (int r = 0; r < 2 && ok; ++r) ok = run() == FBCORR_OK;
        for (int r = 0; r < 7 && ok; ++r) {
            cudaEventRecord(e0, s);
            ok = run() == FBCORR_OK;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms_list.push_back(ms);
        }
        if (!ok) {
            status = set_error(FBCORR_ERR_CUDA, "autotune run of %s (%s) failed", sp.c_str(), what);
            break;
        }
        std::sort(ms_list.begin(), ms_list.end());
        const float med = ms_list[ms_list.size() / 2];
        logf("autotune %s %s: %.4f ms", what, sp.c_str(), med);
        timed.push_back({med, sp});
    }
    // Finalists: the six fastest timed again, round-robin over three rounds, as
    // runs of 10 back-to-back launches (single launches separate them within
    // their noise); the best round of each decides.
    if (status == FBCORR_OK && !timed.empty()) {
        std::sort(timed.begin(), timed.end());
        const size_t nf = std::min<size_t>(timed.size(), 6);
        std::vector<float> fin(nf, 1e30f);
        std::vector<Kernel> fk(nf);
        std::vector<DirectTile> ft(nf);
        std::vector<bool> fdef(nf, false);
        for (size_t f = 0; f < nf; ++f) {
            fdef[f] = timed[f].second == "default";
            if (!fdef[f] && (!parse_direct_spec(timed[f].second, &ft[f]) || build_direct(pr, ft[f], &fk[f]) != FBCORR_OK))
                fin[f] = 2e30f;   // not re-timed
        }
        for (int round = 0; round < 3 && status == FBCORR_OK; ++round)
            for (size_t f = 0; f < nf; ++f) {
                if (fin[f] > 1.5e30f) continue;
                auto run = [&]() {
                    return fdef[f] ? run_default(pr, x, m, w, y, 0.f, 1.f, s)
                                   : run_direct(fk[f], pr, ft[f], x, m, w, y, 0.f, 1.f, s);
                };
                bool ok = run() == FBCORR_OK;
                cudaEventRecord(e0, s);
                for (int r = 0; r < 10 && ok; ++r) ok = run() == FBCORR_OK;
                cudaEventRecord(e1, s);
                if (!ok || cudaEventSynchronize(e1) != cudaSuccess) {
                    status = set_error(FBCORR_ERR_CUDA, "autotune run of %s (%s) failed", timed[f].second.c_str(), what);
                    break;
                }
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                fin[f] = std::min(fin[f], t / 10.f);
            }
        for (size_t f = 0; f < nf; ++f) {
            if (fin[f] > 1.5e30f) continue;
            logf("autotune %s finalist %s: %.4f ms", what, timed[f].second.c_str(), fin[f]);
            if (fin[f] < best_ms) {
                best_ms = fin[f];
                *best_spec = timed[f].second;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(x); cudaFree(w); cudaFree(y); cudaFree(m);
    if (status != FBCORR_OK) return status;
    if (best_spec->empty()) return set_error(FBCORR_ERR_INTERNAL, "no %s variant ran", what);
    if (best_ms_out) *best_ms_out = best_ms;
    return FBCORR_OK;
}

}  // namespace fbc
