// batched.cu -- many uneven images in one persistent launch, replayed from a
// CUDA graph.
//
// The paper's point about its vision models is that input shapes vary widely
// and a different kernel configuration wins for each (Sec. 6.2).  A batch plan
// therefore specialises one kernel variant per (filter size, depth, filter
// class) present in the batch -- all compiled together by NVRTC into ONE
// kernel that switches on the image's variant -- and schedules every output
// tile of every image through a single launch:
//   * the work list (image, tile_x, tile_y, tile_f) is built at plan time and
//     ordered by tile cost, largest first (longest-processing-time first);
//   * persistent CTAs (as many as are co-resident) take items from an atomic
//     counter, so small and large images balance across SMs;
//   * the launch is a two-node CUDA graph: zero the counter, run the kernel.
//     Image pointers are kernel parameters; when a call passes different
//     pointers the instantiated graph's kernel node is updated in place
//     (launches already enqueued keep their old parameters).
#include <algorithm>
#include <array>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <sstream>
#include <tuple>

#include "internal.h"

using namespace fbc;

namespace {

constexpr int kBatchThreads = 256;
// Three CTAs per SM: while one stages a work item's halo and bank slice, the
// other two compute.  Measured on the 64-image batch (GB300): 3 CTAs of <= 72 KB
// and <= 32 accumulators per thread 7.85 ms, 4 CTAs of <= 54 KB 7.90 ms, 2 CTAs
// of <= 110 KB 8.77 ms (<= 64 accumulators: 8.37 ms), 1 CTA of <= 220 KB 9.54 ms.
constexpr int kBatchMinBlocks = 3;
constexpr int kBatchMaxImages = 256;
constexpr size_t kBatchSmemLimit = 72 * 1024;    // keeps three CTAs resident per SM
constexpr int kMetaInts = 6;
constexpr int kArgsHeader = 40;                   // bytes before the pointer table
constexpr int kPtrEntry = 24;
constexpr int kBatchMaxBlock = 32;                // accumulators per thread (85 registers at 3 CTAs/SM)

struct BatchVariant {
    int fh, fw, d, nclass;
    DirectTile tile;
};

int filter_class(int64_t N) { return N <= 16 ? 16 : (N <= 32 ? 32 : 64); }

}  // namespace

struct fbcorr_batch_plan {
    int n = 0;
    std::vector<std::array<int64_t, 6>> shp;   // H, W, D, N, fh, fw
    std::vector<int> var_of;                    // variant index per image
    std::vector<BatchVariant> variants;
    fbcorr_dtype_t dtype = FBCORR_F32;
    fbcorr_epilogue_t epi{0, 0.f, 0.f};
    DeviceInfo dev;
    Kernel kern;
    int4* work = nullptr;
    int* meta = nullptr;
    int* counter = nullptr;
    int nwork = 0;
    int grid = 0;
    int blocks_per_sm = 0;
    std::vector<unsigned char> args;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t knode = nullptr;
    long long flops = 0;
};

namespace {

std::string batch_source(const fbcorr_batch_plan* b) {
    std::ostringstream o;
    o << rtcg_header_source() << "\n";
    o << "typedef FbcBatchArgs<" << b->n << "> FbcBA;\n";
    // header (3 pointers + 4 words) then the pointer table, no padding anywhere
    o << "static_assert(sizeof(FbcBA) == " << kArgsHeader << " + " << kPtrEntry << " * " << b->n
      << ", \"batch argument layout\");\n";
    o << "static_assert(sizeof(FbcBatchPtrs) == " << kPtrEntry << ", \"batch pointer layout\");\n";
    const int epi = b->epi.kind == FBCORR_EPI_CLAMP ? 1 : 0;
    for (size_t v = 0; v < b->variants.size(); ++v) {
        const BatchVariant& bv = b->variants[v];
        const DirectTile& t = bv.tile;
        if (t.ks > 1)   // the K-split tile (short reductions: lanes split the depth)
            o << "typedef FbcDirectKS<" << bv.fh << "," << bv.fw << "," << bv.d << "," << t.tr << "," << t.tf << ","
              << t.ks << "," << t.wq << "," << t.wr << "," << t.wf << "," << epi << "," << t.pk << "," << t.sh
              << "> FbcV" << v << ";\n";
        else
            o << "typedef FbcDirect<" << bv.fh << "," << bv.fw << "," << bv.d << "," << t.tr << "," << t.tf
              << "," << t.wr << "," << t.wf << ",0," << epi << ",0," << t.chunk(bv.d) << "," << t.pk << "> FbcV"
              << v << ";\n";
        // one non-inlined function per variant: each gets its own register
        // allocation instead of the maximum over every variant of the switch
        o << "__device__ __noinline__ void fbc_run_v" << v
          << "(const FbcDirectArgs& da, float* sm, int x, int y, int z) { FbcV" << v
          << "::run(da, sm, x, y, z); }\n";
    }
    o << "extern \"C\" __global__ void __launch_bounds__(" << kBatchThreads
      << ", " << kBatchMinBlocks << ") fbc_batch(const __grid_constant__ FbcBA a) {\n"
      << "  extern __shared__ __align__(16) float fbc_smem[];\n"
      << "  __shared__ int s_item;\n"
      << "  int4 wk;\n"
      << "  while (fbc_batch_next(a.counter, a.nwork, &s_item, &wk, a.work)) {\n"
      << "    const int* md = a.meta + " << kMetaInts << " * wk.x;\n"
      << "    FbcDirectArgs da;\n"
      << "    da.x = a.img[wk.x].x; da.m = nullptr; da.w = a.img[wk.x].w; da.y = a.img[wk.x].y;\n"
      << "    da.in_h = md[0]; da.in_w = md[1]; da.out_h = md[2]; da.out_w = md[3]; da.nf = md[4];\n"
      << "    da.pad_y = 0; da.pad_x = 0; da.lo = a.lo; da.hi = a.hi;\n"
      << "    switch (md[5]) {\n";
    for (size_t v = 0; v < b->variants.size(); ++v)
        o << "      case " << v << ": fbc_run_v" << v << "(da, fbc_smem, wk.y, wk.z, wk.w); break;\n";
    o << "      default: break;\n"
      << "    }\n"
      << "    __syncthreads();\n"
      << "  }\n"
      << "}\n";
    return o.str();
}

void write_ptr_entry(std::vector<unsigned char>& args, int k, const void* x, const void* w, void* y) {
    unsigned char* e = args.data() + kArgsHeader + (size_t)k * kPtrEntry;
    memcpy(e, &x, 8);
    memcpy(e + 8, &w, 8);
    memcpy(e + 16, &y, 8);
}

void destroy(fbcorr_batch_plan* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->work) cudaFree(b->work);
    if (b->meta) cudaFree(b->meta);
    if (b->counter) cudaFree(b->counter);
    delete b;
}

// One tile per (fh, fw, D, filter class), 256 threads per CTA.  The tile comes
// from, in order: a measurement when FBCORR_AUTOTUNE is 1 or force (the
// variant's largest image, timed as a single-image launch under the batch
// kernel's constraints, result stored in the tuning cache), the tuning cache,
// or the analytic ranking.
fbcorr_status_t select_variants(fbcorr_batch_plan* b, bool allow_tuning) {
    std::map<std::tuple<int, int, int, int>, int> key_to_var;
    std::vector<int> rep_image;   // per variant: its largest image
    b->var_of.resize(b->n);
    b->variants.clear();
    for (int k = 0; k < b->n; ++k) {
        const auto& s = b->shp[k];
        const auto key = std::make_tuple((int)s[4], (int)s[5], (int)s[2], filter_class(s[3]));
        auto it = key_to_var.find(key);
        if (it == key_to_var.end()) {
            key_to_var[key] = (int)b->variants.size();
            b->variants.push_back(BatchVariant{(int)s[4], (int)s[5], (int)s[2], filter_class(s[3]), DirectTile{}});
            rep_image.push_back(k);
            it = key_to_var.find(key);
        }
        const int v = it->second;
        b->var_of[k] = v;
        auto work = [&](int img) {
            const auto& t = b->shp[img];
            return (t[0] - t[4] + 1) * (t[1] - t[5] + 1) * t[3];
        };
        if (work(k) > work(rep_image[v])) rep_image[v] = k;
    }
    const std::string at = env_str("FBCORR_AUTOTUNE", "0");
    const bool tune = allow_tuning && (at == "1" || at == "force");
    const int topk = std::max(1, atoi(env_str("FBCORR_TUNE_TOPK_BATCH", "4").c_str()));
    const int epi = b->epi.kind == FBCORR_EPI_CLAMP ? 1 : 0;
    if (tune) {
        // compile the candidates of every variant at once, in parallel
        std::vector<std::string> srcs;
        for (size_t v = 0; v < b->variants.size(); ++v) {
            const BatchVariant& bv = b->variants[v];
            const auto& s = b->shp[rep_image[v]];
            DirectProblem rep{(int)s[0], (int)s[1], bv.d, (int)(s[0] - s[4] + 1), (int)(s[1] - s[5] + 1),
                              (int)s[3], bv.fh, bv.fw, 0, 0, 0, epi, 0};
            auto ranked = direct_ranked(rep, kBatchSmemLimit, b->dev.sm_count, kBatchThreads, kBatchMaxBlock);
            for (const auto& sp : direct_tuning_specs(ranked, topk)) {
                DirectTile t;
                if (parse_direct_spec(sp, &t))
                    srcs.push_back(direct_kernel_source(rep, t, kname_for("fbc_direct", rep, t)));
            }
        }
        rtcg_precompile(srcs);
    }
    for (size_t v = 0; v < b->variants.size(); ++v) {
        BatchVariant& bv = b->variants[v];
        const auto& s = b->shp[rep_image[v]];
        DirectProblem rep{(int)s[0], (int)s[1], bv.d, (int)(s[0] - s[4] + 1), (int)(s[1] - s[5] + 1),
                          (int)s[3], bv.fh, bv.fw, 0, 0, 0, epi, 0};
        char key_s[96];
        snprintf(key_s, sizeof key_s, "batchvar|f%dx%d|c%d|n%d|t%d", bv.fh, bv.fw, bv.d, bv.nclass,
                 kBatchThreads);
        const std::string key = tune_key(b->dev, key_s);
        std::string spec;
        DirectTile t;
        bool have = false;
        if (env_str("FBCORR_BATCH_KS", "0") == "1") {
            // tests and profiling: the model's first K-split tile wherever one fits
            // (the tuner itself is offered them only with FBCORR_TUNE_KS_BATCH=1)
            for (const auto& c : direct_ranked(rep, kBatchSmemLimit, b->dev.sm_count, kBatchThreads, kBatchMaxBlock))
                if (c.ks > 1 && !c.ks_chunked()) {
                    t = c;
                    t.pk = 1;
                    have = true;
                    break;
                }
        }
        if (!have && tune && (at == "force" || !tune_lookup(key, &spec))) {
            float ms = 0.f;
            if (tune_direct_problem(b->dev, rep, nullptr, kBatchThreads, kBatchMaxBlock, kBatchSmemLimit,
                                    topk, false, "batch", &spec, &ms) == FBCORR_OK &&
                parse_direct_spec(spec, &t)) {
                tune_store(key, spec);
                have = true;
            }
        }
        if (!have && tune_lookup(key, &spec) && parse_direct_spec(spec, &t) &&
            t.threads() == kBatchThreads && !t.ks_chunked() && t.tr * t.tf <= kBatchMaxBlock &&
            direct_smem_bytes(t, bv.fh, bv.fw, bv.d) <= kBatchSmemLimit)
            have = true;
        if (!have) t = direct_heuristic(rep, kBatchSmemLimit, b->dev.sm_count, kBatchThreads, kBatchMaxBlock);
        if (t.threads() != kBatchThreads || t.ks_chunked() || direct_smem_bytes(t, bv.fh, bv.fw, bv.d) > kBatchSmemLimit)
            return set_error(FBCORR_ERR_UNSUPPORTED, "no batched tile fits filter %dx%d at depth %d", bv.fh,
                             bv.fw, bv.d);
        bv.tile = t;
    }
    clear_error();
    return FBCORR_OK;
}

size_t batch_smem(const fbcorr_batch_plan* b) {
    size_t smem = 0;
    for (const auto& bv : b->variants)
        smem = std::max(smem, direct_smem_bytes(bv.tile, bv.fh, bv.fw, bv.d));
    return smem;
}

fbcorr_status_t build(fbcorr_batch_plan* b) {
    FBC_TRY(select_variants(b, true));
    const size_t smem = batch_smem(b);

    // ---- one generated kernel for the whole batch
    char name[64];
    snprintf(name, sizeof name, "fbc_batch");
    FBC_TRY(rtcg_kernel(batch_source(b), name, smem, kBatchThreads, &b->kern));

    // ---- work list, largest tiles first
    struct Item {
        long long cost;
        int4 w;
    };
    std::vector<Item> items;
    std::vector<int> meta(kMetaInts * b->n);
    b->flops = 0;
    for (int k = 0; k < b->n; ++k) {
        const auto& s = b->shp[k];
        const int Ho = (int)(s[0] - s[4] + 1), Wo = (int)(s[1] - s[5] + 1), N = (int)s[3];
        const BatchVariant& bv = b->variants[b->var_of[k]];
        const DirectTile& t = bv.tile;
        const int gx = (Wo + t.bw() - 1) / t.bw(), gy = (Ho + t.bh() - 1) / t.bh(), gz = (N + t.bn() - 1) / t.bn();
        const long long cost = (long long)t.bh() * t.bw() * t.bn() * bv.fh * bv.fw * bv.d;
        for (int z = 0; z < gz; ++z)
            for (int y = 0; y < gy; ++y)
                for (int x = 0; x < gx; ++x) items.push_back(Item{cost, make_int4(k, x, y, z)});
        meta[kMetaInts * k + 0] = (int)s[0];
        meta[kMetaInts * k + 1] = (int)s[1];
        meta[kMetaInts * k + 2] = Ho;
        meta[kMetaInts * k + 3] = Wo;
        meta[kMetaInts * k + 4] = N;
        meta[kMetaInts * k + 5] = b->var_of[k];
        b->flops += 2LL * Ho * Wo * N * s[4] * s[5] * s[2];
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const Item& a, const Item& c) { return a.cost > c.cost; });
    b->nwork = (int)items.size();
    std::vector<int4> work(items.size());
    for (size_t i = 0; i < items.size(); ++i) work[i] = items[i].w;

    FBC_CUDA(cudaMalloc(&b->work, sizeof(int4) * work.size()));
    FBC_CUDA(cudaMalloc(&b->meta, sizeof(int) * meta.size()));
    FBC_CUDA(cudaMalloc(&b->counter, sizeof(int)));
    FBC_CUDA(cudaMemcpy(b->work, work.data(), sizeof(int4) * work.size(), cudaMemcpyHostToDevice));
    FBC_CUDA(cudaMemcpy(b->meta, meta.data(), sizeof(int) * meta.size(), cudaMemcpyHostToDevice));
    FBC_CUDA(cudaMemset(b->counter, 0, sizeof(int)));

    // ---- persistent grid: every co-resident CTA, at most one per work item
    FBC_TRY(kernel_occupancy(b->kern, &b->blocks_per_sm));
    if (b->blocks_per_sm < 1)
        return set_error(FBCORR_ERR_UNSUPPORTED, "batched kernel cannot be resident (smem %zu)", smem);
    b->grid = std::min(b->nwork, b->blocks_per_sm * std::max(1, b->dev.sm_count));

    // ---- kernel argument image (layout checked by the generated static_asserts)
    b->args.assign(kArgsHeader + (size_t)kPtrEntry * b->n, 0);
    unsigned char* a = b->args.data();
    const void* wp = b->work;
    const void* mp = b->meta;
    const void* cp = b->counter;
    const float lo = b->epi.lo, hi = b->epi.hi;
    memcpy(a + 0, &wp, 8);
    memcpy(a + 8, &mp, 8);
    memcpy(a + 16, &cp, 8);
    memcpy(a + 24, &b->nwork, 4);
    memcpy(a + 28, &lo, 4);
    memcpy(a + 32, &hi, 4);

    // ---- the graph: zero the counter, then the persistent kernel
    FBC_CUDA(cudaGraphCreate(&b->graph, 0));
    cudaMemsetParams ms;
    memset(&ms, 0, sizeof ms);
    ms.dst = b->counter;
    ms.value = 0;
    ms.elementSize = sizeof(int);
    ms.width = 1;
    ms.height = 1;
    cudaGraphNode_t mnode;
    FBC_CUDA(cudaGraphAddMemsetNode(&mnode, b->graph, nullptr, 0, &ms));
    void* kargs[] = {b->args.data()};
    FBC_TRY(graph_add_kernel(b->graph, &mnode, 1, b->kern, dim3(b->grid), kargs, &b->knode));
    FBC_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return FBCORR_OK;
}

}  // namespace

extern "C" {

fbcorr_status_t fbcorr_batch_plan_create(fbcorr_batch_plan_t* out, int n, const int64_t (*in_shapes)[3],
                                         const int64_t (*filt_shapes)[4], fbcorr_dtype_t dtype,
                                         fbcorr_epilogue_t epilogue) {
    clear_error();
    if (!out) return set_error(FBCORR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > kBatchMaxImages)
        return set_error(FBCORR_ERR_INVALID_ARG, "a batch holds 1..%d images (got %d)", kBatchMaxImages, n);
    if (!in_shapes || !filt_shapes) return set_error(FBCORR_ERR_INVALID_ARG, "NULL shape arrays");
    for (int k = 0; k < n; ++k) {
        if (epilogue.kind == FBCORR_EPI_SNIPPET)
            return set_error(FBCORR_ERR_UNSUPPORTED, "batch plans have no snippet epilogue");
        fbcorr_status_t s = validate_shapes(in_shapes[k], filt_shapes[k], dtype, epilogue);
        if (s != FBCORR_OK) return set_error(s, "image %d: %s", k, fbcorr_last_error());
    }
    if (dtype != FBCORR_F32)
        return set_error(FBCORR_ERR_UNSUPPORTED, "batched plans compute in FBCORR_F32");
    DeviceInfo dev;
    FBC_TRY(device_info(&dev));
    if (dev.cc_major != 10 || dev.cc_minor != 3)
        return set_error(FBCORR_ERR_UNSUPPORTED, "libfbcorr is built for sm_103a (GB300)");
    fbcorr_batch_plan* b = new (std::nothrow) fbcorr_batch_plan();
    if (!b) return set_error(FBCORR_ERR_OOM, "host allocation failed");
    b->n = n;
    b->dtype = dtype;
    b->epi = epilogue;
    if (b->epi.kind == FBCORR_EPI_NONE) b->epi.lo = b->epi.hi = 0.f;
    b->dev = dev;
    for (int k = 0; k < n; ++k)
        b->shp.push_back({in_shapes[k][0], in_shapes[k][1], in_shapes[k][2], filt_shapes[k][0],
                          filt_shapes[k][1], filt_shapes[k][2]});
    fbcorr_status_t s = build(b);
    if (s != FBCORR_OK) {
        destroy(b);
        return s;
    }
    *out = b;
    return FBCORR_OK;
}

fbcorr_status_t fbcorr_batch_rtcg_check(int n, const int64_t (*in_shapes)[3],
                                        const int64_t (*filt_shapes)[4], fbcorr_epilogue_t epilogue,
                                        char* log, size_t cap) {
    clear_error();
    if (log && cap) log[0] = '\0';
    if (n < 1 || n > kBatchMaxImages || !in_shapes || !filt_shapes)
        return set_error(FBCORR_ERR_INVALID_ARG, "bad batch description");
    if (epilogue.kind == FBCORR_EPI_SNIPPET)
        return set_error(FBCORR_ERR_UNSUPPORTED, "batch plans have no snippet epilogue");
    for (int k = 0; k < n; ++k) FBC_TRY(validate_shapes(in_shapes[k], filt_shapes[k], FBCORR_F32, epilogue));
    fbcorr_batch_plan tmp;
    tmp.n = n;
    tmp.epi = epilogue;
    tmp.dev.sm_count = 148;
    snprintf(tmp.dev.name, sizeof tmp.dev.name, "offline-check");
    for (int k = 0; k < n; ++k)
        tmp.shp.push_back({in_shapes[k][0], in_shapes[k][1], in_shapes[k][2], filt_shapes[k][0],
                           filt_shapes[k][1], filt_shapes[k][2]});
    FBC_TRY(select_variants(&tmp, false));
    std::string lg;
    fbcorr_status_t s = rtcg_compile_only(batch_source(&tmp), &lg);
    if (s != FBCORR_OK && log && cap) snprintf(log, cap, "%s", lg.c_str());
    return s;
}

fbcorr_status_t fbcorr_batch_plan_destroy(fbcorr_batch_plan_t b) {
    clear_error();
    destroy(b);
    return FBCORR_OK;
}

fbcorr_status_t fbcorr_batch_plan_workspace_size(fbcorr_batch_plan_t b, size_t* bytes) {
    clear_error();
    if (!b || !bytes) return set_error(FBCORR_ERR_INVALID_ARG, "NULL argument");
    *bytes = 0;
    return FBCORR_OK;
}

fbcorr_status_t fbcorr_batch_plan_info(fbcorr_batch_plan_t b, char* buf, size_t cap) {
    clear_error();
    if (!b || !buf || cap == 0) return set_error(FBCORR_ERR_INVALID_ARG, "NULL argument");
    std::ostringstream o;
    o << "{\"images\":" << b->n << ",\"work_items\":" << b->nwork << ",\"grid\":" << b->grid
      << ",\"blocks_per_sm\":" << b->blocks_per_sm << ",\"threads\":" << kBatchThreads
      << ",\"smem\":" << b->kern.smem << ",\"flops\":" << b->flops << ",\"launches\":1"
      << ",\"variants\":[";
    for (size_t v = 0; v < b->variants.size(); ++v) {
        const auto& bv = b->variants[v];
        o << (v ? "," : "") << "{\"f\":[" << bv.fh << "," << bv.fw << "],\"d\":" << bv.d
          << ",\"filters\":" << bv.nclass << ",\"spec\":\"" << direct_tile_spec(bv.tile) << "\"}";
    }
    o << "]}";
    snprintf(buf, cap, "%s", o.str().c_str());
    return FBCORR_OK;
}

fbcorr_status_t fbcorr_forward_batched(fbcorr_batch_plan_t b, const float* const* x,
                                       const float* const* w, float* const* y, void* ws,
                                       size_t ws_bytes, fbcorr_stream_t stream) {
    clear_error();
    (void)ws;
    (void)ws_bytes;
    if (!b || !x || !w || !y) return set_error(FBCORR_ERR_INVALID_ARG, "NULL argument");
    bool changed = false;
    for (int k = 0; k < b->n; ++k) {
        if (!x[k] || !w[k] || !y[k]) return set_error(FBCORR_ERR_INVALID_ARG, "NULL pointer for image %d", k);
        if ((((uintptr_t)x[k]) | ((uintptr_t)w[k]) | ((uintptr_t)y[k])) & 15u)
            return set_error(FBCORR_ERR_ALIGNMENT, "image %d: tensors must be 16-byte aligned", k);
        const unsigned char* e = b->args.data() + kArgsHeader + (size_t)k * kPtrEntry;
        const void* old[3];
        memcpy(old, e, 24);
        if (old[0] != x[k] || old[1] != w[k] || old[2] != y[k]) {
            write_ptr_entry(b->args, k, x[k], w[k], y[k]);
            changed = true;
        }
    }
    if (changed) {
        void* kargs[] = {b->args.data()};
        FBC_TRY(graph_set_kernel(b->exec, b->knode, b->kern, dim3(b->grid), kargs));
    }
    FBC_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return FBCORR_OK;
}

}  // extern "C"
