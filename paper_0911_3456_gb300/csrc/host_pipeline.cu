// host_pipeline.cu -- forward from host buffers with the transfers overlapped.
//
// The output rows are split into bands; band b reads input rows
// [r0_b, r1_b + fh - 1) and writes output rows [r0_b, r1_b).  Three streams
// form a pipeline: host->device copies of each band's new input rows, the
// band's correlation (on the caller's stream), and device->host copies of the
// band's output rows, ordered by events, so the host link (the bound on a
// GB300: ~0.2 TB/s each way against 6.7 TB/s of HBM) carries the output of
// band b while band b+1 is computed.  Each band runs through an ordinary plan
// of its own shape (two shapes at most: the regular band and the last one).
#include <algorithm>
#include <map>
#include <new>

#include "internal.h"

namespace fbc {

struct HostPipe {
    int64_t band_rows = 0;                       // output rows per band (a multiple of 4)
    int bands = 0;
    std::map<int64_t, fbcorr_plan_t> plans;      // by band output height
    float *x = nullptr, *w = nullptr, *y = nullptr;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    std::vector<cudaEvent_t> in_ready, out_ready;
};

namespace {

void free_buffers(HostPipe* hp) {
    if (hp->h2d) cudaStreamSynchronize(hp->h2d);
    if (hp->d2h) cudaStreamSynchronize(hp->d2h);
    for (auto& kv : hp->plans) fbcorr_plan_destroy(kv.second);
    hp->plans.clear();
    for (auto e : hp->in_ready) cudaEventDestroy(e);
    for (auto e : hp->out_ready) cudaEventDestroy(e);
    hp->in_ready.clear();
    hp->out_ready.clear();
    cudaFree(hp->ws);
    hp->ws = nullptr;
    hp->ws_bytes = 0;
    hp->bands = 0;
    hp->band_rows = 0;
}

// Band height for `bands` bands of Ho output rows: a multiple of 4 rows, so that
// every band's x and y offsets stay 16-byte aligned.
int64_t band_height(int64_t Ho, int bands) {
    const int64_t h = (Ho + bands - 1) / bands;
    return std::max<int64_t>(4, (h + 3) / 4 * 4);
}

fbcorr_status_t setup(fbcorr_plan_t p, int bands, cudaStream_t s) {
    HostPipe* hp = p->hostpipe;
    const int64_t hb = band_height(p->Ho, bands);
    if (hb == hp->band_rows) return FBCORR_OK;
    free_buffers(hp);   // band_rows stays 0 until everything below succeeded
    hp->bands = (int)((p->Ho + hb - 1) / hb);
    std::vector<int64_t> heights = {std::min(hb, p->Ho)};
    const int64_t last = p->Ho - (hp->bands - 1) * hb;
    if (last != heights[0]) heights.push_back(last);
    for (int64_t ho : heights) {
        const int64_t in[3] = {ho + p->fh - 1, p->W, p->D};
        const int64_t fs[4] = {p->N, p->fh, p->fw, p->D};
        fbcorr_plan_t bp = nullptr;
        FBC_TRY(fbcorr_plan_create(&bp, in, fs, p->dtype, p->epi));
        hp->plans[ho] = bp;
        // a tuned plan gets tuned band plans (first call only; cached by shape)
        if (p->fwd_source == "tuned" && bp->fwd_source != "cache") FBC_TRY(fbcorr_autotune(bp, s));
        size_t need = 0;
        FBC_TRY(fbcorr_plan_workspace_size(bp, &need, nullptr));
        hp->ws_bytes = std::max(hp->ws_bytes, need);
    }
    if (hp->ws_bytes) FBC_CUDA(cudaMalloc(&hp->ws, hp->ws_bytes));
    for (int b = 0; b < hp->bands; ++b) {
        cudaEvent_t a, c;
        FBC_CUDA(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
        hp->in_ready.push_back(a);
        FBC_CUDA(cudaEventCreateWithFlags(&c, cudaEventDisableTiming));
        hp->out_ready.push_back(c);
    }
    hp->band_rows = hb;
    return FBCORR_OK;
}

fbcorr_status_t create(fbcorr_plan_t p) {
    HostPipe* hp = new (std::nothrow) HostPipe();
    if (!hp) return set_error(FBCORR_ERR_OOM, "host allocation failed");
    p->hostpipe = hp;
    const size_t xb = (size_t)(p->H * p->W * p->D) * 4, wb = (size_t)(p->N * p->fh * p->fw * p->D) * 4,
                 yb = (size_t)(p->Ho * p->Wo * p->N) * 4;
    if (cudaMalloc(&hp->x, xb) != cudaSuccess || cudaMalloc(&hp->w, wb) != cudaSuccess ||
        cudaMalloc(&hp->y, yb) != cudaSuccess) {
        cudaGetLastError();
        return set_error(FBCORR_ERR_OOM, "device buffers for the host pipeline (%zu bytes)", xb + wb + yb);
    }
    FBC_CUDA(cudaStreamCreateWithFlags(&hp->h2d, cudaStreamNonBlocking));
    FBC_CUDA(cudaStreamCreateWithFlags(&hp->d2h, cudaStreamNonBlocking));
    FBC_CUDA(cudaEventCreateWithFlags(&hp->start, cudaEventDisableTiming));
    FBC_CUDA(cudaEventCreateWithFlags(&hp->done, cudaEventDisableTiming));
    return FBCORR_OK;
}

}  // namespace

void hostpipe_destroy(HostPipe* hp) {
    if (!hp) return;
    free_buffers(hp);
    cudaFree(hp->x);
    cudaFree(hp->w);
    cudaFree(hp->y);
    if (hp->h2d) cudaStreamDestroy(hp->h2d);
    if (hp->d2h) cudaStreamDestroy(hp->d2h);
    if (hp->start) cudaEventDestroy(hp->start);
    if (hp->done) cudaEventDestroy(hp->done);
    delete hp;
}

fbcorr_status_t hostpipe_device_status(HostPipe* hp, int clear) {
    fbcorr_status_t st = FBCORR_OK;
    if (!hp) return st;
    for (auto& kv : hp->plans) {
        const fbcorr_status_t s = fbcorr_plan_device_status(kv.second, clear);
        if (s != FBCORR_OK) st = s;
    }
    return st;
}

}  // namespace fbc

using namespace fbc;

extern "C" {

fbcorr_status_t fbcorr_forward_host(fbcorr_plan_t p, const float* x_host, const float* w_host, float* y_host,
                                    int bands, fbcorr_stream_t stream) {
    clear_error();
    if (!p || !x_host || !w_host || !y_host) return set_error(FBCORR_ERR_INVALID_ARG, "NULL argument");
    if (bands < 0) return set_error(FBCORR_ERR_INVALID_ARG, "bands must be >= 0 (0: automatic)");
    cudaStream_t s = (cudaStream_t)stream;
    if (!p->hostpipe) {
        const fbcorr_status_t st = create(p);
        if (st != FBCORR_OK) {
            hostpipe_destroy(p->hostpipe);
            p->hostpipe = nullptr;
            return st;
        }
    }
    HostPipe* hp = p->hostpipe;
    // automatic: eight bands (the first band's copy-in and compute, 1/8 of the
    // total each, are all that the output transfer does not hide), at least 4 rows each
    const int nb = bands ? bands : 8;
    FBC_TRY(setup(p, (int)std::max<int64_t>(1, std::min<int64_t>(nb, (p->Ho + 3) / 4)), s));

    const int64_t in_row = p->W * p->D, out_row = p->Wo * p->N;
    FBC_CUDA(cudaEventRecord(hp->start, s));
    FBC_CUDA(cudaStreamWaitEvent(hp->h2d, hp->start, 0));
    FBC_CUDA(cudaStreamWaitEvent(hp->d2h, hp->start, 0));
    FBC_CUDA(cudaMemcpyAsync(hp->w, w_host, (size_t)(p->N * p->fh * p->fw * p->D) * 4, cudaMemcpyHostToDevice,
                             hp->h2d));
    int64_t copied = 0;   // input rows already on the device
    for (int b = 0; b < hp->bands; ++b) {
        const int64_t r0 = b * hp->band_rows, r1 = std::min(p->Ho, r0 + hp->band_rows);
        const int64_t need = (b == hp->bands - 1) ? p->H : r1 + p->fh - 1;
        if (need > copied) {
            FBC_CUDA(cudaMemcpyAsync(hp->x + copied * in_row, x_host + copied * in_row,
                                     (size_t)((need - copied) * in_row) * 4, cudaMemcpyHostToDevice, hp->h2d));
            copied = need;
        }
        FBC_CUDA(cudaEventRecord(hp->in_ready[b], hp->h2d));
        FBC_CUDA(cudaStreamWaitEvent(s, hp->in_ready[b], 0));
        FBC_TRY(fbcorr_forward(hp->plans.at(r1 - r0), hp->x + r0 * in_row, hp->w, hp->y + r0 * out_row, hp->ws,
                               hp->ws_bytes, stream));
        FBC_CUDA(cudaEventRecord(hp->out_ready[b], s));
        FBC_CUDA(cudaStreamWaitEvent(hp->d2h, hp->out_ready[b], 0));
        FBC_CUDA(cudaMemcpyAsync(y_host + r0 * out_row, hp->y + r0 * out_row, (size_t)((r1 - r0) * out_row) * 4,
                                 cudaMemcpyDeviceToHost, hp->d2h));
    }
    FBC_CUDA(cudaEventRecord(hp->done, hp->d2h));
    FBC_CUDA(cudaStreamWaitEvent(s, hp->done, 0));
    return FBCORR_OK;
}

}  // extern "C"
