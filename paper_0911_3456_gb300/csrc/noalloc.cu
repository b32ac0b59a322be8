// noalloc.cu -- a forward entry point that allocates nothing.
//
// fbcorr_forward needs a caller-provided device workspace for the tensor-core
// plans (the BF16 hi/lo copies of x and w that the split pre-pass writes and
// the tcgen05 kernel reads).  Some callers cannot obtain one at call time:
// code that may not call cudaMalloc after start-up (real-time loops, plugin
// hosts whose device allocator belongs to another runtime, processes that
// budget every device byte at initialisation), or code running where an
// allocation would synchronise the device.  fbcorr_forward_noalloc serves them:
// it runs exactly the same pre-pass and kernels, with the scratch placed in a
// fixed-size array compiled into this library instead of a workspace.
//
// The array's name is a host-side stand-in, not a device address, so host code
// never passes it to a kernel.  Its device address is looked up once per device
// with cudaGetSymbolAddress (with that device current) on the first call made
// on that device, and cached; the plan's device must be the current one.  The
// cache is not refreshed after cudaDeviceReset, so the entry point must not be
// used once the device has been reset in this process.
#include <mutex>
#include <vector>

#include "internal.h"

using namespace fbc;

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)48 << 20;   // 48 MiB

// Shared by every call on a device; keeps whatever the last call wrote.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
std::vector<void*> g_scratch_ptr;   // device address per device ordinal

// The scratch address on `plan_dev`, which must be the current device: the
// address belongs to the device current when it was looked up, and a kernel of
// the plan given another device's address would touch that device's memory.
fbcorr_status_t scratch_address(int plan_dev, void** out) {
    int dev = -1;
    FBC_CUDA(cudaGetDevice(&dev));
    if (dev != plan_dev)
        return set_error(FBCORR_ERR_INVALID_ARG,
                         "the plan was created on device %d but device %d is current; make the plan's "
                         "device current before calling fbcorr_forward_noalloc",
                         plan_dev, dev);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if ((int)g_scratch_ptr.size() <= dev) g_scratch_ptr.resize(dev + 1, nullptr);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(FBCORR_ERR_CUDA, "cudaGetSymbolAddress(scratch) on device %d: %s", dev,
                             cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return FBCORR_OK;
}

}  // namespace

extern "C" fbcorr_status_t fbcorr_forward_noalloc(fbcorr_plan_t plan, const float* x, const float* w,
                                                  float* y, fbcorr_stream_t stream) {
    clear_error();
    if (!plan || !x || !w || !y) return set_error(FBCORR_ERR_INVALID_ARG, "NULL argument");
    size_t need = 0;
    FBC_TRY(fbcorr_plan_workspace_size(plan, &need, nullptr));
    if (need > kNoAllocScratchBytes)
        return set_error(FBCORR_ERR_WORKSPACE,
                         "this plan needs %zu bytes of scratch; the built-in scratch array holds %zu "
                         "bytes -- use fbcorr_forward with a workspace",
                         need, kNoAllocScratchBytes);
    // Nothing in the scratch needs clearing: the pre-pass writes every byte the
    // kernel reads (zero padding included) before the kernel runs.
    void* ws = nullptr;
    FBC_TRY(scratch_address(plan->dev.device, &ws));
    return fbcorr_forward(plan, x, w, y, ws, kNoAllocScratchBytes, stream);
}
