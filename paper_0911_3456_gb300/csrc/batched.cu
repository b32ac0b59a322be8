// batched.cu -- placeholder until the persistent batched kernel lands.
#include "internal.h"

using namespace fbc;

extern "C" {
fbcorr_status_t fbcorr_batch_plan_create(fbcorr_batch_plan_t* out, int, const int64_t (*)[3],
                                         const int64_t (*)[4], fbcorr_dtype_t, fbcorr_epilogue_t) {
    if (out) *out = nullptr;
    return set_error(FBCORR_ERR_UNSUPPORTED, "batched plans are not built yet");
}
fbcorr_status_t fbcorr_batch_plan_destroy(fbcorr_batch_plan_t) { return FBCORR_OK; }
fbcorr_status_t fbcorr_batch_plan_workspace_size(fbcorr_batch_plan_t, size_t* b) {
    if (b) *b = 0;
    return FBCORR_OK;
}
fbcorr_status_t fbcorr_batch_plan_info(fbcorr_batch_plan_t, char* buf, size_t cap) {
    if (buf && cap) buf[0] = 0;
    return FBCORR_OK;
}
fbcorr_status_t fbcorr_forward_batched(fbcorr_batch_plan_t, const float* const*, const float* const*,
                                       float* const*, void*, size_t, fbcorr_stream_t) {
    return set_error(FBCORR_ERR_UNSUPPORTED, "batched plans are not built yet");
}
}
