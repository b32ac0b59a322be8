// tc_kernel.cu -- placeholder until the tcgen05 path lands.
#include "internal.h"

namespace fbc {
struct TcPlan { int dummy; };
fbcorr_status_t tc_plan_create(TcPlan** out, int, int, int, int, int, int, int, int, float, float,
                               const DeviceInfo&) {
    *out = nullptr;
    return set_error(FBCORR_ERR_UNSUPPORTED, "tensor-core modes are not built yet");
}
void tc_plan_destroy(TcPlan*) {}
size_t tc_workspace_bytes(const TcPlan*) { return 0; }
fbcorr_status_t tc_forward(TcPlan*, const float*, const float*, float*, void*, int*, cudaStream_t) {
    return set_error(FBCORR_ERR_UNSUPPORTED, "tensor-core modes are not built yet");
}
std::string tc_describe(const TcPlan*) { return "none"; }
}  // namespace fbc
