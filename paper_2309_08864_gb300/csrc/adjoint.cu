// adjoint.cu -- adjoint / loss / inner-product pipelines (stubs; built next).
#include "run.hpp"

using namespace so2dr;

namespace so2dr {
size_t adjoint_workspace_bytes(const Plan& p) { (void)p; return 0; }
}

extern "C" {
int so2dr_adjoint(so2dr_plan_t, const void*, const void*, const void*, void*, void*, void*, size_t, int,
                  double*, so2dr_stats_t*) {
    return set_error(SO2DR_E_UNSUPPORTED, "not built yet");
}
int so2dr_loss(so2dr_plan_t, const void*, const void*, const void*, void*, size_t, double*) {
    return set_error(SO2DR_E_UNSUPPORTED, "not built yet");
}
int so2dr_dot(so2dr_plan_t, const void*, const void*, int64_t, int, double*) {
    return set_error(SO2DR_E_UNSUPPORTED, "not built yet");
}
}
