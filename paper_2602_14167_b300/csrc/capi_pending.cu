// Entry points whose kernels are not in this build yet: they fail loudly.
#include "capi_internal.hpp"

using namespace tcng;

extern "C" {

tcng_status tcng_apply_shared_unitary(tcng_state*, const int*, int, const double*, void*) {
    return fail(TCNG_EUNSUPPORTED, "tcng_apply_shared_unitary is not built yet");
}
tcng_status tcng_mlp_forward(const float*, int, int, int, int, const float*, const float*,
                             const float*, const float*, const float*, const float*, float*, float*,
                             void*) {
    return fail(TCNG_EUNSUPPORTED, "tcng_mlp_forward is not built yet");
}
tcng_status tcng_mlp_backward(const float*, int, int, int, int, const float*, const float*,
                              const float*, const float*, const float*, const float*, const float*,
                              float*, double*, void*) {
    return fail(TCNG_EUNSUPPORTED, "tcng_mlp_backward is not built yet");
}
tcng_status tcng_autotune(int, tcng_dtype, int, const char*) {
    return fail(TCNG_EUNSUPPORTED, "tcng_autotune is not built yet");
}

}  // extern "C"
