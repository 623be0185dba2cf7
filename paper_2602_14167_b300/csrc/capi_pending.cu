// Entry points whose kernels are not in this build yet: they fail loudly.
#include "capi_internal.hpp"

using namespace tcng;

extern "C" {

tcng_status tcng_autotune(int, tcng_dtype, int, const char*) {
    return fail(TCNG_EUNSUPPORTED, "tcng_autotune is not built yet");
}

}  // extern "C"
