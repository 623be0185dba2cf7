// Entry points whose kernels are not in this build yet: they fail loudly.
#include "capi_internal.hpp"

using namespace tcng;

extern "C" {

}  // extern "C"
