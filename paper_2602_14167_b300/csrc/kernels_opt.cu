// Device Adam update (the optimiser of the paper's training listings,
// optax.adam).  Kingma & Ba: m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
// theta <- theta - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
// The step counter lives on the device so the update can be replayed from a
// CUDA graph: the update kernel reads t = *step + 1, a one-thread kernel then
// stores it.
#include <cuda_runtime.h>

#include <algorithm>

#include "capi_internal.hpp"

namespace tcng {

template <typename T>
__global__ void adam_kernel(T* __restrict__ theta, T* __restrict__ m, T* __restrict__ v,
                            const T* __restrict__ g, size_t n, T lr, T b1, T b2, T eps,
                            const int* __restrict__ step) {
    const int t = *step + 1;
    const T c1 = T(1) / (T(1) - pow(b1, (T)t));
    const T c2 = T(1) / (T(1) - pow(b2, (T)t));
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const T gi = g[i];
        const T mi = b1 * m[i] + (T(1) - b1) * gi;
        const T vi = b2 * v[i] + (T(1) - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi * c1) / (sqrt(vi * c2) + eps);
    }
}

__global__ void step_increment_kernel(int* step) { *step += 1; }

template <typename T>
static tcng_status adam_impl(T* theta, T* m, T* v, const T* g, size_t n, T lr, T b1, T b2, T eps,
                             int* step, void* stream) {
    if (!theta || !m || !v || !g || !step) return fail(TCNG_EINVAL, "null argument");
    if (!(b1 >= 0 && b1 < 1 && b2 >= 0 && b2 < 1 && eps > 0))
        return fail(TCNG_EINVAL, "need 0 <= b1, b2 < 1 and eps > 0");
    if (n == 0) return TCNG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int threads = 256;
    const size_t blocks = std::min<size_t>((n + threads - 1) / threads, (size_t)num_sms() * 8);
    {
        ProfScope ps("adam", s);
        adam_kernel<T><<<(unsigned)blocks, threads, 0, s>>>(theta, m, v, g, n, lr, b1, b2, eps, step);
        count_launch();
        step_increment_kernel<<<1, 1, 0, s>>>(step);
        count_launch();
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "adam kernel");
    return TCNG_OK;
}

}  // namespace tcng

using namespace tcng;

extern "C" {

tcng_status tcng_adam_step(double* theta, double* m, double* v, const double* grad, size_t n,
                           double lr, double b1, double b2, double eps, int* step_dev, void* stream) {
    return adam_impl<double>(theta, m, v, grad, n, lr, b1, b2, eps, step_dev, stream);
}

tcng_status tcng_adam_step_f32(float* theta, float* m, float* v, const float* grad, size_t n,
                               float lr, float b1, float b2, float eps, int* step_dev, void* stream) {
    return adam_impl<float>(theta, m, v, grad, n, lr, b1, b2, eps, step_dev, stream);
}

}  // extern "C"
