// pizza_fp64_fma_rate: the FP64 fused multiply-add rate of the current device,
// measured.  The explicit and implicit stages of the step are bound by FP64
// issue on this GPU (its FP64 rate is a small fraction of its FP32 rate), so
// their roofline denominator is this rate; the kernel below is the measurement.
#include <cuda_runtime.h>

#include "../../include/pizza.h"
#include "pizza_internal.h"

namespace pz {
namespace {

constexpr int FMA_CHAINS = 8;     // independent dependency chains per thread
constexpr int FMA_THREADS = 256;

// Each thread runs FMA_CHAINS independent chains x <- x * b + c for `iters`
// rounds (2 flops each).  b < 1 keeps every chain bounded and normal; the final
// values are summed and stored so that nothing is eliminated.
__global__ void __launch_bounds__(FMA_THREADS) k_fma_rate(int iters, double b, double c, double* __restrict__ out) {
    double x[FMA_CHAINS];
#pragma unroll
    for (int i = 0; i < FMA_CHAINS; ++i) x[i] = 1.0 + 1e-3 * (threadIdx.x + i);
    for (int r = 0; r < iters; ++r) {
#pragma unroll
        for (int i = 0; i < FMA_CHAINS; ++i) x[i] = fma(x[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < FMA_CHAINS; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace pz

using namespace pz;

extern "C" int pizza_fp64_fma_rate(int iters, double* tflops, double* ms) {
    if (!tflops || iters < 1) {
        set_global_error("pizza_fp64_fma_rate: iters >= 1 and an output pointer are required");
        return PIZZA_EINVAL;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_global_error("pizza_fp64_fma_rate: no CUDA device");
        return PIZZA_ECUDA;
    }
    const int blocks = sms * 8;  // 8 x 256 threads: every warp slot of an SM busy
    double* out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(double) * (size_t)blocks * FMA_THREADS);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) {
        k_fma_rate<<<blocks, FMA_THREADS>>>(iters / 8 + 1, 0.9999999, 1e-7, out);  // warm-up
        cudaEventRecord(a);
        k_fma_rate<<<blocks, FMA_THREADS>>>(iters, 0.9999999, 1e-7, out);
        cudaEventRecord(b);
        e = cudaEventSynchronize(b);
    }
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (out) cudaFree(out);
    if (e != cudaSuccess) {
        set_global_error(cudaGetErrorString(e));
        return PIZZA_ECUDA;
    }
    const double flops = 2.0 * FMA_CHAINS * (double)iters * blocks * FMA_THREADS;
    *tflops = flops / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return PIZZA_OK;
}
