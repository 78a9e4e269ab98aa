// calibrate.cu -- device measurements the library reports beside its roofline and uses to
// calibrate its planner: the float64 FMA rate of the current GPU.
//
// The constraint solve keeps its violations, multiplier sums and position updates in
// float64 (mixed mode), and on this GPU the float64 pipe is narrow, so its measured rate
// is the second ceiling of the solve next to HBM bandwidth.
#include <cuda_runtime.h>

#include <cstdint>

#include "ilves.h"

namespace ilves {

// Eight independent FMA chains per thread: x <- x * a + b, a fixed point contraction, so
// values stay finite; the result is stored so the chains are not removed.
__global__ void __launch_bounds__(256) k_fp64_fma_probe(double* __restrict__ out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1e-3 * (threadIdx.x + 1) + 0.125 * k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace ilves

using namespace ilves;

extern "C" ilves_status ilves_measure_fp64_fma(int32_t iters, double* gflops, void* stream) {
    if (!gflops || iters < 1) return ILVES_ERR_INVALID_ARG;
    *gflops = 0.0;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ILVES_ERR_CUDA;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ILVES_ERR_CUDA;
    const int threads = 256, blocks = 8 * n_sm;  // 64 warps per SM: every FP64 unit kept busy
    cudaStream_t s = (cudaStream_t)stream;
    double* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ilves_status st = ILVES_OK;
    if (cudaMalloc((void**)&out, sizeof(double) * threads * blocks) != cudaSuccess) return ILVES_ERR_OOM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = ILVES_ERR_CUDA;
    } else {
        k_fp64_fma_probe<<<blocks, threads, 0, s>>>(out, iters / 8 + 1, 0.999, 1e-3);  // warm-up
        cudaEventRecord(e0, s);
        k_fp64_fma_probe<<<blocks, threads, 0, s>>>(out, iters, 0.999, 1e-3);
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) {
            st = ILVES_ERR_CUDA;
        } else {
            const double flops = 2.0 * 8.0 * (double)iters * (double)threads * (double)blocks;
            *gflops = flops / ((double)ms * 1e-3) / 1e9;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return st;
}
