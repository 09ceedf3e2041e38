// probe.cu -- FP64 and FP32 FMA throughput probe (roofline denominator for ALU-bound kernels).
// Each thread runs independent FMA chains; the result is folded into one store so the
// compiler cannot drop the work.
#include "internal.cuh"

namespace pmeft {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* __restrict__ out, int iters, T a, T b)
{
    T x0 = (T)threadIdx.x * T(1e-3), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
    T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == T(-12345.678)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace pmeft

using namespace pmeft;

// Measured FMA throughput in GFLOP/s (2 flops per FMA) of this device, FP64 and FP32.
extern "C" pm_status pm_probe_fma(pm_ctx* ctx, double* fp64_gflops, double* fp32_gflops)
{
    if (!ctx || !fp64_gflops || !fp32_gflops) return PM_ERR_INVALID_ARG;
    const int blocks = ctx->num_sms * 8, threads = 256;
    double* dout = nullptr;
    PM_CUDA(cudaMalloc(&dout, (size_t)blocks * threads * sizeof(double)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int pass = 0; pass < 2; ++pass) {
        const int iters = pass == 0 ? 4096 : 32768;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, ctx->stream);
            if (pass == 0) k_fma_probe<double><<<blocks, threads, 0, ctx->stream>>>(dout, iters, 0.999999, 1e-7);
            else k_fma_probe<float><<<blocks, threads, 0, ctx->stream>>>((float*)dout, iters, 0.999999f, 1e-7f);
            cudaEventRecord(e1, ctx->stream);
            cudaEventSynchronize(e1);
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
        (pass == 0 ? *fp64_gflops : *fp32_gflops) = flops / (ms * 1e-3) / 1e9;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dout);
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}
