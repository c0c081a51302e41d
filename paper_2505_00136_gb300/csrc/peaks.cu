// Measurement aid (no counterpart in the paper): the FP64 arithmetic peaks of
// the current GPU, the denominators of the FP64 path's roofline fractions.
//
// Register-only throughput loops: every thread keeps eight independent
// accumulator chains (DMMA: m8n8k4 products, 512 flops per warp instruction;
// DFMA: fused multiply-adds, 2 flops), 152 x 8 CTAs x 256 threads, no memory
// traffic inside the timed loop.  The operands are loaded from a buffer so the
// compiler cannot fold the chains, and the sums are stored so it cannot drop
// them.
#include <stdint.h>

#include "../../include/gprat_gb.h"

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;

__global__ __launch_bounds__(PK_THREADS) void k_peak_dmma(const double* in, double* out, int iters)
{
    const double a = in[threadIdx.x & 7], b = in[8 + (threadIdx.x & 7)];
    double c[PK_CHAINS][2];
#pragma unroll
    for (int q = 0; q < PK_CHAINS; ++q) c[q][0] = c[q][1] = 0.0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < PK_CHAINS; ++q)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                         : "+d"(c[q][0]), "+d"(c[q][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < PK_CHAINS; ++q) s += c[q][0] + c[q][1];
    out[(int64_t)blockIdx.x * PK_THREADS + threadIdx.x] = s;
}

__global__ __launch_bounds__(PK_THREADS) void k_peak_dfma(const double* in, double* out, int iters)
{
    const double a = in[threadIdx.x & 7], b = in[8 + (threadIdx.x & 7)];
    double c[PK_CHAINS];
#pragma unroll
    for (int q = 0; q < PK_CHAINS; ++q) c[q] = (double)q;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < PK_CHAINS; ++q) c[q] = fma(a, c[q], b);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < PK_CHAINS; ++q) s += c[q];
    out[(int64_t)blockIdx.x * PK_THREADS + threadIdx.x] = s;
}

}  // namespace

extern "C" gp_status gp_measure_fp64_peaks(double* dmma_tflops, double* dfma_tflops, void* cuda_stream)
{
    if (!dmma_tflops || !dfma_tflops) return GP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GP_ERR_CUDA;
    const int blocks = sms * 8, iters = 4096;
    double *in = nullptr, *out = nullptr;
    if (cudaMalloc(&in, 16 * sizeof(double)) != cudaSuccess) return GP_ERR_OOM;
    if (cudaMalloc(&out, (size_t)blocks * PK_THREADS * sizeof(double)) != cudaSuccess) {
        cudaFree(in);
        return GP_ERR_OOM;
    }
    const double h_in[16] = {1.0, 1e-3, 2e-3, 3e-3, 4e-3, 5e-3, 6e-3, 7e-3,
                             1e-6, 2e-6, 3e-6, 4e-6, 5e-6, 6e-6, 7e-6, 8e-6};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    gp_status s = GP_OK;
    float ms_dmma = 0.f, ms_dfma = 0.f;
    if (cudaMemcpyAsync(in, h_in, sizeof(h_in), cudaMemcpyHostToDevice, st) != cudaSuccess) s = GP_ERR_CUDA;
    for (int rep = 0; rep < 3 && s == GP_OK; ++rep) {   // the third repetition is kept
        cudaEventRecord(e0, st);
        k_peak_dmma<<<blocks, PK_THREADS, 0, st>>>(in, out, iters);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) s = GP_ERR_CUDA;
        cudaEventElapsedTime(&ms_dmma, e0, e1);
        cudaEventRecord(e0, st);
        k_peak_dfma<<<blocks, PK_THREADS, 0, st>>>(in, out, iters);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) s = GP_ERR_CUDA;
        cudaEventElapsedTime(&ms_dfma, e0, e1);
    }
    if (cudaGetLastError() != cudaSuccess) s = GP_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(in);
    cudaFree(out);
    if (s != GP_OK) return s;
    const double warps = (double)blocks * PK_THREADS / 32.0;
    *dmma_tflops = warps * iters * PK_CHAINS * 512.0 / (ms_dmma * 1e-3) / 1e12;
    *dfma_tflops = (double)blocks * PK_THREADS * iters * PK_CHAINS * 2.0 / (ms_dfma * 1e-3) / 1e12;
    return GP_OK;
}
