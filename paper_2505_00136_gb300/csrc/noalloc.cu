// Allocation-free predictive mean, gp_predict_mean_noalloc (see include/gprat_gb.h).
//
// Some callers cannot call cudaMalloc at all: serving processes whose device
// memory is fixed at start-up by a pool they do not own, latency-bound loops
// that must not enter the allocator, or plug-ins of a host application that
// forbids allocation after initialisation.  This entry point serves them: it
// computes mean = K_{Z*,Z} alpha (Eq. 3) from caller-owned device buffers and
// keeps its only scratch - per-chunk partial sums - in the file-scope device
// array below, which every GPU that loads the library holds until exit.
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "../../include/gprat_gb.h"
#include "se_common.cuh"

namespace {

constexpr int64_t NOALLOC_MAX_M = GP_NOALLOC_MAX_TEST;      // test points per call
constexpr int64_t NOALLOC_CHUNKS = GP_NOALLOC_CHUNKS;      // training-point chunks
constexpr int NTH = 256;

// NOALLOC_CHUNKS x NOALLOC_MAX_M partial sums (16 MiB).  In host code this
// name is only a stand-in: kernels receive the address from cudaGetSymbolAddress.
static __device__ __align__(256) double g_mean_scratch[NOALLOC_CHUNKS * NOALLOC_MAX_M];

std::mutex g_setup_mutex;
constexpr int MAX_DEVICES = 64;
double* g_scratch_ptr[MAX_DEVICES] = {};

// Partial sums over one chunk of training points for 64 test points:
// part[chunk * m + i] = sum_{j in chunk} nu exp(-|x*_i - x_j|^2 / (2 l^2)) alpha_j.
__global__ __launch_bounds__(NTH) void k_mean_partials_noalloc(const double* X, int64_t n, int64_t d,
                                                               const double* alpha, const double* Xs, int64_t m,
                                                               double nu, double inv2l2, int64_t rows_per_chunk,
                                                               double* part)
{
    __shared__ double sm[2 * 64 * 17];
    const int64_t m0 = (int64_t)blockIdx.x * 64, c = blockIdx.y;
    const int64_t j0 = c * rows_per_chunk;
    const int64_t j1 = (j0 + rows_per_chunk < n) ? j0 + rows_per_chunk : n;
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t n0 = j0; n0 < j1; n0 += 64) {
        double r2[4][4];
        gpk::dist_block(r2, Xs, m0, m, X, n0, j1, d, sm);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t gj = n0 + tx + 16 * q;
                if (gj < j1) s[a] = fma(nu * exp(-r2[a][q] * inv2l2), alpha[gj], s[a]);
            }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) s[a] += __shfl_xor_sync(0xffffffffu, s[a], o);
        const int64_t gi = m0 + ty + 16 * a;
        if (tx == 0 && gi < m) part[c * m + gi] = s[a];
    }
}

__global__ void k_mean_reduce_noalloc(const double* part, int64_t chunks, int64_t m, double* mean)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double s = 0.0;
    for (int64_t c = 0; c < chunks; ++c) s += part[c * m + i];
    mean[i] = s;
}

// True for device memory of the current device, or managed memory.  Device
// memory of another GPU is refused: the kernels would dereference it
// without peer access.
bool on_device(const void* p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does this set-up).
cudaError_t scratch_for_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_mean_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (double*)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" gp_status gp_predict_mean_noalloc(const double* X, const double* alpha, int64_t n, int64_t d,
                                             const double* Xs, int64_t m, double lengthscale, double vertical,
                                             double* mean, void* cuda_stream)
{
    if (!X || !alpha || !Xs || !mean || n < 1 || d < 1 || d > 1024 || m < 1 || m > NOALLOC_MAX_M ||
        !(lengthscale > 0.0) || !(vertical > 0.0) || !isfinite(lengthscale) || !isfinite(vertical))
        return GP_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GP_ERR_CUDA;
    if (!on_device(X, dev) || !on_device(alpha, dev) || !on_device(Xs, dev) || !on_device(mean, dev))
        return GP_ERR_ARG;
    double* part = nullptr;
    if (scratch_for_current_device(&part) != cudaSuccess) return GP_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int64_t chunks = (n + 63) / 64;
    if (chunks > NOALLOC_CHUNKS) chunks = NOALLOC_CHUNKS;
    const int64_t rows_per_chunk = ((n + chunks - 1) / chunks + 63) / 64 * 64;
    chunks = (n + rows_per_chunk - 1) / rows_per_chunk;
    // every partial read below is written first by this call: nothing needs clearing
    k_mean_partials_noalloc<<<dim3((unsigned)((m + 63) / 64), (unsigned)chunks), NTH, 0, st>>>(
        X, n, d, alpha, Xs, m, vertical, 1.0 / (2.0 * lengthscale * lengthscale), rows_per_chunk, part);
    k_mean_reduce_noalloc<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(part, chunks, m, mean);
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}
