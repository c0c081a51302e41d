// Device helpers shared by the FP64 and mixed-precision kernels.
#pragma once
#include <stdint.h>

namespace gpk {

__device__ __forceinline__ bool failed(const unsigned long long* info)
{
    return *(volatile const unsigned long long*)info != ~0ull;
}

// Row index i' of the u-th entry of a lower triangle enumerated row by row.
__device__ __forceinline__ void tri_decode(int64_t u, int64_t& i, int64_t& j)
{
    int64_t r = (int64_t)((sqrt(8.0 * (double)u + 1.0) - 1.0) * 0.5);
    while (r * (r + 1) / 2 > u) --r;
    while ((r + 1) * (r + 2) / 2 <= u) ++r;
    i = r;
    j = u - r * (r + 1) / 2;
}

// ---------------------------------------------------------------- distances
// r2[a][c] for rows p0 + ty + 16a of P and rows q0 + tx + 16c of Q
// (ty = tid / 16, tx = tid % 16), summed over the d coordinates by direct
// differences.  Rows at or beyond np / nq contribute garbage that callers mask.
__device__ __forceinline__ void dist_block(double (&r2)[4][4], const double* P, int64_t p0, int64_t np,
                           const double* Q, int64_t q0, int64_t nq, int64_t d, double* sm)
{
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    double* sp = sm;
    double* sq = sm + 64 * 17;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) r2[a][c] = 0.0;
    for (int64_t d0 = 0; d0 < d; d0 += 16) {
        __syncthreads();
        for (int idx = tid; idx < 1024; idx += 256) {
            int r = idx >> 4, k = idx & 15;
            int64_t gp = p0 + r, gq = q0 + r;
            bool kin = d0 + k < d;
            sp[r * 17 + k] = (gp < np && kin) ? P[gp * d + d0 + k] : 0.0;
            sq[r * 17 + k] = (gq < nq && kin) ? Q[gq * d + d0 + k] : 0.0;
        }
        __syncthreads();
        const int kmax = (int)((d - d0) < 16 ? (d - d0) : 16);
        for (int k = 0; k < kmax; ++k) {
            double pa[4], qc[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) pa[a] = sp[(ty + 16 * a) * 17 + k];
#pragma unroll
            for (int c = 0; c < 4; ++c) qc[c] = sq[(tx + 16 * c) * 17 + k];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    double t = pa[a] - qc[c];
                    r2[a][c] = fma(t, t, r2[a][c]);
                }
        }
    }
}

}  // namespace gpk
