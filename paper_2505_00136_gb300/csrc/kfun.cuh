// The covariance functions of the library as functions of the squared
// distance r^2: Eq. 2's squared exponential nu exp(-r^2 / (2 l^2)) and the
// Matern kernels nu m(r) of order 1/2, 3/2, 5/2 (s = sqrt(2p) r / l;
// m = exp(-s), (1 + s) exp(-s), (1 + s + s^2 / 3) exp(-s)), with the summand
// of the length-scale derivative that the adjoint reductions accumulate.
#pragma once
#include <math.h>

#include "gp_internal.cuh"

namespace gpk {

// 2p for the Matern order p of a kernel kind (1, 3, 5).
__host__ __device__ __forceinline__ double matern_2p(int kind) { return kind == 1 ? 1.0 : (kind == 2 ? 3.0 : 5.0); }

// k(r^2) without the noise term.
__device__ __forceinline__ double kval(double r2, const GpHyperDev* h)
{
    const int kind = h->kernel;
    if (kind == GP_KERNEL_SE) return h->nu * exp(-r2 * h->inv2l2);
    const double s = sqrt(r2 * matern_2p(kind)) / h->l;
    const double e = exp(-s);
    if (kind == GP_KERNEL_MATERN12) return h->nu * e;
    if (kind == GP_KERNEL_MATERN32) return h->nu * (1.0 + s) * e;
    return h->nu * (1.0 + s + s * s / 3.0) * e;
}

// dk/d(log l) = kdl_term(r^2, k) * kdl_scale: for the squared exponential
// k r^2 (scale 1 / l^2, applied once after the reduction); for a Matern
// kernel, with ds/dlog l = -s, k s, k s^2 / (1 + s) and
// k s^2 (1 + s) / (3 + 3 s + s^2) for p = 1/2, 3/2, 5/2 (scale 1).
__device__ __forceinline__ double kdl_term(double r2, double kf, const GpHyperDev* h)
{
    const int kind = h->kernel;
    if (kind == GP_KERNEL_SE) return kf * r2;
    const double s = sqrt(r2 * matern_2p(kind)) / h->l;
    if (kind == GP_KERNEL_MATERN12) return kf * s;
    if (kind == GP_KERNEL_MATERN32) return kf * s * s / (1.0 + s);
    return kf * s * s * (1.0 + s) / (3.0 + 3.0 * s + s * s);
}

__device__ __forceinline__ float kdl_term_f(float r2, float kf, int kind, float l)
{
    if (kind == GP_KERNEL_SE) return kf * r2;
    const float s = sqrtf(r2 * (float)matern_2p(kind)) / l;
    if (kind == GP_KERNEL_MATERN12) return kf * s;
    if (kind == GP_KERNEL_MATERN32) return kf * s * s / (1.f + s);
    return kf * s * s * (1.f + s) / (3.f + 3.f * s + s * s);
}

__host__ __device__ __forceinline__ double kdl_scale(const GpHyperDev* h)
{
    return h->kernel == GP_KERNEL_SE ? 1.0 / (h->l * h->l) : 1.0;
}

}  // namespace gpk
