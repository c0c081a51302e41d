// FP64 Cholesky factor and inverse of one diagonal tile, spread over the
// whole GPU (GP_FP64_OZAKI).
//
// On this part one SM retires about 1.7 FP64 FMAs per clock, so the b x b
// diagonal tile's factor and inverse (b^3 / 3 FMAs, 5.6e6 at b = 256) take
// milliseconds on the one CTA of the native path.  Here one cooperative launch
// of about one CTA per SM does the same arithmetic in 32 x 32 blocks (P = b /
// 32 block rows):
//
//  - right-looking blocked Cholesky (Fig. 1's POTRF / TRSM / SYRK-GEMM at the
//    block level), for p = 0 .. P-1:
//      (a) CTA 0 factors the 32 x 32 block A_pp = L_pp L_pp^T and inverts it
//          (X_pp = L_pp^{-1}), both in shared memory;
//      (b) every CTA takes 8-row strips of the panel L_rp = A_rp X_pp^T, r > p;
//      (c) every CTA takes 8-row strips of the trailing update
//          A_ij -= L_ip L_jp^T, p < j <= i;
//  - then the inverse X = L^{-1} by recursive doubling: groups of w blocks
//    merge pairwise, w = 1, 2, 4, ...; for a pair with first half A and
//    second half C, X_CA = -X_CC (L_CA X_AA), the inner product T = L_CA X_AA
//    kept in the (still unused) strict upper triangle of X;
//  - phases are separated by a grid barrier (arrival counter and generation
//    word; every wait bounded, a timeout sets *err and the kernel leaves).
//
// A non-positive pivot records its global row in *info (as the one-CTA
// factor does); every CTA sees it after the next barrier and leaves.  On
// return A holds L (strict upper triangle zero), X = L^{-1} (strict upper
// triangle zero), *logdet_slot = sum of log L_jj (summed in block order).
#include <math.h>

#include "gp_internal.cuh"
#include "se_common.cuh"

namespace gpk {
namespace {

constexpr int PG_NB = 32;       // block edge
constexpr int PG_TH = 256;      // threads per CTA (8 warps)
constexpr int PG_ROWS = 8;      // rows of one work unit: 8 x 32 outputs, one per thread
constexpr int PG_LD = PG_NB + 1;

struct PgArgs {
    double* A;                  // b x b tile, row-major (row stride b), lower triangle meaningful
    double* X;                  // b x b output L^{-1}
    int64_t b;
    int64_t row0;               // global row of the tile's first row (pivot reports)
    double* logdet_slot;
    unsigned long long* info;
    unsigned* bar;              // arrival count, generation (zeroed before the launch)
    int* err;
    long long limit;            // bound on one barrier wait, in SM clock cycles
};

__device__ bool pg_barrier(const PgArgs& a, int* okb)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned* count = a.bar;
        unsigned* gen = a.bar + 1;
        unsigned g;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(g) : "l"(gen) : "memory");
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            *count = 0;
            __threadfence();
            asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(gen), "r"(g + 1) : "memory");
        } else {
            const long long t0 = clock64();
            while (true) {
                unsigned v;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(gen) : "memory");
                if (v != g) break;
                if (clock64() - t0 > a.limit) {
                    atomicExch(a.err, 1);
                    *okb = 0;
                    break;
                }
            }
        }
    }
    __syncthreads();
    return *okb != 0;
}

// Element (r, c) of block (bi, bj) of a b x b row-major matrix.
__device__ __forceinline__ double* blk(double* M, int64_t b, int bi, int bj)
{
    return M + (int64_t)bi * PG_NB * b + (int64_t)bj * PG_NB;
}

// acc += Aop(strip rows r0 .. r0+7 of block Ab) x Bop, with Bop(kk, c) = Bb[c][kk]
// (trans) or Bb[kk][c]; both operands staged in shared memory; thread (warp r,
// lane c) owns output (r, c).
__device__ __forceinline__ void pg_term(double& acc, const double* Ab, int r0, const double* Bb, bool trans,
                                        int64_t b, double* As, double* Bs)
{
    const int tid = threadIdx.x, r = tid >> 5, c = tid & 31;
    __syncthreads();   // the previous term's operands are no longer read
    As[r * PG_LD + c] = __ldcg(Ab + (int64_t)(r0 + r) * b + c);
#pragma unroll
    for (int q = 0; q < PG_NB / PG_ROWS; ++q) {
        const int rr = r + PG_ROWS * q;   // row rr of the B block, column c
        const double v = __ldcg(Bb + (int64_t)rr * b + c);
        if (trans) Bs[c * PG_LD + rr] = v;   // Bs[kk][c'] = Bb[c'][kk]
        else Bs[rr * PG_LD + c] = v;
    }
    __syncthreads();
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int kk = 0; kk < PG_NB; kk += 2) {
        s0 = fma(As[r * PG_LD + kk], Bs[kk * PG_LD + c], s0);
        s1 = fma(As[r * PG_LD + kk + 1], Bs[(kk + 1) * PG_LD + c], s1);
    }
    acc += s0 + s1;
}

// (a): factor and invert block (p, p) in shared memory (CTA 0).  Returns false
// on a non-positive pivot (recorded in *info).
__device__ bool pg_diag(const PgArgs& a, int p, double* S, double* Iv, double* logacc, int* fail)
{
    const int tid = threadIdx.x;
    double* App = blk(a.A, a.b, p, p);
    for (int e = tid; e < PG_NB * PG_NB; e += PG_TH) {
        const int r = e >> 5, c = e & 31;
        S[r * PG_LD + c] = (c <= r) ? __ldcg(App + (int64_t)r * a.b + c) : 0.0;
        Iv[r * PG_LD + c] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    // right-looking: pivot, column scaling, rank-1 update of the trailing lower triangle
    for (int j = 0; j < PG_NB; ++j) {
        if (tid == 0) {
            const double piv = S[j * PG_LD + j];
            if (piv > 0.0) {
                S[j * PG_LD + j] = sqrt(piv);
            } else {
                *fail = 1;
                atomicMin(a.info, (unsigned long long)(a.row0 + (int64_t)p * PG_NB + j));
            }
        }
        __syncthreads();
        if (*fail) return false;
        const double djj = S[j * PG_LD + j];
        if (tid > j && tid < PG_NB) S[tid * PG_LD + j] /= djj;
        __syncthreads();
        const int n = PG_NB - 1 - j;   // trailing order
        for (int e = tid; e < n * n; e += PG_TH) {
            const int r = j + 1 + e / n, c = j + 1 + e % n;
            if (c <= r) S[r * PG_LD + c] = fma(-S[r * PG_LD + j], S[c * PG_LD + j], S[r * PG_LD + c]);
        }
        __syncthreads();
    }
    if (tid < 32) {
        double lg = log(S[tid * PG_LD + tid]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lg += __shfl_xor_sync(0xffffffffu, lg, o);
        if (tid == 0) *logacc += lg;
    }
    // inverse by column-oriented forward substitution: for t = 0 .. 31, row t of
    // X is final after dividing by L_tt; then X(r, c) -= L(r, t) X(t, c) for r > t
    for (int t = 0; t < PG_NB; ++t) {
        if (tid <= t) Iv[t * PG_LD + tid] /= S[t * PG_LD + t];
        __syncthreads();
        const int n = PG_NB - 1 - t;
        for (int e = tid; e < n * (t + 1); e += PG_TH) {
            const int r = t + 1 + e / (t + 1), c = e % (t + 1);
            Iv[r * PG_LD + c] = fma(-S[r * PG_LD + t], Iv[t * PG_LD + c], Iv[r * PG_LD + c]);
        }
        __syncthreads();
    }
    double* Xpp = blk(a.X, a.b, p, p);
    for (int e = tid; e < PG_NB * PG_NB; e += PG_TH) {
        const int r = e >> 5, c = e & 31;
        App[(int64_t)r * a.b + c] = S[r * PG_LD + c];
        Xpp[(int64_t)r * a.b + c] = Iv[r * PG_LD + c];
    }
    return true;
}

__global__ __launch_bounds__(PG_TH) void k_potrf_grid(const PgArgs a)
{
    __shared__ double As[PG_ROWS * PG_LD];
    __shared__ double Bs[PG_NB * PG_LD];
    __shared__ double S[PG_NB * PG_LD];
    __shared__ double Iv[PG_NB * PG_LD];
    __shared__ double logacc;
    __shared__ int okb, fail;
    // No early exit on an earlier failure here: CTA 0 may record a failing
    // pivot before a late CTA starts, and a CTA that left before the first
    // barrier would stall the others.  Every CTA reads *info after the first
    // barrier instead, where it is the same for all of them.
    const int tid = threadIdx.x, r = tid >> 5, c = tid & 31;
    if (tid == 0) {
        okb = 1;
        fail = 0;
        logacc = 0.0;
    }
    __syncthreads();
    const int P = (int)(a.b / PG_NB);
    const int64_t b = a.b;
    const int units_per_blk = PG_NB / PG_ROWS;

    for (int p = 0; p < P; ++p) {
        if (blockIdx.x == 0) pg_diag(a, p, S, Iv, &logacc, &fail);
        if (!pg_barrier(a, &okb) || failed(a.info)) return;
        if (p + 1 == P) break;
        // (b) panel strips: L_rp = A_rp X_pp^T, in place (the strip is staged first)
        const int nb_ = (P - 1 - p) * units_per_blk;
        for (int u = blockIdx.x; u < nb_; u += gridDim.x) {
            const int bi = p + 1 + u / units_per_blk, r0 = (u % units_per_blk) * PG_ROWS;
            double* Arp = blk(a.A, b, bi, p);
            double acc = 0.0;
            pg_term(acc, Arp, r0, blk(a.X, b, p, p), true, b, As, Bs);
            Arp[(int64_t)(r0 + r) * b + c] = acc;
        }
        if (!pg_barrier(a, &okb)) return;
        // (c) trailing update strips: A_ij -= L_ip L_jp^T, p < j <= i
        const int n = P - 1 - p;
        const int nu = n * (n + 1) / 2 * units_per_blk;
        for (int u = blockIdx.x; u < nu; u += gridDim.x) {
            int64_t ii, jj;
            tri_decode(u / units_per_blk, ii, jj);
            const int bi = p + 1 + (int)ii, bj = p + 1 + (int)jj, r0 = (u % units_per_blk) * PG_ROWS;
            double acc = 0.0;
            pg_term(acc, blk(a.A, b, bi, p), r0, blk(a.A, b, bj, p), true, b, As, Bs);
            double* q = blk(a.A, b, bi, bj) + (int64_t)(r0 + r) * b + c;
            *q = __ldcg(q) - acc;
        }
        if (!pg_barrier(a, &okb)) return;
    }
    // inverse: pairs of w-block groups, A = [a0, a0 + w), C = [a0 + w, min(a0 + 2w, P))
    for (int w = 1; w < P; w *= 2) {
        const int npair = (P + 2 * w - 1) / (2 * w);
        // T(i, j) = sum_{k = j}^{a0 + w - 1} L(i, k) X(k, j), i in C, j in A; kept in block (j, i)
        // of X (strict upper triangle, unused until the end)
        {
            int nu = 0;
            for (int g = 0; g < npair; ++g) {
                const int c0 = 2 * w * g + w, c1 = min(2 * w * g + 2 * w, P);
                nu += (c1 > c0 ? c1 - c0 : 0) * w * units_per_blk;
            }
            for (int u = blockIdx.x; u < nu; u += gridDim.x) {
                int rem = u, g = 0;
                for (;; ++g) {
                    const int c0 = 2 * w * g + w, c1 = min(2 * w * g + 2 * w, P);
                    const int cnt = (c1 > c0 ? c1 - c0 : 0) * w * units_per_blk;
                    if (rem < cnt) break;
                    rem -= cnt;
                }
                const int a0 = 2 * w * g, c0 = a0 + w;
                const int bi = c0 + rem / (w * units_per_blk);
                const int bj = a0 + (rem / units_per_blk) % w;
                const int r0 = (rem % units_per_blk) * PG_ROWS;
                double acc = 0.0;
                for (int k = bj; k < a0 + w; ++k)
                    pg_term(acc, blk(a.A, b, bi, k), r0, blk(a.X, b, k, bj), false, b, As, Bs);
                blk(a.X, b, bj, bi)[(int64_t)(r0 + r) * b + c] = acc;
            }
        }
        if (!pg_barrier(a, &okb)) return;
        // X(i, j) = -sum_{k = c0}^{i} X(i, k) T(k, j), i in C, j in A
        {
            int nu = 0;
            for (int g = 0; g < npair; ++g) {
                const int c0 = 2 * w * g + w, c1 = min(2 * w * g + 2 * w, P);
                nu += (c1 > c0 ? c1 - c0 : 0) * w * units_per_blk;
            }
            for (int u = blockIdx.x; u < nu; u += gridDim.x) {
                int rem = u, g = 0;
                for (;; ++g) {
                    const int c0 = 2 * w * g + w, c1 = min(2 * w * g + 2 * w, P);
                    const int cnt = (c1 > c0 ? c1 - c0 : 0) * w * units_per_blk;
                    if (rem < cnt) break;
                    rem -= cnt;
                }
                const int a0 = 2 * w * g, c0 = a0 + w;
                const int bi = c0 + rem / (w * units_per_blk);
                const int bj = a0 + (rem / units_per_blk) % w;
                const int r0 = (rem % units_per_blk) * PG_ROWS;
                double acc = 0.0;
                for (int k = c0; k <= bi; ++k)
                    pg_term(acc, blk(a.X, b, bi, k), r0, blk(a.X, b, bj, k), false, b, As, Bs);
                blk(a.X, b, bi, bj)[(int64_t)(r0 + r) * b + c] = -acc;
            }
        }
        if (!pg_barrier(a, &okb)) return;
    }
    // strict upper triangles of L and X (the latter held the products T)
    for (int64_t e = (int64_t)blockIdx.x * PG_TH + tid; e < b * b; e += (int64_t)gridDim.x * PG_TH) {
        const int64_t rr = e / b, cc = e % b;
        if (cc > rr) {
            a.A[e] = 0.0;
            a.X[e] = 0.0;
        }
    }
    if (blockIdx.x == 0 && tid == 0) *a.logdet_slot = logacc;
}

}  // namespace

// One cooperative launch per diagonal tile; b must be a multiple of 32.
bool potrf_diag_grid(gp_t h, double* A, double* X, int64_t b, int64_t row0, double* logdet_slot)
{
    static int grid_dev = -1, grid_blocks = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (grid_dev != dev) {   // every CTA resident at once: the blocks wait on one another
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_potrf_grid, PG_TH, 0);
        grid_blocks = per >= 1 ? sms : 0;   // one CTA per SM: the FP64 pipe, not occupancy, sets the pace
        grid_dev = dev;
    }
    if (grid_blocks < 1 || b % PG_NB) return false;
    PgArgs a;
    a.A = A;
    a.X = X;
    a.b = b;
    a.row0 = row0;
    a.logdet_slot = logdet_slot;
    a.info = h->info;
    a.bar = (unsigned*)h->solve_flags;
    a.err = tc_error_dev();
    a.limit = 4000000000ll;
    if (!a.err || !a.bar) return false;
    void* args[] = {(void*)&a};
    cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), h->st);   // fresh barrier words
    const bool p_ = h->prof_on && prof_begin(h, GP_PH_POTRF);
    // a failed launch leaves its error for the caller's check of the last launch error
    cudaLaunchCooperativeKernel((const void*)k_potrf_grid, dim3((unsigned)grid_blocks), dim3(PG_TH), args, 0, h->st);
    h->launches++;
    if (p_) prof_end(h);
    h->tc_pending = true;
    return true;
}

}  // namespace gpk
