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

#include <utility>

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

// Step J of the 32 x 32 factor held in one warp's registers (lane l holds
// row l): pivot, column J scaled by 1 / L_JJ, rank-1 update of the later
// columns.  Entries above the diagonal are scratch.  bad = first pivot that
// is not positive; dinv = 1 / L_ll on lane l.
template <int J>
__device__ __forceinline__ void chol32_step(double (&row)[32], int l, int& bad, double& dinv)
{
    const double d = __shfl_sync(0xffffffffu, row[J], J);
    if (!(d > 0.0) && bad < 0) bad = J;
    const double dj = sqrt(d), inv = 1.0 / dj;
    if (l == J) dinv = inv;
    row[J] = (l == J) ? dj : row[J] * inv;
#pragma unroll
    for (int c = J + 1; c < 32; ++c) row[c] = fma(-row[J], __shfl_sync(0xffffffffu, row[J], c), row[c]);
}

template <int... J>
__device__ __forceinline__ void chol32_steps(double (&row)[32], int l, int& bad, double& dinv,
                                             std::integer_sequence<int, J...>)
{
    (chol32_step<J>(row, l, bad, dinv), ...);
}

// Row R of the forward substitution L x = e_c (L in S, row stride PG_LD;
// dv[R] = 1 / L_RR): rows above c come out exactly zero.
template <int R>
__device__ __forceinline__ void trinv32_row(const double* S, const double* dv, int c, double (&x)[32])
{
    double s4[4] = {(R == c) ? 1.0 : 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int t = 0; t < R; ++t) s4[t & 3] = fma(-S[R * PG_LD + t], x[t], s4[t & 3]);
    x[R] = ((s4[0] + s4[1]) + (s4[2] + s4[3])) * dv[R];
}

template <int... R>
__device__ __forceinline__ void trinv32_rows(const double* S, const double* dv, int c, double (&x)[32],
                                             std::integer_sequence<int, R...>)
{
    (trinv32_row<R>(S, dv, c, x), ...);
}

// (a): factor and invert block (p, p) (CTA 0).  Warp 0 factors the block in
// registers and then, lane c for column c, inverts it by forward
// substitution; the other warps only stage the block in and out.  Returns
// false on a pivot that is not positive (recorded in *info).
__device__ bool pg_diag(const PgArgs& a, int p, double* S, double* Iv, double* logacc, int* fail)
{
    const int tid = threadIdx.x;
    double* App = blk(a.A, a.b, p, p);
    double* dv = Iv + PG_NB * PG_LD;   // 32 reciprocals of the pivots
    for (int e = tid; e < PG_NB * PG_NB; e += PG_TH) {
        const int r = e >> 5, c = e & 31;
        S[r * PG_LD + c] = (c <= r) ? __ldcg(App + (int64_t)r * a.b + c) : 0.0;
    }
    __syncthreads();
    if (tid < 32) {
        const int l = tid;
        double row[32], dinv = 0.0;
#pragma unroll
        for (int c = 0; c < 32; ++c) row[c] = S[l * PG_LD + c];
        int bad = -1;
        chol32_steps(row, l, bad, dinv, std::make_integer_sequence<int, 32>{});
        if (bad >= 0) {   // the same pivot on every lane
            if (l == 0) {
                *fail = 1;
                atomicMin(a.info, (unsigned long long)(a.row0 + (int64_t)p * PG_NB + bad));
            }
        } else {
#pragma unroll
            for (int c = 0; c < 32; ++c) S[l * PG_LD + c] = (c <= l) ? row[c] : 0.0;
            dv[l] = dinv;
            double dl = 1.0;
#pragma unroll
            for (int c = 0; c < 32; ++c)
                if (c == l) dl = row[c];
            double lg = log(dl);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) lg += __shfl_xor_sync(0xffffffffu, lg, o);
            if (l == 0) *logacc += lg;
        }
        __syncwarp();
        if (!*fail) {
            double x[32];
            trinv32_rows(S, dv, l, x, std::make_integer_sequence<int, 32>{});
#pragma unroll
            for (int r = 0; r < 32; ++r) Iv[r * PG_LD + l] = x[r];
        }
    }
    __syncthreads();
    if (*fail) return false;
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
    __shared__ double Iv[PG_NB * PG_LD + PG_NB];
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
    // strict upper triangles of L and X are zero (X's held the products T)
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
    if (grid_blocks < 1 || b % PG_NB || b < PG_NB) return false;
    PgArgs a{};
    a.A = A;
    a.X = X;
    a.b = b;
    a.row0 = row0;
    a.logdet_slot = logdet_slot;
    a.info = h->info;
    a.bar = (unsigned*)h->solve_flags;
    a.err = tc_error_dev();
    a.limit = 4000000000ll;   // about 2 s at the maximum SM clock
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
