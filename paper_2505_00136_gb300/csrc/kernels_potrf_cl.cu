// FP32 Cholesky factor and inverse of one diagonal tile (GP_MIXED) on one
// thread-block cluster of CL_CTAS CTAs.
//
// The diagonal tiles sit on the critical path of the tiled factorisation
// (Fig. 1: POTRF(k) precedes every TRSM and update of step k).  One CTA
// alone takes about 0.3 ms for a tile of 256, so here eight CTAs of one
// cluster share it, synchronised by the cluster's hardware barrier instead
// of a grid barrier, with the tile itself in L2 (global memory, loads that
// bypass L1).  Blocks of 32 x 32, P = b / 32 block rows:
//
//  - right-looking blocked Cholesky, for p = 0 .. P-1:
//      (a) one warp factors A_pp = L_pp L_pp^T in its registers (lane l holds
//          row l, pivots and multipliers broadcast by shuffles) and inverts
//          it (lane c solves L_pp x = e_c), X_pp = L_pp^{-1};
//      (b) every warp of the cluster takes 8-row strips of the panel
//          L_rp = A_rp X_pp^T, r > p;
//      (c) every warp takes 8-row strips of the trailing update
//          A_ij -= L_ip L_jp^T, p < j <= i, with one step of lookahead: four
//          warps of CTA 0 update block (p+1, p+1) first and one of them then
//          factors it (step (a) of p+1) while the other warps finish (c), so
//          each block column costs two cluster barriers and the diagonal
//          factor is off the critical path;
//  - then X = L^{-1} by recursive doubling: groups of w blocks merge
//    pairwise, w = 1, 2, 4, ...; for a pair with first half A and second half
//    C, X_CA = -X_CC (L_CA X_AA), the product L_CA X_AA kept in the strict
//    upper triangle of X until the end;
//  - finally L and X with zero strict upper triangles, the three BF16 planes
//    of X, and sum log L_jj (FP64) into *logdet_slot.
//
// A warp's unit is an 8 x 32 strip: lane c owns column c of the strip, the
// strip of the left operand is held one column per lane and broadcast by
// shuffles, so a unit needs neither shared memory nor a block barrier.
// A pivot that is not positive records its global row in *info; every CTA
// reads *info after the next cluster barrier and all leave together, so no
// CTA ever waits at a barrier that another has left.
#include <math.h>

#include <utility>

#include "gp_internal.cuh"
#include "se_common.cuh"
#include "split_bf16.cuh"

namespace gpk {
namespace {

constexpr int CL_CTAS = 8;                 // CTAs of the cluster
constexpr int CL_TH = 512;                 // threads per CTA
constexpr int CL_WARPS = CL_CTAS * CL_TH / 32;
constexpr int CL_NB = 32;                  // block edge
constexpr int CL_R = 8;                    // rows of a warp unit
constexpr int CL_UPB = CL_NB / CL_R;       // units per block

__device__ __forceinline__ void cluster_sync()
{
    __threadfence();
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

__device__ __forceinline__ float* cblk(float* M, int64_t b, int bi, int bj)
{
    return M + (int64_t)bi * CL_NB * b + (int64_t)bj * CL_NB;
}

// acc[r] += sum_k A(r0 + r, k) Bop(k, lane) over one 32-wide k block, with
// A the block at Ab (row stride b), Bop(k, c) = B[c][k] (trans) or B[k][c].
__device__ __forceinline__ void strip_term(float (&acc)[CL_R], const float* Ab, int r0, const float* Bb, bool trans,
                                           int64_t b, int lane)
{
    float a[CL_R], bc[CL_NB];
#pragma unroll
    for (int r = 0; r < CL_R; ++r) a[r] = __ldcg(Ab + (int64_t)(r0 + r) * b + lane);
    if (trans) {
#pragma unroll
        for (int q = 0; q < CL_NB / 4; ++q) {
            const float4 v = __ldcg(reinterpret_cast<const float4*>(Bb + (int64_t)lane * b) + q);
            bc[4 * q] = v.x;
            bc[4 * q + 1] = v.y;
            bc[4 * q + 2] = v.z;
            bc[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < CL_NB; ++k) bc[k] = __ldcg(Bb + (int64_t)k * b + lane);
    }
#pragma unroll
    for (int k = 0; k < CL_NB; ++k)
#pragma unroll
        for (int r = 0; r < CL_R; ++r) acc[r] = fmaf(__shfl_sync(0xffffffffu, a[r], k), bc[k], acc[r]);
}

// Step J of the register-resident 32 x 32 factor (lane l holds row l).
template <int J>
__device__ __forceinline__ void chol32f_step(float (&row)[32], int l, int& bad, float& dinv)
{
    const float d = __shfl_sync(0xffffffffu, row[J], J);
    if (!(d > 0.f) && bad < 0) bad = J;
    const float inv = rsqrtf(d), dj = d * inv;   // the factor is FP32-level: approximate 1/sqrt suffices
    if (l == J) dinv = inv;
    row[J] = (l == J) ? dj : row[J] * inv;
#pragma unroll
    for (int c = J + 1; c < 32; ++c) row[c] = fmaf(-row[J], __shfl_sync(0xffffffffu, row[J], c), row[c]);
}

template <int... J>
__device__ __forceinline__ void chol32f_steps(float (&row)[32], int l, int& bad, float& dinv,
                                              std::integer_sequence<int, J...>)
{
    (chol32f_step<J>(row, l, bad, dinv), ...);
}

// Row R of L x = e_c (L in S, row stride 33; dv[R] = 1 / L_RR).
template <int R>
__device__ __forceinline__ void trinv32f_row(const float* S, const float* dv, int c, float (&x)[32])
{
    float s4[4] = {(R == c) ? 1.f : 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int t = 0; t < R; ++t) s4[t & 3] = fmaf(-S[R * 33 + t], x[t], s4[t & 3]);
    x[R] = ((s4[0] + s4[1]) + (s4[2] + s4[3])) * dv[R];
}

template <int... R>
__device__ __forceinline__ void trinv32f_rows(const float* S, const float* dv, int c, float (&x)[32],
                                              std::integer_sequence<int, R...>)
{
    (trinv32f_row<R>(S, dv, c, x), ...);
}

struct ClArgs {
    float* A;                   // b x b tile (lower triangle read), in place: L
    float* X;                   // b x b: L^{-1}
    __nv_bfloat16* XP;          // three planes of X (plane q at XP + q b^2)
    int64_t b;
    int64_t row0;               // global row of the tile's first row (pivot reports)
    double* logdet_slot;
    unsigned long long* info;
};

// (a) on one warp: factor and invert block (p, p); sum of log L_jj added to
// *logacc.  A failing pivot is recorded in *info.
__device__ void cl_diag(const ClArgs& a, int p, float* S, float* dv, double* logacc, int lane)
{
    const int64_t b = a.b;
    float* App = cblk(a.A, b, p, p);
    float row[32];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 v = __ldcg(reinterpret_cast<const float4*>(App + (int64_t)lane * b) + q);
        row[4 * q] = v.x;
        row[4 * q + 1] = v.y;
        row[4 * q + 2] = v.z;
        row[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int c = 0; c < 32; ++c)
        if (c > lane) row[c] = 0.f;
    int bad = -1;
    float dinv = 0.f;
    chol32f_steps(row, lane, bad, dinv, std::make_integer_sequence<int, 32>{});
    if (bad >= 0) {   // the same pivot on every lane
        if (lane == 0) atomicMin(a.info, (unsigned long long)(a.row0 + (int64_t)p * CL_NB + bad));
        return;
    }
    float dl = 1.f;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        if (c == lane) dl = row[c];
        if (c > lane) row[c] = 0.f;
        S[lane * 33 + c] = row[c];
    }
    dv[lane] = dinv;
    double lg = log((double)dl);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lg += __shfl_xor_sync(0xffffffffu, lg, o);
    if (lane == 0) *logacc += lg;
#pragma unroll
    for (int q = 0; q < 8; ++q)
        reinterpret_cast<float4*>(App + (int64_t)lane * b)[q] =
            make_float4(row[4 * q], row[4 * q + 1], row[4 * q + 2], row[4 * q + 3]);
    __syncwarp();
    float x[32];
    trinv32f_rows(S, dv, lane, x, std::make_integer_sequence<int, 32>{});
    float* Xpp = cblk(a.X, b, p, p);
#pragma unroll
    for (int r = 0; r < 32; ++r) Xpp[(int64_t)r * b + lane] = x[r];
}

// Pairs of w-block groups of the inverse: the u-th 8-row unit of the pairs'
// blocks (i in C, j in A): bi = i, bj = j, r0 its first row; false past the end.
__device__ __forceinline__ bool pair_unit(int u, int w, int P, int& a0, int& c0, int& bi, int& bj, int& r0)
{
    for (int g = 0;; ++g) {
        a0 = 2 * w * g;
        if (a0 + w >= P) return false;
        c0 = a0 + w;
        const int c1 = min(a0 + 2 * w, P);
        const int cnt = (c1 - c0) * w * CL_UPB;
        if (u < cnt) {
            bi = c0 + u / (w * CL_UPB);
            bj = a0 + (u / CL_UPB) % w;
            r0 = (u % CL_UPB) * CL_R;
            return true;
        }
        u -= cnt;
    }
}

// One 8-row strip of the trailing update of step p: A_ij -= L_ip L_jp^T for
// the u-th unit of the lower block triangle below block (p, p).
__device__ __forceinline__ void cl_update_unit(const ClArgs& a, int p, int u, int lane)
{
    const int64_t b = a.b;
    int64_t ii, jj;
    tri_decode(u / CL_UPB, ii, jj);
    const int bi = p + 1 + (int)ii, bj = p + 1 + (int)jj, r0 = (u % CL_UPB) * CL_R;
    float acc[CL_R] = {};
    strip_term(acc, cblk(a.A, b, bi, p), r0, cblk(a.A, b, bj, p), true, b, lane);
    float* q = cblk(a.A, b, bi, bj) + (int64_t)r0 * b + lane;
#pragma unroll
    for (int r = 0; r < CL_R; ++r) q[(int64_t)r * b] = __ldcg(q + (int64_t)r * b) - acc[r];
}

__global__ __launch_bounds__(CL_TH, 1) void k_potrf_cl(const ClArgs a)
{
    __shared__ float S[32 * 33];
    __shared__ float dv[32];
    double logacc = 0.0;   // lane 0 of warp 0 of CTA 0
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * (CL_TH / 32) + warp;
    const bool lead = blockIdx.x == 0 && warp < CL_UPB;   // the lookahead warps
    const int P = (int)(a.b / CL_NB);
    const int64_t b = a.b;

    if (gw == 0) cl_diag(a, 0, S, dv, &logacc, lane);
    cluster_sync();
    if (failed(a.info)) return;   // every CTA reads the same word after the same barrier
    for (int p = 0; p + 1 < P; ++p) {
        // (b) panel strips L_rp = A_rp X_pp^T, in place (each strip is read by its own warp only)
        const int np = (P - 1 - p) * CL_UPB;
        for (int u = gw; u < np; u += CL_WARPS) {
            const int bi = p + 1 + u / CL_UPB, r0 = (u % CL_UPB) * CL_R;
            float acc[CL_R] = {};
            float* Arp = cblk(a.A, b, bi, p);
            strip_term(acc, Arp, r0, cblk(a.X, b, p, p), true, b, lane);
#pragma unroll
            for (int r = 0; r < CL_R; ++r) Arp[(int64_t)(r0 + r) * b + lane] = acc[r];
        }
        cluster_sync();
        // (c) trailing update; units 0 .. CL_UPB-1 are block (p+1, p+1), taken by the
        // lookahead warps, which then factor it (step (a) of p+1)
        const int n = P - 1 - p;
        const int nu = n * (n + 1) / 2 * CL_UPB;
        if (lead) {
            cl_update_unit(a, p, warp, lane);
            __threadfence();
            asm volatile("bar.sync 1, %0;\n" ::"n"(CL_UPB * 32) : "memory");
            if (warp == 0) cl_diag(a, p + 1, S, dv, &logacc, lane);
        } else {
            // the other warps, numbered from 0 (the lookahead warps are gw 0 .. CL_UPB-1)
            for (int u = gw; u < nu; u += CL_WARPS - CL_UPB) cl_update_unit(a, p, u, lane);
        }
        cluster_sync();
        if (failed(a.info)) return;
    }
    // inverse by recursive doubling
    for (int w = 1; w < P; w *= 2) {
        // T(i, j) = sum_{k = j}^{a0 + w - 1} L(i, k) X(k, j) into block (j, i) of X
        for (int u = gw;; u += CL_WARPS) {
            int a0, c0, bi, bj, r0;
            if (!pair_unit(u, w, P, a0, c0, bi, bj, r0)) break;
            float acc[CL_R] = {};
            for (int k = bj; k < a0 + w; ++k)
                strip_term(acc, cblk(a.A, b, bi, k), r0, cblk(a.X, b, k, bj), false, b, lane);
            float* q = cblk(a.X, b, bj, bi) + (int64_t)r0 * b + lane;
#pragma unroll
            for (int r = 0; r < CL_R; ++r) q[(int64_t)r * b] = acc[r];
        }
        cluster_sync();
        // X(i, j) = -sum_{k = c0}^{i} X(i, k) T(k, j)
        for (int u = gw;; u += CL_WARPS) {
            int a0, c0, bi, bj, r0;
            if (!pair_unit(u, w, P, a0, c0, bi, bj, r0)) break;
            float acc[CL_R] = {};
            for (int k = c0; k <= bi; ++k)
                strip_term(acc, cblk(a.X, b, bi, k), r0, cblk(a.X, b, bj, k), false, b, lane);
            float* q = cblk(a.X, b, bi, bj) + (int64_t)r0 * b + lane;
#pragma unroll
            for (int r = 0; r < CL_R; ++r) q[(int64_t)r * b] = -acc[r];
        }
        cluster_sync();
    }
    // zero strict upper triangles (X's held the products T), planes of X
    const int64_t bb = b * b;
    for (int64_t e = (int64_t)blockIdx.x * CL_TH + threadIdx.x; e < bb; e += (int64_t)CL_CTAS * CL_TH) {
        const int64_t rr = e / b, cc = e % b;
        float xv = 0.f;
        if (cc > rr) {
            a.A[e] = 0.f;
            a.X[e] = 0.f;
        } else {
            xv = __ldcg(a.X + e);
        }
        __nv_bfloat16 hi, mid, lo;
        split3(xv, hi, mid, lo);
        a.XP[e] = hi;
        a.XP[bb + e] = mid;
        a.XP[2 * bb + e] = lo;
    }
    if (gw == 0 && lane == 0) *a.logdet_slot = logacc;
}

}  // namespace

bool potrf_diag_cl32(gp_t h, float* A32, float* X32, __nv_bfloat16* XP, int64_t b, int64_t row0, double* logdet_slot)
{
    if (b % CL_NB || b < CL_NB) return false;
    ClArgs a{A32, X32, XP, b, row0, logdet_slot, h->info};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL_CTAS);
    cfg.blockDim = dim3(CL_TH);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = h->st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL_CTAS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool p_ = h->prof_on && prof_begin(h, GP_PH_POTRF);
    // a failed launch leaves its error for the caller's check of the last launch error
    cudaLaunchKernelEx(&cfg, k_potrf_cl, a);
    h->launches++;
    if (p_) prof_end(h);
    return true;
}

}  // namespace gpk
