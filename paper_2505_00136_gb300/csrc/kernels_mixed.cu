// Mixed-precision hot path (GP_MIXED): FP32-accurate split-BF16 tile products
// on the BF16 tensor pipe, FP64 where accuracy is decided.
//
//  - K is assembled once in FP64 (kept for residuals, the exact product and
//    the gradient) and in FP32 (working copy).
//  - Tiled right-looking Cholesky (Fig. 1) on the FP32 copy, in super-panels
//    of SWEEP_BLOCK tile columns: each diagonal tile is factored and inverted
//    in FP32 by one cluster of eight CTAs (kernels_potrf_cl.cu), the panel
//    TRSM (L_ik = A_ik Linv_kk^T) and the trailing SYRK/GEMM run as bf16x6
//    products with FP32 accumulation on the tensor cores (kernels_tgemm.cu).  Every finished off-diagonal
//    tile of L is also kept as three BF16 planes, the operand format of later
//    products.
//  - log|K| = 2 sum log L_jj, the logarithms taken and summed in FP64.
//  - alpha = K^{-1} y by iterative refinement: FP32 triangular solves with the
//    mixed factor (one cooperative launch per solve, k_solve32p), residual
//    y - K alpha in FP64 against the FP64 K (k_sym_resid).
//  - Prediction: the mean is K_{Z*,Z} alpha in FP64 (fused into the cross-
//    covariance assembly).  Variances: W = K_{Z*,Z} L^{-T} from bf16x6
//    products gives x0 = L^{-T} W^T, rounded to x~0 (14 bits per test point);
//    with r0 = k* - K x~0 from the exact digit product (kernels_tc.cu) the
//    quadratic form is k*^T x~0 + x~0^T r0 + ||L^{-1} r0||^2, FP64-accurate up
//    to a third-order term; without the correction var = k** - rowsum(W^2).
#include <cuda_bf16.h>
#include <math.h>

#include <utility>

#include "digits.cuh"
#include "split_bf16.cuh"
#include "gp_internal.cuh"
#include "se_common.cuh"
#include "kfun.cuh"

namespace gpk {

constexpr int NTH = 256;

// Planes of the panel tiles A32_(i,k), i = k+1..T-1, into PA (one slot per tile).
__global__ void k_split_panel(const float* A32, __nv_bfloat16* PA, int64_t b, int64_t k)
{
    const int64_t bb = b * b;
    const int64_t i = k + 1 + blockIdx.y;
    const float* src = A32 + tri_index(i, k) * bb;
    __nv_bfloat16* dst = PA + (int64_t)blockIdx.y * 3 * bb;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < bb;
         e += (int64_t)gridDim.x * blockDim.x) {
        __nv_bfloat16 hi, mid, lo;
        split3(src[e], hi, mid, lo);
        dst[e] = hi;
        dst[bb + e] = mid;
        dst[2 * bb + e] = lo;
    }
}

// ---------------------------------------------------------------- FP32 triangular solves
// The refinement's solves run in super-blocks of SB_TILES diagonal tiles
// (edge B = SB_TILES b): the T-step recurrence over tiles becomes a
// ceil(T / SB_TILES)-step recurrence over super-blocks, each step one
// product with the super-block's inverse X_I = L~_II^{-1} and one sweep of
// the factor's rows below (or columns left of) it.  X_I is built once per
// factorisation from the tile inverses by recursive doubling, exactly as the
// tile inverses are built from 32-blocks: groups of w tiles merge pairwise,
// X_CA = -X_CC (L_CA X_AA), with the product T = L_CA X_AA kept in the
// (otherwise unused) upper tiles of X_I.  Each X_I is dense row-major with
// row stride B; only its lower tiles are read by the solves.
constexpr int SB_TILES = GP_SOLVE_SB;

// acc += A (64 x K, row stride lda) * B (K x 64, row stride ldb), FP32; 256
// threads, thread (tr, tc) owns rows 4 tr .. 4 tr + 3, columns 4 tc .. 4 tc + 3.
// K a multiple of 32; both operands 16-byte aligned rows.
constexpr int SBG_LD = 68;   // padded k-major chunk row (16-byte aligned)
__device__ void sb_gemm64(float (&acc)[4][4], const float* A, int64_t lda, const float* B, int64_t ldb, int64_t K,
                          float* As, float* Bs)
{
    const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
    for (int64_t k0 = 0; k0 < K; k0 += 32) {
        float4 a[2], bv[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int e = tid + q * NTH;               // 512 float4 of each chunk
            const int ar = e >> 3, ak = (e & 7) * 4;   // A: 64 rows x 8 float4
            a[q] = __ldcg((const float4*)(A + (int64_t)ar * lda + k0 + ak));
            const int bk = e >> 4, bc = (e & 15) * 4;  // B: 32 rows x 16 float4
            bv[q] = __ldcg((const float4*)(B + (k0 + bk) * ldb + bc));
        }
        __syncthreads();   // the previous chunk is no longer read
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int e = tid + q * NTH;
            const int ar = e >> 3, ak = (e & 7) * 4;
            As[(ak + 0) * SBG_LD + ar] = a[q].x;
            As[(ak + 1) * SBG_LD + ar] = a[q].y;
            As[(ak + 2) * SBG_LD + ar] = a[q].z;
            As[(ak + 3) * SBG_LD + ar] = a[q].w;
            const int bk = e >> 4, bc = (e & 15) * 4;
            *(float4*)(Bs + bk * SBG_LD + bc) = bv[q];
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            const float4 a4 = *(const float4*)(As + kk * SBG_LD + 4 * tr);
            const float4 b4 = *(const float4*)(Bs + kk * SBG_LD + 4 * tc);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bw[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(av[x], bw[y], acc[x][y]);
        }
    }
}

// Diagonal tiles of every X_I: the tile inverses.
__global__ void k_sbinv_diag(const float* Linv32, float* Xsb, int64_t b, int64_t T)
{
    const int64_t t = blockIdx.y, I = t / SB_TILES, r = t % SB_TILES, SBb = SB_TILES * b;
    const float* src = Linv32 + t * b * b;
    float* dst = Xsb + I * SBb * SBb + r * b * SBb + r * b;
    for (int64_t e = (int64_t)blockIdx.x * NTH + threadIdx.x; e < b * b; e += (int64_t)gridDim.x * NTH)
        dst[(e / b) * SBb + e % b] = __ldcg(src + e);
}

// One phase of the recursive doubling at group width w for every
// super-block: grid (b / 64)^2 sub-tiles x pairs (i in C, j in A) x
// super-blocks.  Phase 1: T(i, j) = sum_{k=j}^{a0+w-1} L(i, k) X(k, j) into
// tile (j, i); phase 2: X(i, j) = -sum_{k=c0}^{i} X(i, k) T(k, j).
__global__ __launch_bounds__(NTH) void k_sbinv_level(const float* A32, float* Xsb, int64_t b, int64_t T, int w,
                                                     int phase)
{
    __shared__ __align__(16) float As[32 * SBG_LD];
    __shared__ __align__(16) float Bs[32 * SBG_LD];
    const int64_t I = blockIdx.z, t0 = I * SB_TILES, SBb = SB_TILES * b;
    const int st = (int)(T - t0 < SB_TILES ? T - t0 : SB_TILES);
    // the blockIdx.y-th (i, j) pair of the super-block at width w
    int u = blockIdx.y, a0 = 0, c0 = 0, i = -1, j = -1;
    for (int g = 0;; ++g) {
        a0 = 2 * w * g;
        if (a0 + w >= st) break;
        c0 = a0 + w;
        const int c1 = min(a0 + 2 * w, st), cnt = (c1 - c0) * w;
        if (u < cnt) {
            i = c0 + u / w;
            j = a0 + u % w;
            break;
        }
        u -= cnt;
    }
    if (i < 0) return;   // fewer pairs in this (ragged) super-block: the whole CTA leaves
    const int nsub = (int)(b / 64), sr = blockIdx.x / nsub, sc = blockIdx.x % nsub;
    float* X = Xsb + I * SBb * SBb;
    auto xt = [&](int r, int c) { return X + (int64_t)r * b * SBb + (int64_t)c * b; };
    float acc[4][4] = {};
    if (phase == 1) {
        for (int k = j; k < a0 + w; ++k)
            sb_gemm64(acc, A32 + tri_index(t0 + i, t0 + k) * b * b + (int64_t)sr * 64 * b, b,
                      xt(k, j) + sc * 64, SBb, b, As, Bs);
    } else {
        for (int k = c0; k <= i; ++k)
            sb_gemm64(acc, xt(i, k) + (int64_t)sr * 64 * SBb, SBb, xt(j, k) + sc * 64, SBb, b, As, Bs);
    }
    float* out = (phase == 1 ? xt(j, i) : xt(i, j)) + (int64_t)sr * 64 * SBb + sc * 64;
    const float sg = phase == 1 ? 1.f : -1.f;
    const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
#pragma unroll
    for (int x = 0; x < 4; ++x)
        *(float4*)(out + (int64_t)(4 * tr + x) * SBb + 4 * tc) =
            make_float4(sg * acc[x][0], sg * acc[x][1], sg * acc[x][2], sg * acc[x][3]);
}

// The three BF16 planes of every X_I (plane q at XsbP + q TS B^2), the
// upper tiles (which held the products T of the doubling) and the unused
// tiles of a short last super-block written as zero: the operand of the
// multi-RHS sweeps' super-block steps.
__global__ void k_split_sbx(const float* Xsb, int64_t b, int64_t T, __nv_bfloat16* XsbP)
{
    const int64_t SBb = SB_TILES * b, TS = (T + SB_TILES - 1) / SB_TILES, total = TS * SBb * SBb;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t I = e / (SBb * SBb), r = (e / SBb) % SBb, c = e % SBb;
        const int64_t st = T - I * SB_TILES < SB_TILES ? T - I * SB_TILES : SB_TILES;   // tiles of super-block I
        const float v = (c / b > r / b || r / b >= st) ? 0.f : __ldcg(Xsb + e);
        __nv_bfloat16 hi, mid, lo;
        split3(v, hi, mid, lo);
        XsbP[e] = hi;
        XsbP[total + e] = mid;
        XsbP[2 * total + e] = lo;
    }
}

// One cooperative launch per solve, every CTA on every step: out = L~^{-1} in
// (upper = 0) or out = L~^{-T} in (upper = 1), FP32 throughout, over
// super-blocks I of st <= SB_TILES tiles (edge B = st b, first tile t0).
// Lower, I = 0 .. TS-1: (A) x_I = X_I (in_I - s_I); (B) s_i += L_iI x_I for
// every row below the super-block.  Upper, I = TS-1 .. 0: (A) x_I = X_I^T
// (in_I - s_I); (B) s_j += L_Ij^T x_I for every tile column j < t0.  A grid
// barrier separates (A) and (B), and (B) from the next (A).  (A): every CTA
// stages v_I = in_I - s_I in shared memory; the rows (lower) or four-column
// groups (upper) of the product are spread over all warps of the grid.
// (B), lower: chunks of SV_CH rows below the super-block, one per CTA at a
// time, eight rows per warp, each row's dot product over the super-block's
// columns held by one warp (one copy of s).  (B), upper: a unit is one tile
// (t0 + r, j); its column sums over the tile's rows are reduced over the
// CTA's warps and added to copy r of s (SB_TILES copies, summed in (A)), so
// every element has one writer per step and the result is deterministic.
// Grid barrier: arrival counter and generation word, each wait bounded by
// wait_limit clock cycles; a timeout sets *err and the kernel leaves.
constexpr int SV_CH = 64;     // rows per chunk in phase (B)
constexpr int SV_SEG = 256;   // columns per pass: lanes hold 4 lane + 128 u, u = 0, 1

__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned nblocks, int* err,
                                             int* okb, long long limit)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned g;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(g) : "l"(gen) : "memory");
        if (atomicAdd(count, 1u) == nblocks - 1) {
            *count = 0;
            __threadfence();
            asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(gen), "r"(g + 1) : "memory");
        } else {
            const long long t0 = clock64();
            while (true) {
                unsigned v;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(gen) : "memory");
                if (v != g) break;
                if (clock64() - t0 > limit) {
                    atomicExch(err, 1);
                    *okb = 0;
                    break;
                }
            }
        }
    }
    __syncthreads();
    return *okb != 0;
}

__device__ __forceinline__ float dot4(const float4& a, const float4& x)
{
    return fmaf(a.x, x.x, fmaf(a.y, x.y, fmaf(a.z, x.z, a.w * x.w)));
}

// Dynamic shared memory: 2 SB_TILES b floats (v_I, x_I).
__global__ __launch_bounds__(NTH) void k_solve32p(const float* Lt, const float* Xsb, int64_t b, int64_t T,
                                                  const float* in, float* out, float* sbuf, int upper, unsigned* bar,
                                                  int* err, long long wait_limit, int stall_last)
{
    static_assert(NTH == 256 && NTH / 32 * 8 == SV_CH && NTH >= SV_SEG, "chunk of 8 warps x 8 rows");
    extern __shared__ __align__(16) float sv_dyn[];
    __shared__ int okb;
    __shared__ __align__(16) float red[8 * SV_SEG];
    const int64_t SBb = SB_TILES * b;
    float* vs = sv_dyn;
    float* xs = sv_dyn + SBb;
    if (threadIdx.x == 0) okb = 1;
    // test aid: the last CTA never arrives, so every other CTA's first barrier wait runs out
    if (stall_last && blockIdx.x == gridDim.x - 1) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * (NTH / 32) + warp, nw = (int64_t)gridDim.x * (NTH / 32);
    const int64_t Np = T * b, TS = (T + SB_TILES - 1) / SB_TILES;
    const int np = upper ? SB_TILES : 1;
    for (int64_t e = (int64_t)blockIdx.x * NTH + threadIdx.x; e < np * Np; e += (int64_t)gridDim.x * NTH)
        sbuf[e] = 0.f;
    if (!grid_barrier(bar, bar + 1, gridDim.x, err, &okb, wait_limit)) return;
    for (int64_t q = 0; q < TS; ++q) {
        const int64_t I = upper ? TS - 1 - q : q, t0 = I * SB_TILES;
        const int st = (int)(T - t0 < SB_TILES ? T - t0 : SB_TILES);
        const int64_t B = st * b, R0 = t0 * b;
        const float* X = Xsb + I * SBb * SBb;
        // (A) v_I in shared memory, then x_I = X_I v_I (rows over the grid's warps) or X_I^T v_I
        for (int64_t e = threadIdx.x; e < B; e += NTH) {
            float v = __ldcg(in + R0 + e);
            for (int k = 0; k < np; ++k) v -= __ldcg(sbuf + k * Np + R0 + e);
            vs[e] = v;
        }
        __syncthreads();
        if (!upper) {
            for (int64_t r = gw; r < B; r += nw) {   // row r: lower tiles only, columns < (r / b + 1) b
                const int64_t ce = (r / b + 1) * b;
                float sum = 0.f;
                for (int64_t c = 4 * lane; c < ce; c += 128)
                    sum += dot4(__ldcg((const float4*)(X + r * SBb + c)), *(const float4*)(vs + c));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                if (lane == 0) out[R0 + r] = sum;
            }
        } else {
            for (int64_t c4 = 4 * gw; c4 < B; c4 += 4 * nw) {   // columns c4 .. c4+3: rows >= (c4 / b) b
                float4 sm = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int64_t r = (c4 / b) * b + lane; r < B; r += 32) {
                    const float4 m = __ldcg((const float4*)(X + r * SBb + c4));
                    const float vr = vs[r];
                    sm.x = fmaf(m.x, vr, sm.x);
                    sm.y = fmaf(m.y, vr, sm.y);
                    sm.z = fmaf(m.z, vr, sm.z);
                    sm.w = fmaf(m.w, vr, sm.w);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    sm.x += __shfl_xor_sync(0xffffffffu, sm.x, o);
                    sm.y += __shfl_xor_sync(0xffffffffu, sm.y, o);
                    sm.z += __shfl_xor_sync(0xffffffffu, sm.z, o);
                    sm.w += __shfl_xor_sync(0xffffffffu, sm.w, o);
                }
                if (lane == 0) *(float4*)(out + R0 + c4) = sm;
            }
        }
        if (!grid_barrier(bar, bar + 1, gridDim.x, err, &okb, wait_limit)) return;
        // (B) partial sums of the rows (columns) still to solve
        for (int64_t e = threadIdx.x; e < B; e += NTH) xs[e] = __ldcg(out + R0 + e);
        __syncthreads();
        if (!upper) {
            const int64_t nch = (Np - R0 - B) / SV_CH;   // chunks of SV_CH rows below the super-block
            for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
                const int64_t row = R0 + B + ch * SV_CH + warp * 8, i = row / b, ro = row % b;
                float acc[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) acc[k] = 0.f;
                for (int rt = 0; rt < st; ++rt) {
                    const float* Lb = Lt + tri_index(i, t0 + rt) * b * b + ro * b;
                    for (int64_t seg = 0; seg < b; seg += SV_SEG) {
                        float4 xv[2], v[8][2];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int64_t c = seg + 4 * lane + 128 * u;
                            xv[u] = c < b ? *(const float4*)(xs + rt * b + c) : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
#pragma unroll
                        for (int k = 0; k < 8; ++k)
#pragma unroll
                            for (int u = 0; u < 2; ++u) {
                                const int64_t c = seg + 4 * lane + 128 * u;
                                v[k][u] = c < b ? __ldcs((const float4*)(Lb + k * b + c))
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
                            }
#pragma unroll
                        for (int k = 0; k < 8; ++k) acc[k] += dot4(v[k][0], xv[0]) + dot4(v[k][1], xv[1]);
                    }
                }
#pragma unroll
                for (int k = 0; k < 8; ++k)
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
                if (lane < 8) {
                    float a = acc[0];
#pragma unroll
                    for (int k = 1; k < 8; ++k)
                        if (lane == k) a = acc[k];
                    sbuf[row + lane] = __ldcg(sbuf + row + lane) + a;
                }
            }
        } else {
            const int64_t nu = t0 * st;   // units (j, rt): tile (t0 + rt, j), j < t0
            for (int64_t u = blockIdx.x; u < nu; u += gridDim.x) {
                const int64_t j = u / st;
                const int rt = (int)(u % st);
                const float* Lc = Lt + tri_index(t0 + rt, j) * b * b;
                float* sc = sbuf + rt * Np + j * b;
                for (int64_t seg = 0; seg < b; seg += SV_SEG) {
                    float4 a[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
                    for (int64_t r0 = warp * 8; r0 < b; r0 += SV_CH) {   // the warp's rows of each chunk
                        float4 v[8][2];
                        float xr[8];
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            xr[k] = xs[rt * b + r0 + k];
#pragma unroll
                            for (int u2 = 0; u2 < 2; ++u2) {
                                const int64_t c = seg + 4 * lane + 128 * u2;
                                v[k][u2] = c < b ? __ldcs((const float4*)(Lc + (r0 + k) * b + c))
                                                 : make_float4(0.f, 0.f, 0.f, 0.f);
                            }
                        }
#pragma unroll
                        for (int u2 = 0; u2 < 2; ++u2)
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                a[u2].x = fmaf(v[k][u2].x, xr[k], a[u2].x);
                                a[u2].y = fmaf(v[k][u2].y, xr[k], a[u2].y);
                                a[u2].z = fmaf(v[k][u2].z, xr[k], a[u2].z);
                                a[u2].w = fmaf(v[k][u2].w, xr[k], a[u2].w);
                            }
                    }
#pragma unroll
                    for (int u2 = 0; u2 < 2; ++u2) *(float4*)(red + warp * SV_SEG + 4 * lane + 128 * u2) = a[u2];
                    __syncthreads();
                    const int64_t c = seg + threadIdx.x;
                    if (threadIdx.x < SV_SEG && c < b) {
                        float sum = 0.f;
#pragma unroll
                        for (int w = 0; w < 8; ++w) sum += red[w * SV_SEG + threadIdx.x];
                        sc[c] = __ldcg(sc + c) + sum;
                    }
                    __syncthreads();
                }
            }
        }
        if (!grid_barrier(bar, bar + 1, gridDim.x, err, &okb, wait_limit)) return;
    }
}

// ---------------------------------------------------------------- FP64 residual r = y - K x
// One CTA per 64 rows: row part from the lower tiles (j <= i), transposed
// part from the tiles below (j > i).  Every product in FP64; deterministic.
__global__ __launch_bounds__(NTH) void k_sym_resid(const double* K64, const double* x, const double* y,
                                                   double* r, int64_t b, int64_t T)
{
    __shared__ double acc_s[64];
    __shared__ double red[4][64];
    const int64_t R0 = (int64_t)blockIdx.x * 64;
    const int64_t i = R0 / b, ro = R0 % b;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < 64) acc_s[threadIdx.x] = 0.0;
    __syncthreads();
    // row part: sum_{j < i} K_ij[ro + rr][:] . x_j, plus the diagonal tile's
    // lower triangle (t <= ro + rr); the upper triangle of a diagonal tile is
    // never read (it is taken from the transposed lower triangle below)
    for (int rr = warp; rr < 64; rr += 8) {
        double s = 0.0;
        for (int64_t j = 0; j <= i; ++j) {
            const double* row = K64 + tri_index(i, j) * b * b + (ro + rr) * b;
            const double* xj = x + j * b;
            const int64_t tend = (j == i) ? ro + rr + 1 : b;
            for (int64_t t = lane; t < tend; t += 32) s = fma(row[t], xj[t], s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) acc_s[rr] = s;
    }
    // transposed part: sum_{j > i} K_ji[:, ro + c] . x_j and, in the diagonal
    // tile, rows t > ro + c of column ro + c
    const int c = threadIdx.x & 63, q = threadIdx.x >> 6;
    double s = 0.0;
    for (int64_t j = i; j < T; ++j) {
        const double* tile = K64 + tri_index(j, i) * b * b + ro + c;
        const double* xj = x + j * b;
        const int64_t t0 = (j == i) ? ro + c + 1 : 0;
        for (int64_t t = t0 + ((q - t0) % 4 + 4) % 4; t < b; t += 4) s = fma(tile[t * b], xj[t], s);
    }
    red[q][c] = s;
    __syncthreads();
    if (threadIdx.x < 64) {
        int64_t row = R0 + threadIdx.x;
        double kx = acc_s[threadIdx.x] + red[0][threadIdx.x] + red[1][threadIdx.x] + red[2][threadIdx.x] +
                    red[3][threadIdx.x];
        r[row] = y[row] - kx;
    }
}

// out[0] = ||a||^2, out[1] = ||b||^2 (single CTA, deterministic)
__global__ void k_norms2(const double* a, const double* b, int64_t n, double* out)
{
    __shared__ double ra[NTH], rb[NTH];
    double sa = 0.0, sb = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += NTH) {
        sa = fma(a[e], a[e], sa);
        sb = fma(b[e], b[e], sb);
    }
    ra[threadIdx.x] = sa;
    rb[threadIdx.x] = sb;
    __syncthreads();
    for (int o = NTH / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ra[threadIdx.x] += ra[threadIdx.x + o];
            rb[threadIdx.x] += rb[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = ra[0];
        out[1] = rb[0];
    }
}

__global__ void k_d2f(const double* a, float* b, int64_t n)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        b[e] = (float)a[e];
}

__global__ void k_axpy_f(double* x, const float* d, int64_t n)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        x[e] += (double)d[e];
}

// NLML from the refined alpha: 1/2 y^T alpha + sum log L_ii + n/2 log(2 pi).
__global__ void k_nlml_mixed(const double* y, const double* alpha, int64_t n, const double* logdet_part,
                             int64_t T, double* scal)
{
    __shared__ double red[NTH];
    double s = 0.0, ld = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += NTH) s = fma(y[e], alpha[e], s);
    for (int64_t e = threadIdx.x; e < T; e += NTH) ld += logdet_part[e];
    red[threadIdx.x] = 0.5 * s + ld;
    __syncthreads();
    for (int o = NTH / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) scal[0] = red[0] + 0.5 * (double)n * log(2.0 * M_PI);
}

// ---------------------------------------------------------------- mixed prediction
// R32 (ldr = Np) = fp32(K_{Z*,Z}) for a 64 x 64 block, and the FP64 partial
// sums of K_{Z*,Z} alpha over the block's 64 training points (Eq. 3).
__global__ __launch_bounds__(NTH) void k_cross_mixed(const double* Xs, int64_t m, const double* X, int64_t n,
                                                     int64_t d, const double* alpha, const GpHyperDev* hyp,
                                                     float* R32, int64_t ldr, double* mpart, int64_t ldp,
                                                     double* R64)
{
    __shared__ double sm[2 * 64 * 17];
    const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
    double r2[4][4];
    dist_block(r2, Xs, m0, m, X, n0, n, d, sm);
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t gm = m0 + ty + 16 * a;
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t gn = n0 + tx + 16 * c;
            double kv = (gm < m && gn < n) ? kval(r2[a][c], hyp) : 0.0;
            R32[gm * ldr + gn] = (float)kv;
            if (R64) R64[gm * ldr + gn] = kv;
            if (gn < n) s = fma(kv, alpha[gn], s);
        }
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (tx == 0) mpart[(int64_t)blockIdx.x * ldp + gm] = s;
    }
}

// Planes of the column block R32[:, j*b .. (j+1)*b) into RP ([3][ldm][b]).
// Planes of columns col0 .. col0 + width - 1 of R32 (rows x ldr) into RP
// (three planes of rows x ldp).
__global__ void k_split_cols(const float* R32, int64_t ldr, int64_t col0, int64_t width, int64_t ldp, int64_t rows,
                             __nv_bfloat16* RP)
{
    const int64_t total = rows * width, ps = rows * ldp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / width, c = e % width;
        __nv_bfloat16 hi, mid, lo;
        split3(R32[r * ldr + col0 + c], hi, mid, lo);
        RP[r * ldp + c] = hi;
        RP[ps + r * ldp + c] = mid;
        RP[2 * ps + r * ldp + c] = lo;
    }
}

// mean = sum of the mean partials, var = k** - sum of the variance partials.
__global__ void k_mixed_finish(const double* mpart, int64_t nmp, const double* vpart, int64_t nvp, int64_t ldm,
                               int64_t m, const GpHyperDev* hyp, int noisy, double* mean, double* var)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    double sm = 0.0, sv = 0.0;
    for (int64_t q = 0; q < nmp; ++q) sm += mpart[q * ldm + c];
    for (int64_t q = 0; q < nvp; ++q) sv += vpart[q * ldm + c];
    if (mean) mean[c] = sm;
    if (var) var[c] = hyp->nu + (noisy ? hyp->s2 : 0.0) - sv;
}

// ---------------------------------------------------------------- mixed inverse for the gradient
// With X = L^{-1} (lower tiles X_ij), the tiles Z_ij = X_ij^T satisfy
//   Z_jj = Linv_jj^T,
//   U_ij = sum_{t=j}^{i-1} Z_tj L_it^T,   Z_ij = -U_ij Linv_ii^T   (i > j),
// and K^{-1}_ij = sum_{t >= i} Z_ti Z_tj^T, all products in NT form.

// ZP_tt = planes of Linv_tt^T, for every t.
__global__ void k_zdiag(const float* Linv32, __nv_bfloat16* ZP, int64_t b)
{
    const int64_t bb = b * b, t = blockIdx.y;
    const float* src = Linv32 + t * bb;
    __nv_bfloat16* dst = ZP + tri_index(t, t) * 3 * bb;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < bb;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = e / b, c = e % b;
        __nv_bfloat16 hi, mid, lo;
        split3(src[c * b + a], hi, mid, lo);
        dst[e] = hi;
        dst[bb + e] = mid;
        dst[2 * bb + e] = lo;
    }
}

// Planes of U32 tiles (t, j), j < t, into PA slots j.
__global__ void k_split_row(const float* U32, __nv_bfloat16* PA, int64_t b, int64_t t)
{
    const int64_t bb = b * b, j = blockIdx.y;
    const float* src = U32 + tri_index(t, j) * bb;
    __nv_bfloat16* dst = PA + j * 3 * bb;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < bb;
         e += (int64_t)gridDim.x * blockDim.x) {
        __nv_bfloat16 hi, mid, lo;
        split3(src[e], hi, mid, lo);
        dst[e] = hi;
        dst[bb + e] = mid;
        dst[2 * bb + e] = lo;
    }
}

// ---------------------------------------------------------------- variance correction
// With any x0 and r0 = k* - K x0,
//   k*^T K^{-1} k* = k*^T x0 + x0^T r0 + r0^T K^{-1} r0
// holds exactly.  x0 is the mixed-factor solution (L~ L~^T)^{-1} k* rounded to
// 14 bits per test point (x~0, k_yslices), and the last term is taken with the
// mixed factor, ||L~^{-1} r0||^2 (its error is third order).  Only K x~0 must
// be accurate to FP64 level; it is formed from exactly-accumulated BF16 digit
// slices (Ozaki et al. 2012): each row of x~0^T and all of K are scaled by a
// power of two and split into 7-bit signed integer digits (|d| <= 128, exact
// in BF16), every digit product is exact (|d e| <= 2^14), sums of at most 1024
// of them are exact in FP32 (<= 2^24), and the partial sums are carried in
// double-FP32.

constexpr int OZ_S = GP_OZ_SLICES;   // digit slices of K
constexpr int OZ_B = GP_OZ_BITS;     // bits per digit

constexpr int OZ_YS = GP_OZ_YSLICES;   // digit slices of x~0

// Rounds each row of Y (R32, ldm x Np) to OZ_YS digits and splits it:
// mu[row] = power of two >= max |Y|, q = rint(Y 2^(OZ_B OZ_YS) / mu)
// (|q| <= 2^(OZ_B OZ_YS)), YS[s][row][col] = s-th digit of q, and Y is
// overwritten by x~0 = q mu 2^{-OZ_B OZ_YS}, exact in FP32.  The variance
// correction then uses this x~0 in every term, which makes it exact for x~0
// whatever the rounding (the identity behind it holds for any x0); only
// r0 = k* - K x~0 grows, to about 2^{-14} of k*, and its quadratic term
// stays far below the FP64 target.  A row whose rounded values would fall
// below the FP32 grid (max |Y| < 2^-135) is taken as zero.  One CTA per row.
__global__ void k_yslices(float* Y, int64_t Np, __nv_bfloat16* YS, int64_t ps, double* mu)
{
    __shared__ float red[NTH];
    const int64_t row = blockIdx.x;
    float* y = Y + row * Np;
    float mx = 0.f;
    for (int64_t c = threadIdx.x; c < Np; c += NTH) mx = fmaxf(mx, fabsf(y[c]));
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int o = NTH / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    const double m = red[0] > 0.f ? pow2_ceil((double)red[0]) : 1.0;
    if (threadIdx.x == 0) mu[row] = m;
    const int ex = pow2_exp(m);
    const int sc = OZ_B * OZ_YS - ex;   // y / m 2^(OZ_B OZ_YS) = y 2^sc
    const bool tiny = ex - OZ_B * OZ_YS < -149;
    for (int64_t c = threadIdx.x; c < Np; c += NTH) {
        const long long q = tiny ? 0ll : rint_scaled(y[c], sc);
        __nv_bfloat16 d[OZ_YS];
        oz_digits<OZ_YS>(q, d);
#pragma unroll
        for (int s = 0; s < OZ_YS; ++s) YS[s * ps + row * Np + c] = d[s];
        y[c] = ldexpf((float)q, -sc);
    }
}

// Rows of Z - c (row-major, d columns, c a row of d values; rows at or
// beyond `valid` read as zero) as digit slices for the tensor-core squared
// distances (kernels_dist.cu).  Distances do not change under the shift, and
// with the origin c inside the data the rows stay short, so the cancellation
// in |z_i|^2 + |z_j|^2 - 2 z_i . z_j stays small.  With z the shifted row:
// mu[row] = power of two >= max_k |z_k|, q = rint(z 2^(OZ_B OZ_S) / mu),
// ZS[s][row][k] = s-th balanced digit of q (zero for d <= k < dp), and
// nrm[row] = sum_k zhat_k^2 in FP64 for the quantised row zhat = q mu 2^-42,
// so that |zhat_i|^2 + |zhat_j|^2 - 2 zhat_i . zhat_j is the squared distance
// of the quantised rows.  One warp per row, eight rows per CTA.
__global__ void k_zslices(const double* Z, const double* c, int64_t rows, int64_t valid, int64_t d, int64_t dp,
                          __nv_bfloat16* ZS, int64_t ps, double* mu, double* nrm)
{
    const int64_t row = (int64_t)blockIdx.x * (NTH / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const bool live = row < valid;
    const double* z = Z + row * d;
    double mx = 0.0;
    if (live)
        for (int64_t k = lane; k < d; k += 32) mx = fmax(mx, fabs(z[k] - c[k]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const double m = mx > 0.0 ? pow2_ceil(mx) : 1.0;
    const int sc = OZ_B * OZ_S - pow2_exp(m);   // z / m 2^(OZ_B OZ_S) = z 2^sc
    double acc = 0.0;
    for (int64_t k = lane; k < dp; k += 32) {
        const long long q = (live && k < d) ? rint_scaled(z[k] - c[k], sc) : 0ll;
        __nv_bfloat16 dg[OZ_S];
        oz_digits<OZ_S>(q, dg);
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) ZS[s * ps + row * dp + k] = dg[s];
        const double zh = ldexp((double)q, -sc);   // exact: |q| <= 2^42
        acc = fma(zh, zh, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        mu[row] = m;
        nrm[row] = acc;
    }
}

void zslices(gp_t h, const double* Z, const double* center, int64_t rows, int64_t valid, __nv_bfloat16* ZS,
             double* mu, double* nrm, int phase)
{
    GPK_LAUNCH(h, phase, k_zslices, (unsigned)((rows + NTH / 32 - 1) / (NTH / 32)), NTH, 0, Z, center, rows, valid,
               h->d, h->dp, ZS, rows * h->dp, mu, nrm);
}

// Digits of the full symmetric K (from the lower FP64 tiles) scaled by
// kappa = power of two >= max(nu + sigma^2, 1).  One CTA per 64 x 64 block of
// K: the block at (max, min) of its block indices is read row-wise from the
// lower tiles into shared memory and written out directly or transposed, so
// both the reads and the digit writes are coalesced.
__global__ void k_kslices(const double* K64, int64_t b, int64_t Np, const GpHyperDev* hyp, __nv_bfloat16* KS,
                          int64_t ps, double* kappa_out)
{
    __shared__ double tile[64][65];
    const double kappa = pow2_ceil(fmax(hyp->nu + hyp->s2, 1.0));
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *kappa_out = kappa;
    const int sc = OZ_B * OZ_S - pow2_exp(kappa);   // v / kappa 2^(OZ_B OZ_S) = v 2^sc
    const int64_t R0 = (int64_t)blockIdx.y * 64, C0 = (int64_t)blockIdx.x * 64;
    const int64_t LR = R0 >= C0 ? R0 : C0, LC = R0 >= C0 ? C0 : R0;   // lower block
    const double* src = K64 + tri_index(LR / b, LC / b) * b * b + (LR % b) * b + (LC % b);
    for (int e = threadIdx.x; e < 64 * 64; e += NTH) {
        const int r = e >> 6, c = e & 63;
        tile[r][c] = src[(int64_t)r * b + c];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * 64; e += NTH) {
        const int r = e >> 6, c = e & 63;
        // element (R0 + r, C0 + c) of the symmetric K, from the lower triangle
        double v;
        if (R0 > C0) v = tile[r][c];
        else if (R0 < C0) v = tile[c][r];
        else v = (c <= r) ? tile[r][c] : tile[c][r];
        __nv_bfloat16 d[OZ_S];
        oz_digits<OZ_S>(rint_scaled(v, sc), d);
        const int64_t o = (R0 + r) * Np + C0 + c;
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) KS[s * ps + o] = d[s];
    }
}

// var = k** - (sum k*^T x0 + sum x0^T r0 + ||L~^{-1} r0||^2), mean untouched.
__global__ void k_var_finish(const double* qpart, int64_t nqb, const double* vpart2, int64_t nvp, int64_t ldm,
                             int64_t m, const GpHyperDev* hyp, int noisy, double* var)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    double s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int64_t q = 0; q < nqb; ++q) {
        s1 += qpart[q * ldm + c];
        s2 += qpart[(nqb + q) * ldm + c];
    }
    for (int64_t q = 0; q < nvp; ++q) s3 += vpart2[q * ldm + c];
    var[c] = hyp->nu + (noisy ? hyp->s2 : 0.0) - (s1 + s2 + s3);
}

__global__ void k_factor_dense32(const float* Lt, int64_t b, int64_t n, double* out)
{
    int64_t total = n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e / n, c = e % n;
        out[e] = (c <= r) ? (double)Lt[tri_index(r / b, c / b) * b * b + (r % b) * b + (c % b)] : 0.0;
    }
}

// ================================================================ host launchers
static int grid_for(int64_t work, int per = NTH)
{
    int64_t g = (work + per - 1) / per;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

// Operand planes and steps of the three multi-RHS sweeps of a prediction.  W =
// K_{Z*,Z} L~^{-T} feeds x0 and the full covariance and keeps all three
// planes (FP32 accuracy).  The backward sweep x0^T = W L~^{-1} and the forward
// sweep of r0 take the three plane products of order <= 2^-8 (about 2^-16
// relative): x0 is rounded to 14 bits afterwards and the exact correction
// holds for any x0, and ||L~^{-1} r0||^2 is a small second-order term.
// Measured at N = 32768, M = 8192 against the emulated FP64 path: variance
// error 4.2e-11 with three planes everywhere, 3.4e-11 with these choices;
// two planes on W as well give 1.2e-9 (worst element 5e-8).  The backward
// and r0 sweeps step over super-blocks with their inverses X_I (4.4e-11);
// W takes the tile-by-tile steps: through X_I, whose off-diagonal tiles are
// FP32 products, its variance error rose to 9.5e-10 (worst 3e-8).
constexpr int SWEEP_PLANES_W = 3;
constexpr int SWEEP_PLANES_B = 2;
constexpr int SWEEP_PLANES_R = 2;

// The factorisation and the multi-RHS sweeps update their trailing FP32
// matrix once per block of SWEEP_BLOCK tile columns (one k-segment per
// column), so it is read and written T / SWEEP_BLOCK times, not T.
constexpr int SWEEP_BLOCK = 4;

// Right-looking, in super-panels of SWEEP_BLOCK tile columns: each column k
// of a super-panel is factored (diagonal tile, panel) and applied only to the
// super-panel's later columns; then one update with a k-segment per column
// applies the whole super-panel to the trailing triangle.
static void build_sbinv(gp_t h);

bool factor_mixed(gp_t h)
{
    const int T = (int)h->T;
    const int64_t b = h->b, bb = b * b;
    for (int K0 = 0; K0 < T; K0 += SWEEP_BLOCK) {
        const int e = K0 + SWEEP_BLOCK < T ? K0 + SWEEP_BLOCK : T;
        for (int k = K0; k < e; ++k) {
            // diagonal tile: FP32 factor and inverse on one cluster of eight CTAs
            if (!potrf_diag_cl32(h, h->A32 + tri_index(k, k) * bb, h->Linv32 + k * bb, h->LinvP + k * 3 * bb, b,
                                 (int64_t)k * b, h->logdet_part + k))
                return false;
            if (k + 1 < T) {
                const unsigned tt = (unsigned)(T - k - 1);
                GPK_LAUNCH(h, GP_PH_TRSM, k_split_panel, dim3((unsigned)grid_for(bb) / 4 + 1, tt), NTH, 0,
                           (const float*)h->A32, h->PA, b, (int64_t)k);
                if (!tg_panel(h, k)) return false;
                if (k + 1 < e && !tg_update(h, k, 1, k + 1, e - k - 1)) return false;
            }
        }
        if (e < T && !tg_update(h, K0, e - K0, e, T - e)) return false;
    }
    build_sbinv(h);
    return true;
}


// Super-block inverses X_I of the mixed factor (end of factor_mixed): the
// tile inverses on the diagonal, then the recursive doubling, two launches
// (T, then X) per group width.
static void build_sbinv(gp_t h)
{
    const int64_t b = h->b, T = h->T, TS = (T + SB_TILES - 1) / SB_TILES, nsub = b / 64;
    GPK_LAUNCH(h, GP_PH_POTRF, k_sbinv_diag, dim3((unsigned)grid_for(b * b) / 8 + 1, (unsigned)T), NTH, 0,
               (const float*)h->Linv32, h->Xsb, b, T);
    for (int w = 1; w < SB_TILES; w *= 2) {
        int np = 0;   // (i, j) pairs of a full super-block at width w
        for (int a0 = 0; a0 + w < SB_TILES; a0 += 2 * w)
            np += ((a0 + 2 * w < SB_TILES ? a0 + 2 * w : SB_TILES) - a0 - w) * w;
        for (int phase = 1; phase <= 2; ++phase)
            GPK_LAUNCH(h, GP_PH_POTRF, k_sbinv_level, dim3((unsigned)(nsub * nsub), (unsigned)np, (unsigned)TS), NTH,
                       0, (const float*)h->A32, h->Xsb, b, T, w, phase);
    }
    GPK_LAUNCH(h, GP_PH_POTRF, k_split_sbx, grid_for(TS * SB_TILES * b * SB_TILES * b), NTH, 0,
               (const float*)h->Xsb, b, T, h->XsbP);
}

// out32 = L~^{-1} in32 (lower) or L~^{-T} in32 (upper), FP32 throughout.
static void solve32(gp_t h, const float* in32, float* out32, bool upper)
{
    static int grid_dev = -1, grid_blocks = 0;
    static int64_t grid_b = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t dyn = 2 * (size_t)SB_TILES * h->b * sizeof(float);
    if (grid_dev != dev || grid_b != h->b) {   // every CTA resident at once: the blocks wait on one another
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solve32p, NTH, dyn);
        grid_blocks = sms * (per < 2 ? per : 2);
        grid_dev = dev;
        grid_b = h->b;
    }
    int64_t bb = h->b, TT = h->T;
    int up = upper ? 1 : 0;
    const float* Lt = h->A32;
    const float* Xs = h->Xsb;
    float* sbuf = h->w32;
    unsigned* bar = (unsigned*)h->solve_flags;
    int* err = tc_error_dev();
    long long limit = h->solve_wait_cycles;
    int stall = h->solve_stall ? 1 : 0;
    void* args[] = {(void*)&Lt, (void*)&Xs, (void*)&bb, (void*)&TT, (void*)&in32, (void*)&out32, (void*)&sbuf,
                    (void*)&up, (void*)&bar, (void*)&err, (void*)&limit, (void*)&stall};
    cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), h->st);   // fresh barrier words, whatever a failed solve left
    const bool p_ = h->prof_on && prof_begin(h, GP_PH_SOLVE);
    // a failed launch (including a grid of zero) leaves its error for the caller's check of the last launch error
    cudaLaunchCooperativeKernel((const void*)k_solve32p, dim3((unsigned)grid_blocks), dim3(NTH), args, dyn, h->st);
    h->launches++;
    if (p_) prof_end(h);
    h->tc_pending = true;
}

// One correction sweep: d = L~^{-T} L~^{-1} r32 (FP32), x += d.
static void correct(gp_t h, double* x)
{
    solve32(h, h->r32, h->t32, false);
    solve32(h, h->t32, h->r32, true);
    GPK_LAUNCH(h, GP_PH_REFINE, k_axpy_f, grid_for(h->Np), NTH, 0, x, (const float*)h->r32, h->Np);
}

void residual64(gp_t h, const double* x, const double* y, double* r)
{
    GPK_LAUNCH(h, GP_PH_REFINE, k_sym_resid, (unsigned)(h->Np / 64), NTH, 0, (const double*)h->L, x, y, r,
               h->b, h->T);
}

void refine_start(gp_t h, const double* rhs, double* x)
{
    // x0 = L~^{-T} L~^{-1} rhs
    cudaMemsetAsync(x, 0, h->Np * sizeof(double), h->st);
    GPK_LAUNCH(h, GP_PH_REFINE, k_d2f, grid_for(h->Np), NTH, 0, rhs, h->r32, h->Np);
    correct(h, x);
}

void refine_residual(gp_t h, const double* rhs, const double* x, double* r, double* norms)
{
    residual64(h, x, rhs, r);
    GPK_LAUNCH(h, GP_PH_REFINE, k_norms2, 1, NTH, 0, (const double*)r, rhs, h->Np, norms);
}

void refine_correct(gp_t h, const double* r, double* x)
{
    GPK_LAUNCH(h, GP_PH_REFINE, k_d2f, grid_for(h->Np), NTH, 0, r, h->r32, h->Np);
    correct(h, x);
}

void nlml_mixed(gp_t h)
{
    GPK_LAUNCH(h, GP_PH_REDUCE, k_nlml_mixed, 1, NTH, 0, (const double*)h->y, (const double*)h->alpha, h->n,
               (const double*)h->logdet_part, h->T, h->scal);
}

// Forward multi-RHS solve W = R L~^{-T} in place over R (ldm x Np, FP32): W
// planes into WP, FP32 W over R, FP64 row sums of W^2 into vpart.  Tile by
// tile (sb false): W_j = R_j Linv_jj^T, then the later columns of the same
// block of SWEEP_BLOCK tiles, then one update of every later tile per block.
// By super-blocks (sb true): W_I = R_I X_I^T, then R_i -= sum over the
// super-block's tiles j of W_j L_ij^T for every later tile i.  Either way R
// is read and written once per block of four tile columns.
static bool forward_w(gp_t h, float* R, int64_t ldm, double* vpart, int phase, int planes, bool sb)
{
    const int T = (int)h->T;
    const int64_t b = h->b, Np = h->Np, SBb = SB_TILES * b;
    if (!sb) {
        for (int J = 0; J < T; J += SWEEP_BLOCK) {
            const int e = J + SWEEP_BLOCK < T ? J + SWEEP_BLOCK : T;
            for (int j = J; j < e; ++j) {
                GPK_LAUNCH(h, phase, k_split_cols, grid_for(ldm * b), NTH, 0, (const float*)R, Np, (int64_t)j * b, b, b,
                           ldm, h->RP);
                if (!tg_diag_w(h, phase, R, ldm, vpart, j, planes)) return false;
                if (j + 1 < e && !tg_upd_w(h, phase, R, ldm, j, 1, j + 1, e - j - 1, planes)) return false;
            }
            if (e < T && !tg_upd_w(h, phase, R, ldm, J, e - J, e, T - e, planes)) return false;
        }
        return true;
    }
    for (int t0 = 0; t0 < T; t0 += SB_TILES) {
        const int st = T - t0 < SB_TILES ? T - t0 : SB_TILES;
        GPK_LAUNCH(h, phase, k_split_cols, grid_for(ldm * st * b), NTH, 0, (const float*)R, Np, (int64_t)t0 * b,
                   (int64_t)st * b, SBb, ldm, h->RP);
        if (!tg_diag_w_sb(h, phase, R, ldm, vpart, t0 / SB_TILES, planes)) return false;
        if (t0 + st < T && !tg_upd_w(h, phase, R, ldm, t0, st, t0 + st, T - t0 - st, planes)) return false;
    }
    return true;
}

bool predict_mixed(gp_t h, int64_t m, int64_t ldm, bool want_var, bool want_cov)
{
    const int64_t Np = h->Np;
    const int64_t nmp = Np / 64, nvp = Np / 64;   // variance partials: one slot per 64 columns
    if (h->tc_dist) {   // squared distances on the tensor cores, origin at the first training row
        zslices(h, h->Xs, h->X, ldm, m, h->ZSS, h->zs_mu, h->zs_nrm, GP_PH_CROSS);
        if (!dist_cross_tc(h, m, ldm)) return false;
    } else {
        GPK_LAUNCH(h, GP_PH_CROSS, k_cross_mixed, dim3((unsigned)(Np / 64), (unsigned)(ldm / 64)), NTH, 0,
                   (const double*)h->Xs, m, (const double*)h->X, h->n, h->d, (const double*)h->alpha,
                   (const GpHyperDev*)h->hyp, h->R32, Np, h->mpart, ldm, h->R64);
    }
    if ((want_var || want_cov) &&
        !forward_w(h, h->R32, ldm, h->vpart, GP_PH_VSOLVE, SWEEP_PLANES_W, false))
        return false;
    GPK_LAUNCH(h, GP_PH_REDUCE, k_mixed_finish, (unsigned)((m + 255) / 256), 256, 0, (const double*)h->mpart,
               nmp, (const double*)h->vpart, want_var ? nvp : (int64_t)0, ldm, m, (const GpHyperDev*)h->hyp,
               h->opt.noisy_test_var, h->outm, want_var ? h->outv : (double*)nullptr);
    return true;
}

// Corrected variances into h->outv (needs predict_mixed's forward solve: R32
// holds W, R64 holds K_{Z*,Z}).  Overwrites the W planes (run after full_cov_mixed).
bool var_correction_mixed(gp_t h, int64_t m, int64_t ldm)
{
    const int64_t T = h->T, b = h->b, Np = h->Np;
    // x0^T = W L~^{-1}: backward sweep over super-blocks, in place over R32:
    // Y_I = S_I X_I, then S_j -= sum over the super-block's tiles i of Y_i L_ij
    // for every earlier tile j; Y planes go to the W plane buffer
    const int64_t SBb = SB_TILES * b, TS = (T + SB_TILES - 1) / SB_TILES;
    for (int64_t I = TS - 1; I >= 0; --I) {
        const int t0 = (int)(I * SB_TILES), st = (int)(T - t0 < SB_TILES ? T - t0 : SB_TILES);
        GPK_LAUNCH(h, GP_PH_BSOLVE, k_split_cols, grid_for(ldm * st * b), NTH, 0, (const float*)h->R32, Np,
                   (int64_t)t0 * b, (int64_t)st * b, SBb, ldm, h->RP);
        if (!tg_bdiag_sb(h, ldm, I, SWEEP_PLANES_B)) return false;
        if (t0 > 0 && !tg_bupd(h, ldm, t0, st, 0, t0, SWEEP_PLANES_B)) return false;
    }
    GPK_LAUNCH(h, GP_PH_SLICES, k_yslices, (unsigned)ldm, NTH, 0, h->R32, Np, h->YS, ldm * Np, h->mu);
    if (!h->ks_valid) {
        GPK_LAUNCH(h, GP_PH_SLICES, k_kslices, dim3((unsigned)(Np / 64), (unsigned)(Np / 64)), NTH, 0, (const double*)h->L, b, Np,
                   (const GpHyperDev*)h->hyp, h->KS, Np * Np, h->kappa);
        h->ks_valid = true;
    }
    if (!ozaki_tc(h, m, ldm)) return false;
    if (!forward_w(h, h->Rr32, ldm, h->vpart2, GP_PH_RSOLVE, SWEEP_PLANES_R, true)) return false;
    GPK_LAUNCH(h, GP_PH_REDUCE, k_var_finish, (unsigned)((m + 255) / 256), 256, 0, (const double*)h->qpart, Np / 64,
               (const double*)h->vpart2, Np / 64, ldm, m, (const GpHyperDev*)h->hyp, h->opt.noisy_test_var,
               h->outv);
    return true;
}

bool full_cov_mixed(gp_t h, int64_t m, int64_t ldm, double* cov)
{
    if (h->tc_dist) {   // test digits again, origin at the first test row (test-test distances only)
        zslices(h, h->Xs, h->Xs, ldm, m, h->ZSS, h->zs_mu, h->zs_nrm, GP_PH_COV);
        if (!dist_prior_tc(h, m, ldm, cov)) return false;
    } else {
        assemble_test_prior(h, m, cov);
    }
    return tg_syrk_cov(h, m, ldm, cov);
}

bool inverse_mixed(gp_t h)
{
    const int64_t T = h->T, b = h->b, bb = b * b;
    GPK_LAUNCH(h, GP_PH_TRTRI, k_zdiag, dim3((unsigned)grid_for(bb) / 4 + 1, (unsigned)T), NTH, 0,
               (const float*)h->Linv32, h->ZP, b);
    // blocks of SWEEP_BLOCK steps t: each step's accumulation reaches only the
    // block's rows; one multi-segment accumulation then applies the block to
    // every later row, so U32 is read and written once per block
    const int TT = (int)T;
    for (int T0 = 0; T0 < TT; T0 += SWEEP_BLOCK) {
        const int e = T0 + SWEEP_BLOCK < TT ? T0 + SWEEP_BLOCK : TT;
        for (int t = T0; t < e; ++t) {
            if (t > 0) {
                GPK_LAUNCH(h, GP_PH_TRTRI, k_split_row, dim3((unsigned)grid_for(bb) / 4 + 1, (unsigned)t), NTH, 0,
                           (const float*)h->U32, h->PA, b, (int64_t)t);
                if (!tg_trtri_fin(h, t)) return false;
            }
            if (t + 1 < e && !tg_trtri_acc(h, t, t + 1, t + 1, e - t - 1, t + 1)) return false;
        }
        if (e < TT && !tg_trtri_acc(h, T0, e, e, TT - e, e)) return false;
    }
    return tg_lauum(h);
}

void copy_factor_dense_mixed(gp_t h, double* out)
{
    GPK_LAUNCH(h, GP_PH_OTHER, k_factor_dense32, grid_for(h->n * h->n), NTH, 0, (const float*)h->A32, h->b,
               h->n, out);
}

}  // namespace gpk
