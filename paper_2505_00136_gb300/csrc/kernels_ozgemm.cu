// FP64-accurate tile products on the BF16 tensor cores (the Ozaki scheme:
// Ozaki, Ogita, Oishi & Rump 2012), for the GP_FP64_OZAKI precision.
//
// C = (C or 0) +- A B^T with A (rows x k) and B (cols x k) given as digit slices: every
// row r of an operand is scaled by a power of two mu_r >= max |row| and
// rounded to 49 bits, q = rint(v 2^49 / mu_r), and q is split into seven
// balanced 7-bit digits (|d| <= 2^7, exact in BF16) stored slice-major,
// k contiguous (k_rowslices).  Then
//   (A B^T)_ij ~ mu_i mu_j sum over digit pairs (s, u), s + u <= 8, of
//                2^{-7(s+u)} (A_s B_u^T)_ij,
// every digit product exact (<= 2^14) and every sum of one level l = s + u
// exact in an FP32 TMEM accumulator over chunks of 256 k (at most seven
// pairs, one of them with a leading digit: 7 x 256 x 2^13 <= 2^24).  Chunk
// sums are scaled by 2^{-7l} and added into double-FP32 running sums held in
// registers (about 48 bits); the epilogue forms the FP64 product and adds it
// to (or subtracts it from, or stores it over) the FP64 destination.  The rounding of the operands to
// 49 bits bounds the error of one product by about 2^-49 mu_i mu_j k: FP64
// level for the factorisation and solves of this path.
//
// Operand reuse: the levels run in four groups, (2, 3), (4, 5), (6, 7) and
// (8); a 32-k stage of a group holds the A and B slices that the group's
// pairs use (up to 2 x 7 slices of 128 x 32, 8 KB each, two stages), and all
// of the group's 3 to 11 pair products are issued from it.  Two pairs of
// 128-column level accumulators alternate between successive group chunks
// while the epilogue warps flush the previous one.
//
// Roles (320 threads, one CTA per 128 x 128 output block of an Op): warp 0
// TMA loads, warp 1 MMA issue, warps 2-9 flush and epilogue, with bounded
// waits (tc_common.cuh) that end in GP_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "digits.cuh"
#include "gp_internal.cuh"
#include "se_common.cuh"
#include "tc_common.cuh"

namespace gpk {
namespace {

constexpr int OG_S = GP_OG_SLICES;                        // digit slices per operand (7)
constexpr int OG_KS = 32;                                 // k per stage
constexpr int OG_SLOT = 128 * OG_KS * 2;                  // one 128 x 32 BF16 tile (8 KB)
constexpr int OG_STAGE_BYTES = 2 * OG_S * OG_SLOT;        // A slices 1..7, B slices 1..7
constexpr int OG_STAGES = 2;
constexpr int OG_CHUNK = 256;                             // k per exact chunk
constexpr int OG_SPC = OG_CHUNK / OG_KS;                  // stages per chunk
constexpr int OG_GROUPS = 4;
constexpr int OG_THREADS = 320;
constexpr int OG_EPI_WARPS = 8;
constexpr int OG_BAR_OFF = OG_STAGES * OG_STAGE_BYTES;
constexpr int OG_SMEM = 1024 + OG_BAR_OFF + 256;
constexpr uint32_t OG_IDESC = tc::idesc_bf16(128, 128);
static_assert(OG_S == 7, "the level groups below are laid out for seven slices and levels 2..8");
static_assert(OG_SMEM <= 227 * 1024, "shared memory");
static_assert(7 * OG_CHUNK * (1 << 13) <= (1 << 24), "a level's chunk sum must stay exact in FP32");

// Levels of group g: (2, 3), (4, 5), (6, 7), (8).
__host__ __device__ constexpr int og_l0(int g) { return 2 + 2 * g; }
__host__ __device__ constexpr int og_nl(int g) { return g == 3 ? 1 : 2; }
// Pairs (s, l - s) of level l: s = og_smin(l) .. og_smax(l).
__host__ __device__ constexpr int og_smin(int l) { return l - OG_S > 1 ? l - OG_S : 1; }
__host__ __device__ constexpr int og_smax(int l) { return l - 1 < OG_S ? l - 1 : OG_S; }
// Slices 1 .. og_top(g) of each operand feed group g.
__host__ __device__ constexpr int og_top(int g) { return og_smax(og_l0(g) + og_nl(g) - 1); }

__device__ __forceinline__ bool og_drain(uint32_t mbar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!tc::mbar_try(mbar, parity))
        if (clock64() - t0 > tc::WAIT_CYCLES) return false;
    return true;
}

__device__ __forceinline__ void og_two_sum(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bv = s - hi;
    const float er = (hi - (s - bv)) + (x - bv);
    hi = s;
    lo += er;
}

// Where one output block reads its operands and writes its result.
struct OgUnit {
    int a_row, b_row;      // first row of the block in the A / B slice arrays (slice 1)
    int k0, k1;            // k range (multiple of 32)
    double* dst;           // first element of the 128 x 128 destination block
    int64_t ld;            // its row stride
    const double* muA;     // row scales of the block's 128 A rows
    const double* muB;     // row scales of its 128 B rows
    int rows, cols;        // valid rows / columns of the block (others are not written)
    double sign;           // dst = (overwrite ? 0 : dst) + sign * A B^T
    bool overwrite;
};

template <class Op>
__global__ __launch_bounds__(OG_THREADS, 1) void k_ozgemm(const __grid_constant__ CUtensorMap mapA,
                                                        const __grid_constant__ CUtensorMap mapB, const Op op,
                                                        int* err)
{
    OgUnit un;
    if (!op.unit((int)blockIdx.x, un)) return;

    extern __shared__ unsigned char dyn[];
    unsigned char* base = dyn + ((1024 - (tc::su32(dyn) & 1023)) & 1023);
    const uint32_t sbase = tc::su32(base);
    const uint32_t bar = sbase + OG_BAR_OFF;   // full[S], empty[S], accf[2], acce[2], drain
    auto full = [&](int s) { return bar + 8 * s; };
    auto empty = [&](int s) { return bar + 8 * (OG_STAGES + s); };
    auto accf = [&](int a) { return bar + 8 * (2 * OG_STAGES + a); };
    auto acce = [&](int a) { return bar + 8 * (2 * OG_STAGES + 2 + a); };
    const uint32_t drain = bar + 8 * (2 * OG_STAGES + 4);
    uint32_t* tmem_slot = (uint32_t*)(base + OG_BAR_OFF + 8 * (2 * OG_STAGES + 5));
    volatile int* abort = (volatile int*)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < OG_STAGES; ++s) {
            tc::mbar_init(full(s), 1);
            tc::mbar_init(empty(s), 1);
        }
        tc::mbar_init(accf(0), 1);
        tc::mbar_init(accf(1), 1);
        tc::mbar_init(acce(0), OG_EPI_WARPS);
        tc::mbar_init(acce(1), OG_EPI_WARPS);
        tc::mbar_init(drain, 1);
        *abort = 0;
        tc::mbar_init_fence();
    }
    if (warp == 1) tc::tmem_alloc(tc::su32(tmem_slot), 512);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    const int ks0 = un.k0 / OG_KS, ks1 = un.k1 / OG_KS;       // 32-k stages of the unit
    const int nch = (ks1 - ks0 + OG_SPC - 1) / OG_SPC;         // exact chunks

    if (warp == 0) {
        if (lane == 0) {
            int gs = 0;
            bool ok = true;
            const uint64_t pol = tc::policy_evict_last();
            for (int c = 0; c < nch && ok; ++c)
                for (int g = 0; g < OG_GROUPS && ok; ++g) {
                    const int top = og_top(g);
                    for (int k = ks0 + c * OG_SPC; k < min(ks1, ks0 + (c + 1) * OG_SPC); ++k, ++gs) {
                        const int st = gs % OG_STAGES, use = gs / OG_STAGES;
                        if (use > 0 && !tc::mbar_wait(empty(st), (uint32_t)((use - 1) & 1), abort, err)) {
                            ok = false;
                            break;
                        }
                        const uint32_t dst = sbase + st * OG_STAGE_BYTES;
                        tc::mbar_expect_tx(full(st), (uint32_t)(2 * top * OG_SLOT));
                        for (int s = 0; s < top; ++s) {
                            tc::tma_load_2d_hint(dst + s * OG_SLOT, &mapA, k * OG_KS, s * op.a_ps + un.a_row, full(st),
                                                 pol);
                            tc::tma_load_2d_hint(dst + (OG_S + s) * OG_SLOT, &mapB, k * OG_KS, s * op.b_ps + un.b_row,
                                                 full(st), pol);
                        }
                    }
                }
            if (!ok)   // let the copies in flight land before the CTA exits
                for (int q = gs - 1; q >= 0 && q >= gs - OG_STAGES; --q)
                    og_drain(full(q % OG_STAGES), (uint32_t)((q / OG_STAGES) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int gs = 0, cu = 0;
            bool ok = true;
            constexpr uint64_t slot16 = (uint64_t)(OG_SLOT >> 4);
            for (int c = 0; c < nch && ok; ++c)
                for (int g = 0; g < OG_GROUPS && ok; ++g, ++cu) {
                    const int a = cu & 1;
                    if (cu >= 2 && !tc::mbar_wait(acce(a), (uint32_t)(((cu >> 1) - 1) & 1), abort, err)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const int l0 = og_l0(g), nl = og_nl(g);
                    bool first[2] = {true, true};
                    for (int k = ks0 + c * OG_SPC; k < min(ks1, ks0 + (c + 1) * OG_SPC); ++k, ++gs) {
                        const int st = gs % OG_STAGES;
                        if (!tc::mbar_wait(full(st), (uint32_t)((gs / OG_STAGES) & 1), abort, err)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after();
                        const uint64_t d0 = tc::desc_sw64(sbase + st * OG_STAGE_BYTES);
#pragma unroll
                        for (int kk = 0; kk < OG_KS / 16; ++kk)
                            for (int li = 0; li < nl; ++li) {
                                const int l = l0 + li;
                                const uint32_t d = tmem + (uint32_t)(a * 256 + li * 128);
                                for (int s = og_smin(l); s <= og_smax(l); ++s) {
                                    const uint64_t da = d0 + (uint64_t)(s - 1) * slot16 + 2 * kk;
                                    const uint64_t db = d0 + (uint64_t)(OG_S + l - s - 1) * slot16 + 2 * kk;
                                    if (first[li]) tc::mma_bf16(d, da, db, OG_IDESC, 0u);
                                    else tc::mma_bf16_acc(d, da, db, OG_IDESC);
                                    first[li] = false;
                                }
                            }
                        tc::mma_commit(empty(st));
                    }
                    if (ok) tc::mma_commit(accf(a));
                }
            if (!ok) {   // MMAs in flight finish before TMEM is released
                tc::mma_commit(drain);
                og_drain(drain, 0);
            }
        }
    } else {
        const int wq = warp & 3, row = wq * 32 + lane, cq = ((warp - 2) >> 2) * 64;
        const uint32_t tl = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)cq;
        float hi[64], lo[64];
#pragma unroll
        for (int q = 0; q < 64; ++q) hi[q] = lo[q] = 0.f;
        bool ok = true;
        int cu = 0;
        for (int c = 0; c < nch && ok; ++c)
            for (int g = 0; g < OG_GROUPS; ++g, ++cu) {
                const int a = cu & 1;
                ok = __all_sync(0xffffffffu, tc::mbar_wait(accf(a), (uint32_t)((cu >> 1) & 1), abort, err));
                if (!ok) break;
                tc::fence_after();
                const int l0 = og_l0(g);
                const float sc0 = __int_as_float((127 - 7 * l0) << 23);         // 2^{-7 l0}
                const float sc1 = __int_as_float((127 - 7 * (l0 + 1)) << 23);   // 2^{-7 (l0 + 1)}
                const uint32_t ta = tl + (uint32_t)(a * 256);
                // one code path for both group shapes (two flush paths spilled registers): a
                // one-level group selects zero for the second accumulator, whose columns hold
                // an earlier group's sums
                const bool two = og_nl(g) == 2;
#pragma unroll
                for (int q8 = 0; q8 < 8; ++q8) {
                    float v0[8], v1[8];
                    tc::tmem_ld8x2(ta + 8 * q8, ta + 128 + 8 * q8, v0, v1);
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        og_two_sum(hi[8 * q8 + e], lo[8 * q8 + e], v0[e] * sc0);
                        og_two_sum(hi[8 * q8 + e], lo[8 * q8 + e], two ? v1[e] * sc1 : 0.f);
                    }
                }
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(acce(a));
            }
        // every MMA has completed (the last chunk's commit covers the earlier ones): the
        // running sums go to tensor memory and the epilogue walks them in a rolled loop
        if (ok) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float h16[16], l16[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    h16[e] = hi[16 * q + e];
                    l16[e] = lo[16 * q + e];
                }
                tc::tmem_st16(tl + 16 * q, h16);
                tc::tmem_st16(tl + 128 + 16 * q, l16);
            }
            tc::tmem_st_wait();
        }
        // The TMEM loads are warp-collective: every lane takes part, only live rows store.
        // sign mu_i mu_j is a power of two: when it is a normal FP32 number the scaling of hi and
        // lo is exact in FP32 and the FP64 work per element is two conversions and two adds
        // (the destination's loads are issued before the TMEM loads); otherwise FP64 throughout.
        const bool live = row < un.rows;
        const int ea = live ? pow2_exp(un.muA[row]) : 0;
        const double mi = live ? un.muA[row] : 0.0;
        double* drow = un.dst + (int64_t)row * un.ld + cq;
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            double base[16];
#pragma unroll
            for (int e = 0; e < 16; ++e)
                base[e] = (live && !un.overwrite && cq + 16 * q + e < un.cols) ? drow[16 * q + e] : 0.0;
            float h[16], lw[16];
            if (ok) tc::tmem_ld16x2(tl + 16 * q, tl + 128 + 16 * q, h, lw);
            if (!live) continue;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int col = cq + 16 * q + e;
                if (col >= un.cols) continue;
                double out;
                if (!ok) {
                    out = __longlong_as_double(0x7ff8000000000000ll);
                } else {
                    const double mj = un.muB[col];
                    const int ex = ea + pow2_exp(mj);
                    double v;
                    if (ex >= -126 && ex <= 127) {
                        const float sf = __int_as_float((un.sign < 0.0 ? (int)0x80000000 : 0) | ((127 + ex) << 23));
                        v = (double)(h[e] * sf) + (double)(lw[e] * sf);
                    } else {
                        v = ((double)h[e] + (double)lw[e]) * (un.sign * mi * mj);
                    }
                    out = base[e] + v;
                }
                drow[16 * q + e] = out;
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc::fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

// ---------------------------------------------------------------- operand slicing
// Row r of an operand = n consecutive FP64 values at src(r).  mu[r] = power
// of two >= max |row|, q = rint(v 2^49 / mu), OS[s][r][c] = s-th balanced
// digit of q (slices ps elements apart).  One warp per row, eight rows per CTA.
template <class Src>
__global__ void k_rowslices(Src src, int64_t rows, int64_t n, __nv_bfloat16* OS, int64_t ps, double* mu)
{
    const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const double* v = src(r);
    double mx = 0.0;
    for (int64_t c = lane; c < n; c += 32) mx = fmax(mx, fabs(v[c]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const double m = mx > 0.0 ? pow2_ceil(mx) : 1.0;
    const int sc = GP_OZ_BITS * OG_S - pow2_exp(m);   // v / m 2^49 = v 2^sc
    for (int64_t c = lane; c < n; c += 32) {
        __nv_bfloat16 d[OG_S];
        oz_digits<OG_S>(rint_scaled(v[c], sc), d);
#pragma unroll
        for (int s = 0; s < OG_S; ++s) OS[s * ps + r * n + c] = d[s];
    }
    if (lane == 0) mu[r] = m;
}

// Columns of the row tiles t0 .. t0 + nt - 1 of the lower-triangular
// X = L^{-1} as B-operand rows: row n = j b + c holds column c of the tiles
// (t, j) over their nt b rows (k = (t - t0) b + r), scaled by mu[n] = power of
// two >= its max |.|; entries above the diagonal (t < j, or t = j and r < c)
// are zero.  One CTA per 32 columns.
__global__ __launch_bounds__(256) void k_colslices_tile(const double* X, int64_t b, int64_t t0, int64_t nt,
                                                        __nv_bfloat16* OS, int64_t ps, double* mu)
{
    __shared__ double red[8][32];
    __shared__ double smu[32];
    const int64_t n0 = (int64_t)blockIdx.x * 32, j = n0 / b, c0 = n0 % b, K = nt * b;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    auto at = [&](int64_t k, int64_t c) -> double {   // X at row t0 b + k, column j b + c
        const int64_t t = t0 + k / b, r = k % b;
        if (t < j || (t == j && r < c)) return 0.0;
        return X[tri_index(t, j) * b * b + r * b + c];
    };
    double mx = 0.0;
    for (int64_t k = w; k < K; k += 8) mx = fmax(mx, fabs(at(k, c0 + lane)));
    red[w][lane] = mx;
    __syncthreads();
    if (w == 0) {
        for (int q = 1; q < 8; ++q) mx = fmax(mx, red[q][lane]);
        smu[lane] = mx > 0.0 ? pow2_ceil(mx) : 1.0;
        mu[n0 + lane] = smu[lane];
    }
    __syncthreads();
    for (int64_t k = threadIdx.x; k < K; k += 256)
        for (int c = 0; c < 32; ++c) {
            __nv_bfloat16 d[OG_S];
            oz_digits<OG_S>(rint_scaled(at(k, c0 + c), GP_OZ_BITS * OG_S - pow2_exp(smu[c])), d);
#pragma unroll
            for (int s = 0; s < OG_S; ++s) OS[s * ps + (n0 + c) * K + k] = d[s];
        }
}

// Column maxima of the lower-triangular X = L^{-1} (tiles (t, j), t >= j),
// as the bit patterns of non-negative doubles (ordered like the values):
// bits[n] = max over rows of |X_{.,n}|.  Grid: (column groups of 32, row tiles).
__global__ __launch_bounds__(256) void k_colmax_x(const double* X, int64_t b, unsigned long long* bits)
{
    __shared__ double red[8][32];
    const int64_t n0 = (int64_t)blockIdx.x * 32, j = n0 / b, c0 = n0 % b, t = blockIdx.y;
    if (t < j) return;
    const double* tile = X + tri_index(t, j) * b * b;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double mx = 0.0;
    for (int64_t r = w; r < b; r += 8)
        if (!(j == t && r < c0 + lane)) mx = fmax(mx, fabs(tile[r * b + c0 + lane]));
    red[w][lane] = mx;
    __syncthreads();
    if (w == 0) {
        for (int q = 1; q < 8; ++q) mx = fmax(mx, red[q][lane]);
        atomicMax(bits + n0 + lane, (unsigned long long)__double_as_longlong(mx));
    }
}

// X^T as digit slices for the LAUUM product: row n (column n of X), k = row
// of X, one power-of-two scale per column over all its rows (mu[n], from the
// column maxima); rows of X above the column's tile are never read and are
// not written.  Grid: (column groups of 32, row tiles t >= column tile).
__global__ __launch_bounds__(256) void k_colslices_x(const double* X, int64_t b, int64_t Np,
                                                     const unsigned long long* bits, __nv_bfloat16* OS, double* mu)
{
    __shared__ double smu[32];
    const int64_t n0 = (int64_t)blockIdx.x * 32, j = n0 / b, c0 = n0 % b, t = blockIdx.y;
    if (t < j) return;
    const double* tile = X + tri_index(t, j) * b * b;
    if (threadIdx.x < 32) {
        const double mx = __longlong_as_double((long long)bits[n0 + threadIdx.x]);
        smu[threadIdx.x] = mx > 0.0 ? pow2_ceil(mx) : 1.0;
        if (t == j) mu[n0 + threadIdx.x] = smu[threadIdx.x];
    }
    __syncthreads();
    const int64_t ps = Np * Np;
    for (int64_t r = threadIdx.x; r < b; r += 256)
        for (int c = 0; c < 32; ++c) {
            const double v = (j == t && r < c0 + c) ? 0.0 : tile[r * b + c0 + c];
            __nv_bfloat16 d[OG_S];
            oz_digits<OG_S>(rint_scaled(v, GP_OZ_BITS * OG_S - pow2_exp(smu[c])), d);
#pragma unroll
            for (int s = 0; s < OG_S; ++s) OS[s * ps + (n0 + c) * Np + t * b + r] = d[s];
        }
}

// Column maxima of a dense row-major block (nrows x 32 per CTA column group,
// row stride ld) as ordered bit patterns: bits[n] = max |src[., n]|.  Grid:
// (column groups of 32, row chunks of 256).
__global__ __launch_bounds__(256) void k_colmax_dense(const double* src, int64_t ld, int64_t nrows,
                                                      unsigned long long* bits)
{
    __shared__ double red[8][32];
    const int64_t n0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 256;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double mx = 0.0;
    for (int64_t r = r0 + w; r < nrows && r < r0 + 256; r += 8) mx = fmax(mx, fabs(src[r * ld + n0 + lane]));
    red[w][lane] = mx;
    __syncthreads();
    if (w == 0) {
        for (int q = 1; q < 8; ++q) mx = fmax(mx, red[q][lane]);
        atomicMax(bits + n0 + lane, (unsigned long long)__double_as_longlong(mx));
    }
}

// Columns of a dense row-major block as B-operand rows: row n holds column n
// over rows r0 .. r0 + 255 of src (k = r), scale mu[n] from bits[n] (column
// maxima); when bits is null, over all nrows rows with the scale from their
// own maximum (then one row chunk).  Grid: (column groups of 32, row chunks).
__global__ __launch_bounds__(256) void k_colslices_dense(const double* src, int64_t ld, int64_t nrows,
                                                         const unsigned long long* bits, __nv_bfloat16* OS,
                                                         int64_t ps, int64_t kstride, double* mu)
{
    __shared__ double red[8][32];
    __shared__ double smu[32];
    const int64_t n0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 256;
    // one chunk of 256 rows with given maxima; all rows of the block without
    const int64_t r1 = bits ? (r0 + 256 < nrows ? r0 + 256 : nrows) : nrows;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (bits) {
        if (threadIdx.x < 32) {
            const double mx = __longlong_as_double((long long)bits[n0 + threadIdx.x]);
            smu[threadIdx.x] = mx > 0.0 ? pow2_ceil(mx) : 1.0;
            if (blockIdx.y == 0) mu[n0 + threadIdx.x] = smu[threadIdx.x];
        }
    } else {
        double mx = 0.0;
        for (int64_t r = r0 + w; r < r1; r += 8) mx = fmax(mx, fabs(src[r * ld + n0 + lane]));
        red[w][lane] = mx;
        __syncthreads();
        if (w == 0) {
            for (int q = 1; q < 8; ++q) mx = fmax(mx, red[q][lane]);
            smu[lane] = mx > 0.0 ? pow2_ceil(mx) : 1.0;
            mu[n0 + lane] = smu[lane];
        }
    }
    __syncthreads();
    for (int64_t r = r0 + threadIdx.x; r < r1; r += 256)
        for (int c = 0; c < 32; ++c) {
            __nv_bfloat16 d[OG_S];
            oz_digits<OG_S>(rint_scaled(src[r * ld + n0 + c], GP_OZ_BITS * OG_S - pow2_exp(smu[c])), d);
#pragma unroll
            for (int s = 0; s < OG_S; ++s) OS[s * ps + (n0 + c) * kstride + r] = d[s];
        }
}

// As k_rowslices with the row given element by element (src(r, c)).
template <class Src>
__global__ void k_rowslices_v(Src src, int64_t rows, int64_t n, __nv_bfloat16* OS, int64_t ps, double* mu)
{
    const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    double mx = 0.0;
    for (int64_t c = lane; c < n; c += 32) mx = fmax(mx, fabs(src(r, c)));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const double m = mx > 0.0 ? pow2_ceil(mx) : 1.0;
    const int sc = GP_OZ_BITS * OG_S - pow2_exp(m);
    for (int64_t c = lane; c < n; c += 32) {
        __nv_bfloat16 d[OG_S];
        oz_digits<OG_S>(rint_scaled(src(r, c), sc), d);
#pragma unroll
        for (int s = 0; s < OG_S; ++s) OS[s * ps + r * n + c] = d[s];
    }
    if (lane == 0) mu[r] = m;
}

// Rows of the tiles r0t, r0t + 1, .. over the tile columns K0 .. K0 + w - 1
// (a super-panel): element (r, c) is row r % b, column c % b of tile
// (r0t + r / b, K0 + c / b).
struct SuperPanelRows {
    const double* L;
    int64_t b, K0, r0t;
    __device__ double operator()(int64_t r, int64_t c) const
    {
        return L[tri_index(r0t + r / b, K0 + c / b) * b * b + (r % b) * b + (c % b)];
    }
};

// Row r of the panel below the diagonal tile k: row r % b of tile (k + 1 + r / b, k).
struct PanelRows {
    const double* L;
    int64_t b, k;
    __device__ const double* operator()(int64_t r) const
    {
        return L + tri_index(k + 1 + r / b, k) * b * b + (r % b) * b;
    }
};

// Row r of the inverse Linv_kk of the diagonal tile k (upper triangle zero).
struct LinvRows {
    const double* Linv;
    int64_t b, k;
    __device__ const double* operator()(int64_t r) const { return Linv + k * b * b + r * b; }
};

// Partial sums of the V solve over 64-row blocks of V_j (rows j b ..):
// part[0][q][c] = sum V^2, part[1][q][c] = sum V beta, q = j P + block.
__global__ void k_vparts(const double* V, const double* beta, double* part, int64_t b, int64_t j, int64_t ldm,
                         int64_t nq)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ldm) return;
    const int64_t rb = blockIdx.y, row0 = j * b + rb * 64;
    double sq = 0.0, sb = 0.0;
    for (int r = 0; r < 64; ++r) {
        const double v = V[(row0 + r) * ldm + c];
        sq = fma(v, v, sq);
        sb = fma(v, beta[row0 + r], sb);
    }
    const int64_t q = j * (b / 64) + rb;
    part[q * ldm + c] = sq;
    part[(nq + q) * ldm + c] = sb;
}

// ---------------------------------------------------------------- operations
// Cholesky updates A_ij -= sum_k L_ik L_jk^T over the k range of one slice set:
// rows of the tiles r0t .. T-1 of one panel column (width b) or of one
// super-panel (SP tile columns, width SP b); A and B are both those slices.
// tri: every tile i >= j >= j0 (tt (tt+1) / 2 of them, tt = T - j0); else the
// columns j0 .. j0 + ncol - 1 with i >= j (a rectangle with its upper part skipped).
struct OgChol {
    double* L;
    const double* mu;
    int64_t b;
    int T, j0, ncol, r0t, width, P;
    bool tri;
    int a_ps, b_ps;
    const unsigned long long* info;
    __device__ bool unit(int u, OgUnit& o) const
    {
        if (failed(info)) return false;
        const int per = P * P;
        int64_t i, j;
        if (tri) {
            tri_decode(u / per, i, j);
            i += j0;
            j += j0;
        } else {
            const int q = u / per;
            j = j0 + q % ncol;
            i = j0 + q / ncol;
            if (i < j) return false;
        }
        const int rb = (u % per) / P, cb = (u % per) % P;
        if (i == j && cb > rb) return false;
        o.a_row = (int)((i - r0t) * b + rb * 128);
        o.b_row = (int)((j - r0t) * b + cb * 128);
        o.k0 = 0;
        o.k1 = width;
        o.dst = L + tri_index(i, j) * b * b + (int64_t)rb * 128 * b + cb * 128;
        o.ld = b;
        o.muA = mu + o.a_row;
        o.muB = mu + o.b_row;
        o.rows = o.cols = 128;
        o.sign = -1.0;
        o.overwrite = false;
        return true;
    }
};

// Step t of the triangular inverse: S_ij (+)= L_it X_tj for i > t >= j (the
// first contribution, t == j, stores), A = panel slices of column t, B =
// column slices of the tiles (t, 0 .. t) of X.
struct OgTrtri {
    double* Xinv;
    const double *muA, *muB;
    int64_t b;
    int i0, r0t, njt, T0, width, P;   // rows of tiles i0 .., columns j < njt, store when j >= T0
    int a_ps, b_ps;
    __device__ bool unit(int u, OgUnit& o) const
    {
        const int per = P * P, q = u / per;
        const int ii = q / njt, j = q % njt;
        const int rb = (u % per) / P, cb = (u % per) % P;
        const int64_t i = i0 + ii;
        o.a_row = (int)((i - r0t) * b + rb * 128);
        o.b_row = (int)(j * b + cb * 128);
        o.k0 = 0;
        o.k1 = width;
        o.dst = Xinv + tri_index(i, j) * b * b + (int64_t)rb * 128 * b + cb * 128;
        o.ld = b;
        o.muA = muA + o.a_row;
        o.muB = muB + o.b_row;
        o.rows = o.cols = 128;
        o.sign = 1.0;
        o.overwrite = (j >= T0);   // the first contribution to S_ij
        return true;
    }
};

// K^{-1}_ij = sum_{k >= i b} X_ki X_kj on lower tiles (LAUUM): A and B are
// rows of the column slices of all of X (one scale per column).
struct OgLauum {
    double* Kinv;
    const double* mu;
    int64_t b, Np;
    int P;
    int a_ps, b_ps;
    __device__ bool unit(int u, OgUnit& o) const
    {
        const int per = P * P;
        int64_t i, j;
        tri_decode(u / per, i, j);
        const int rb = (u % per) / P, cb = (u % per) % P;
        if (i == j && cb > rb) return false;
        o.a_row = (int)(i * b + rb * 128);
        o.b_row = (int)(j * b + cb * 128);
        o.k0 = (int)(i * b);
        o.k1 = (int)Np;
        o.dst = Kinv + tri_index(i, j) * b * b + (int64_t)rb * 128 * b + cb * 128;
        o.ld = b;
        o.muA = mu + o.a_row;
        o.muB = mu + o.b_row;
        o.rows = o.cols = 128;
        o.sign = 1.0;
        o.overwrite = true;
        return true;
    }
};

// Step j of the multi-right-hand-side solve V = L^{-1} K_{Z*,Z}^T:
// B_i -= L_ij V_j for i > j, A = panel slices of column j, B = the test
// columns of V_j (rows j b .. j b + b - 1 of V) as rows.
struct OgVsolve {
    double* B;
    const double *muA, *muB;
    int64_t b, ldm;
    int i0, r0t, width, P, nmb;   // rows of the tiles i0 .., slice row 0 = tile r0t, k range width
    int a_ps, b_ps;
    __device__ bool unit(int u, OgUnit& o) const
    {
        const int mb = u % nmb, rest = u / nmb;
        const int rb = rest % P;
        const int64_t i = i0 + rest / P;
        o.a_row = (int)((i - r0t) * b + rb * 128);
        o.b_row = mb * 128;
        o.k0 = 0;
        o.k1 = width;
        o.dst = B + (i * b + (int64_t)rb * 128) * ldm + (int64_t)mb * 128;
        o.ld = ldm;
        o.muA = muA + o.a_row;
        o.muB = muB + o.b_row;
        o.rows = o.cols = 128;
        o.sign = -1.0;
        o.overwrite = false;
        return true;
    }
};

// Full posterior covariance: cov (m x m, row stride m) -= V^T V, every
// 128 x 128 block (both triangles: the blocks are computed independently and
// come out exactly symmetric), A = B = the columns of V as rows.
struct OgCov {
    double* cov;
    const double* mu;
    int64_t m, Np;
    int nmb;
    int a_ps, b_ps;
    __device__ bool unit(int u, OgUnit& o) const
    {
        const int ra = u / nmb, cb = u % nmb;
        o.a_row = ra * 128;
        o.b_row = cb * 128;
        o.k0 = 0;
        o.k1 = (int)Np;
        o.dst = cov + (int64_t)ra * 128 * m + (int64_t)cb * 128;
        o.ld = m;
        o.muA = mu + o.a_row;
        o.muB = mu + o.b_row;
        o.rows = (int)(m - ra * 128 < 128 ? m - ra * 128 : 128);
        o.cols = (int)(m - cb * 128 < 128 ? m - cb * 128 : 128);
        o.sign = -1.0;
        o.overwrite = false;
        return true;
    }
};

// Panel solve of step k: L_ik = A_ik Linv_kk^T over the tiles (i, k), i > k
// (A = panel slices, B = rows of Linv_kk).
struct OgPanel {
    double* L;
    const double *muA, *muB;
    int64_t b;
    int k, P;
    int a_ps, b_ps;
    const unsigned long long* info;
    __device__ bool unit(int u, OgUnit& o) const
    {
        if (failed(info)) return false;   // a failed pivot: the factor is abandoned
        const int per = P * P, ii = u / per, rb = (u % per) / P, cb = (u % per) % P;
        o.a_row = (int)(ii * b + rb * 128);
        o.b_row = cb * 128;
        o.k0 = 0;
        o.k1 = (int)b;
        o.dst = L + tri_index(k + 1 + ii, k) * b * b + (int64_t)rb * 128 * b + cb * 128;
        o.ld = b;
        o.muA = muA + o.a_row;
        o.muB = muB + o.b_row;
        o.rows = o.cols = 128;
        o.sign = 1.0;
        o.overwrite = true;
        return true;
    }
};

// C = sign * A B^T stored over evenly spaced destination blocks, one k range
// of b: the inverse's scaling X_tj = -Linv_tt S_tj (A = rows of Linv_tt, B =
// columns of S_tj) and the V solve's V_j = Linv_jj B_j (A = rows of Linv_jj,
// B = test columns of B_j).
struct OgStore {
    double* base;            // destination of unit (blk, rb, cb): base + blk * bstride + rb 128 ld + cb 128
    int64_t bstride, ld;
    const double *muA, *muB;
    int nrb, ncb;            // 128-blocks per destination block along rows / columns
    int a_blk, b_blk;        // A / B row offset per destination block (0 when shared)
    int64_t b;
    double sign;
    int a_ps, b_ps;
    __device__ bool unit(int u, OgUnit& o) const
    {
        const int per = nrb * ncb, blk = u / per, rb = (u % per) / ncb, cb = (u % per) % ncb;
        o.a_row = blk * a_blk + rb * 128;
        o.b_row = blk * b_blk + cb * 128;
        o.k0 = 0;
        o.k1 = (int)b;
        o.dst = base + (int64_t)blk * bstride + (int64_t)rb * 128 * ld + (int64_t)cb * 128;
        o.ld = ld;
        o.muA = muA + o.a_row;
        o.muB = muB + o.b_row;
        o.rows = o.cols = 128;
        o.sign = sign;
        o.overwrite = true;
        return true;
    }
};

PFN_cuTensorMapEncodeTiled_v12000 og_encode_fn()
{
    static std::mutex mu_;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::lock_guard<std::mutex> lock(mu_);
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// Digit slices (OG_S x rows x n BF16, slice-major) as one 2-D map of
// 32-column x 128-row boxes, 64-byte swizzle.
bool og_map(CUtensorMap* map, const void* p, int64_t rows, int64_t n)
{
    auto enc = og_encode_fn();
    const int64_t all = OG_S * rows;
    if (!enc || ((uintptr_t)p & 15) || n % OG_KS || rows % 128 || all >= (1ll << 31)) return false;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)all};
    cuuint64_t strides[1] = {(cuuint64_t)n * 2};
    cuuint32_t box[2] = {(cuuint32_t)OG_KS, 128}, es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(p), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class Op>
bool og_launch(gp_t h, int phase, const CUtensorMap& mA, const CUtensorMap& mB, const Op& op, int64_t units)
{
    static int done_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (done_dev != dev) {
        cudaFuncSetAttribute(k_ozgemm<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, OG_SMEM);
        done_dev = dev;
    }
    if (units <= 0) return true;
    if (units >= (1ll << 31)) return false;
    int* err = tc_error_dev();
    if (!err) return false;
    GPK_LAUNCH(h, phase, k_ozgemm<Op>, (unsigned)units, OG_THREADS, OG_SMEM, mA, mB, op, err);
    h->tc_pending = true;
    return true;
}

}  // namespace

// Update of the super-panel's own later columns by its column k: A_ij -= L_ik
// L_jk^T for k < j < e, i >= j, from the panel slices of column k.
bool og_chol_update_cols(gp_t h, int64_t k, int64_t e)
{
    const int64_t T = h->T, b = h->b, tt = T - k - 1;
    if (tt <= 0 || e <= k + 1) return true;
    const int64_t rows = tt * b;
    GPK_LAUNCH(h, GP_PH_UPDATE, k_rowslices<PanelRows>, (unsigned)((rows + 7) / 8), 256, 0,
               PanelRows{h->L, b, k}, rows, b, h->OGP, rows * b, h->og_mu);
    CUtensorMap mP;
    if (!og_map(&mP, h->OGP, rows, b)) return false;
    OgChol op;
    op.L = h->L;
    op.mu = h->og_mu;
    op.b = b;
    op.T = (int)T;
    op.j0 = (int)(k + 1);
    op.ncol = (int)(e - k - 1);
    op.r0t = (int)(k + 1);
    op.width = (int)b;
    op.P = (int)(b / 128);
    op.tri = false;
    op.a_ps = op.b_ps = (int)rows;
    op.info = h->info;
    return og_launch(h, GP_PH_UPDATE, mP, mP, op, (T - k - 1) * op.ncol * op.P * op.P);
}

// Trailing update by a whole super-panel (tile columns K0 .. e-1): A_ij -=
// sum_{k in K0..e-1} L_ik L_jk^T for i >= j >= e, one k range of (e - K0) b.
bool og_chol_update_sp(gp_t h, int64_t K0, int64_t e)
{
    const int64_t T = h->T, b = h->b, tt = T - e;
    if (tt <= 0) return true;
    const int64_t rows = tt * b, width = (e - K0) * b;
    GPK_LAUNCH(h, GP_PH_UPDATE, k_rowslices_v<SuperPanelRows>, (unsigned)((rows + 7) / 8), 256, 0,
               SuperPanelRows{h->L, b, K0, e}, rows, width, h->OGS, rows * width, h->og_mu);
    CUtensorMap mP;
    if (!og_map(&mP, h->OGS, rows, width)) return false;
    OgChol op;
    op.L = h->L;
    op.mu = h->og_mu;
    op.b = b;
    op.T = (int)T;
    op.j0 = (int)e;
    op.ncol = (int)tt;
    op.r0t = (int)e;
    op.width = (int)width;
    op.P = (int)(b / 128);
    op.tri = true;
    op.a_ps = op.b_ps = (int)rows;
    op.info = h->info;
    return og_launch(h, GP_PH_UPDATE, mP, mP, op, tt * (tt + 1) / 2 * op.P * op.P);
}

// Step t of the triangular inverse on the tensor cores inside a block of
// rows ending at e (after the scaling X_tj = -Linv_tt S_tj of row block t):
// S_ij (+)= L_it X_tj for t < i < e, j <= t (the first contribution, j = t,
// stores), A = panel slices of column t, B = columns of the row block t of X.
bool og_trtri_accum(gp_t h, int64_t t, int64_t e)
{
    const int64_t b = h->b, ni = e - t - 1;
    if (ni <= 0) return true;
    const int64_t rows = ni * b, cols = (t + 1) * b;
    GPK_LAUNCH(h, GP_PH_TRTRI, k_rowslices<PanelRows>, (unsigned)((rows + 7) / 8), 256, 0,
               PanelRows{h->L, b, t}, rows, b, h->OGP, rows * b, h->og_mu);
    GPK_LAUNCH(h, GP_PH_TRTRI, k_colslices_tile, (unsigned)(cols / 32), 256, 0, (const double*)h->Xinv, b, t,
               (int64_t)1, h->OGT, cols * b, h->ogt_mu);
    CUtensorMap mA, mB;
    if (!og_map(&mA, h->OGP, rows, b) || !og_map(&mB, h->OGT, cols, b)) return false;
    OgTrtri op;
    op.Xinv = h->Xinv;
    op.muA = h->og_mu;
    op.muB = h->ogt_mu;
    op.b = b;
    op.i0 = op.r0t = (int)(t + 1);
    op.njt = (int)(t + 1);
    op.T0 = (int)t;
    op.width = (int)b;
    op.P = (int)(b / 128);
    op.a_ps = (int)rows;
    op.b_ps = (int)cols;
    return og_launch(h, GP_PH_TRTRI, mA, mB, op, ni * (t + 1) * op.P * op.P);
}

// The inverse's accumulation by a whole block of rows T0 .. e-1 of X:
// S_ij (+)= sum_t L_it X_tj for i >= e, j < e (stores for j >= T0, where
// these are the first contributions), one k range of (e - T0) b.
bool og_trtri_accum_sp(gp_t h, int64_t T0, int64_t e)
{
    const int64_t T = h->T, b = h->b, tt = T - e;
    if (tt <= 0) return true;
    const int64_t rows = tt * b, cols = e * b, width = (e - T0) * b;
    GPK_LAUNCH(h, GP_PH_TRTRI, k_rowslices_v<SuperPanelRows>, (unsigned)((rows + 7) / 8), 256, 0,
               SuperPanelRows{h->L, b, T0, e}, rows, width, h->OGS, rows * width, h->og_mu);
    GPK_LAUNCH(h, GP_PH_TRTRI, k_colslices_tile, (unsigned)(cols / 32), 256, 0, (const double*)h->Xinv, b, T0,
               e - T0, h->OGTS, cols * width, h->ogt_mu);
    CUtensorMap mA, mB;
    if (!og_map(&mA, h->OGS, rows, width) || !og_map(&mB, h->OGTS, cols, width)) return false;
    OgTrtri op;
    op.Xinv = h->Xinv;
    op.muA = h->og_mu;
    op.muB = h->ogt_mu;
    op.b = b;
    op.i0 = op.r0t = (int)e;
    op.njt = (int)e;
    op.T0 = (int)T0;
    op.width = (int)width;
    op.P = (int)(b / 128);
    op.a_ps = (int)rows;
    op.b_ps = (int)cols;
    return og_launch(h, GP_PH_TRTRI, mA, mB, op, tt * e * op.P * op.P);
}

// K^{-1} = X^T X (lower tiles) on the tensor cores from X = L^{-1}.
bool og_lauum(gp_t h)
{
    const int64_t T = h->T, b = h->b, Np = h->Np;
    cudaMemsetAsync(h->ogx_bits, 0, (size_t)Np * sizeof(unsigned long long), h->st);
    GPK_LAUNCH(h, GP_PH_LAUUM, k_colmax_x, dim3((unsigned)(Np / 32), (unsigned)T), 256, 0, (const double*)h->Xinv,
               b, h->ogx_bits);
    GPK_LAUNCH(h, GP_PH_LAUUM, k_colslices_x, dim3((unsigned)(Np / 32), (unsigned)T), 256, 0,
               (const double*)h->Xinv, b, Np, (const unsigned long long*)h->ogx_bits, h->OGX, h->ogx_mu);
    CUtensorMap mX;
    if (!og_map(&mX, h->OGX, Np, Np)) return false;
    OgLauum op;
    op.Kinv = h->Kinv;
    op.mu = h->ogx_mu;
    op.b = b;
    op.Np = Np;
    op.P = (int)(b / 128);
    op.a_ps = op.b_ps = (int)Np;
    return og_launch(h, GP_PH_LAUUM, mX, mX, op, T * (T + 1) / 2 * op.P * op.P);
}

// Step j of the V solve on the tensor cores, inside a block of columns
// ending at e: B_i -= L_ij V_j for j < i < e.
bool og_vsolve_update(gp_t h, int64_t j, int64_t e, int64_t ldm)
{
    const int64_t b = h->b, ni = e - j - 1;
    if (ni <= 0) return true;
    const int64_t rows = ni * b;
    GPK_LAUNCH(h, GP_PH_VSOLVE, k_rowslices<PanelRows>, (unsigned)((rows + 7) / 8), 256, 0,
               PanelRows{h->L, b, j}, rows, b, h->OGP, rows * b, h->og_mu);
    GPK_LAUNCH(h, GP_PH_VSOLVE, k_colslices_dense, dim3((unsigned)(ldm / 32), 1), 256, 0,
               (const double*)(h->V + j * b * ldm), ldm, b, (const unsigned long long*)nullptr, h->OGV, ldm * b, b,
               h->ogv_mu);
    CUtensorMap mA, mB;
    if (!og_map(&mA, h->OGP, rows, b) || !og_map(&mB, h->OGV, ldm, b)) return false;
    OgVsolve op;
    op.B = h->B;
    op.muA = h->og_mu;
    op.muB = h->ogv_mu;
    op.b = b;
    op.ldm = ldm;
    op.i0 = op.r0t = (int)(j + 1);
    op.width = (int)b;
    op.P = (int)(b / 128);
    op.nmb = (int)(ldm / 128);
    op.a_ps = (int)rows;
    op.b_ps = (int)ldm;
    return og_launch(h, GP_PH_VSOLVE, mA, mB, op, ni * op.P * op.nmb);
}

// The V solve's update by a whole block of columns J0 .. e-1:
// B_i -= sum_j L_ij V_j for every tile i >= e, one k range of (e - J0) b.
bool og_vsolve_update_sp(gp_t h, int64_t J0, int64_t e, int64_t ldm)
{
    const int64_t T = h->T, b = h->b, tt = T - e;
    if (tt <= 0) return true;
    const int64_t rows = tt * b, width = (e - J0) * b;
    GPK_LAUNCH(h, GP_PH_VSOLVE, k_rowslices_v<SuperPanelRows>, (unsigned)((rows + 7) / 8), 256, 0,
               SuperPanelRows{h->L, b, J0, e}, rows, width, h->OGS, rows * width, h->og_mu);
    GPK_LAUNCH(h, GP_PH_VSOLVE, k_colslices_dense, dim3((unsigned)(ldm / 32), 1), 256, 0,
               (const double*)(h->V + J0 * b * ldm), ldm, width, (const unsigned long long*)nullptr, h->OGVS,
               ldm * width, width, h->ogv_mu);
    CUtensorMap mA, mB;
    if (!og_map(&mA, h->OGS, rows, width) || !og_map(&mB, h->OGVS, ldm, width)) return false;
    OgVsolve op;
    op.B = h->B;
    op.muA = h->og_mu;
    op.muB = h->ogv_mu;
    op.b = b;
    op.ldm = ldm;
    op.i0 = op.r0t = (int)e;
    op.width = (int)width;
    op.P = (int)(b / 128);
    op.nmb = (int)(ldm / 128);
    op.a_ps = (int)rows;
    op.b_ps = (int)ldm;
    return og_launch(h, GP_PH_VSOLVE, mA, mB, op, tt * op.P * op.nmb);
}

// cov -= V^T V on the tensor cores (cov holds the test prior K_{Z*,Z*}).
bool og_full_cov(gp_t h, int64_t m, int64_t ldm, double* cov)
{
    const int64_t Np = h->Np;
    cudaMemsetAsync(h->ogc_bits, 0, (size_t)ldm * sizeof(unsigned long long), h->st);
    const unsigned chunks = (unsigned)((Np + 255) / 256);
    GPK_LAUNCH(h, GP_PH_COV, k_colmax_dense, dim3((unsigned)(ldm / 32), chunks), 256, 0, (const double*)h->V, ldm,
               Np, h->ogc_bits);
    GPK_LAUNCH(h, GP_PH_COV, k_colslices_dense, dim3((unsigned)(ldm / 32), chunks), 256, 0, (const double*)h->V,
               ldm, Np, (const unsigned long long*)h->ogc_bits, h->OGC, ldm * Np, Np, h->ogc_mu);
    CUtensorMap mV;
    if (!og_map(&mV, h->OGC, ldm, Np)) return false;
    OgCov op;
    op.cov = cov;
    op.mu = h->ogc_mu;
    op.m = m;
    op.Np = Np;
    op.nmb = (int)((m + 127) / 128);
    op.a_ps = op.b_ps = (int)ldm;
    return og_launch(h, GP_PH_COV, mV, mV, op, (int64_t)op.nmb * op.nmb);
}

// Row slices of the diagonal-tile inverse Linv_kk (b rows) into OGL.
static void og_linv_slices(gp_t h, int64_t k, int phase)
{
    const int64_t b = h->b;
    GPK_LAUNCH(h, phase, k_rowslices<LinvRows>, (unsigned)((b + 7) / 8), 256, 0, LinvRows{h->Linv, b, k}, b, b,
               h->OGL, b * b, h->ogl_mu);
}

// Panel solve of step k on the tensor cores: L_ik = A_ik Linv_kk^T, i > k.
bool og_panel(gp_t h, int64_t k)
{
    const int64_t T = h->T, b = h->b, tt = T - k - 1;
    if (tt <= 0) return true;
    const int64_t rows = tt * b;
    GPK_LAUNCH(h, GP_PH_TRSM, k_rowslices<PanelRows>, (unsigned)((rows + 7) / 8), 256, 0,
               PanelRows{h->L, b, k}, rows, b, h->OGP, rows * b, h->og_mu);
    og_linv_slices(h, k, GP_PH_TRSM);
    CUtensorMap mA, mB;
    if (!og_map(&mA, h->OGP, rows, b) || !og_map(&mB, h->OGL, b, b)) return false;
    OgPanel op;
    op.L = h->L;
    op.muA = h->og_mu;
    op.muB = h->ogl_mu;
    op.b = b;
    op.k = (int)k;
    op.P = (int)(b / 128);
    op.a_ps = (int)rows;
    op.b_ps = (int)b;
    op.info = h->info;
    return og_launch(h, GP_PH_TRSM, mA, mB, op, tt * op.P * op.P);
}

// Scaling of step t of the triangular inverse on the tensor cores:
// X_tj = -Linv_tt S_tj for j < t, over S_tj.
bool og_trtri_scale(gp_t h, int64_t t)
{
    const int64_t b = h->b, cols = t * b;
    if (t <= 0) return true;
    og_linv_slices(h, t, GP_PH_TRTRI);
    GPK_LAUNCH(h, GP_PH_TRTRI, k_colslices_tile, (unsigned)(cols / 32), 256, 0, (const double*)h->Xinv, b, t,
               (int64_t)1, h->OGT, cols * b, h->ogt_mu);
    CUtensorMap mA, mB;
    if (!og_map(&mA, h->OGL, b, b) || !og_map(&mB, h->OGT, cols, b)) return false;
    OgStore op;
    op.base = h->Xinv + tri_index(t, 0) * b * b;   // tiles (t, 0 .. t-1) are consecutive
    op.bstride = b * b;
    op.ld = b;
    op.muA = h->ogl_mu;
    op.muB = h->ogt_mu;
    op.nrb = op.ncb = (int)(b / 128);
    op.a_blk = 0;
    op.b_blk = (int)b;
    op.b = b;
    op.sign = -1.0;
    op.a_ps = (int)b;
    op.b_ps = (int)cols;
    return og_launch(h, GP_PH_TRTRI, mA, mB, op, t * op.nrb * op.ncb);
}

// Diagonal step j of the V solve on the tensor cores: V_j = Linv_jj B_j (rows
// j b .. of V), then its partial sums of V^2 and V beta.
bool og_vsolve_diag(gp_t h, int64_t j, int64_t ldm)
{
    const int64_t b = h->b;
    og_linv_slices(h, j, GP_PH_VSOLVE);
    GPK_LAUNCH(h, GP_PH_VSOLVE, k_colslices_dense, dim3((unsigned)(ldm / 32), 1), 256, 0,
               (const double*)(h->B + j * b * ldm), ldm, b, (const unsigned long long*)nullptr, h->OGV, ldm * b, b,
               h->ogv_mu);
    CUtensorMap mA, mB;
    if (!og_map(&mA, h->OGL, b, b) || !og_map(&mB, h->OGV, ldm, b)) return false;
    OgStore op;
    op.base = h->V + j * b * ldm;
    op.bstride = 128;   // one destination block per 128 test columns
    op.ld = ldm;
    op.muA = h->ogl_mu;
    op.muB = h->ogv_mu;
    op.nrb = (int)(b / 128);
    op.ncb = 1;
    op.a_blk = 0;
    op.b_blk = 128;
    op.b = b;
    op.sign = 1.0;
    op.a_ps = (int)b;
    op.b_ps = (int)ldm;
    if (!og_launch(h, GP_PH_VSOLVE, mA, mB, op, (ldm / 128) * op.nrb)) return false;
    GPK_LAUNCH(h, GP_PH_VSOLVE, k_vparts, dim3((unsigned)((ldm + 255) / 256), (unsigned)(b / 64)), 256, 0,
               (const double*)h->V, (const double*)h->beta, h->part, b, j, ldm, h->Np / 64);
    return true;
}

}  // namespace gpk
