// Split-BF16 ("bf16x6") block products of the mixed path on tcgen05.
//
// Every FP32 operand X is held as three BF16 planes X = X0 + X1 + X2 (round
// to nearest at each step); a product A B^T is taken as the six plane
// products Aa Bb^T with a + b <= 2, accumulated in FP32, which reproduces the
// FP32 product to about FP32 rounding.  One persistent kernel template,
// k_tgemm<Op>, runs all of them: a work unit is a 128 x N output block (N =
// Op::kN, 256 where the tile edge allows it, else 128) with one or more
// k-segments; Op names the operand tiles, the units and the epilogue.
//
// A 128 x 256 x 16 MMA reads 12 KB of operands from shared memory in 128
// clocks, a 128 x 128 x 16 one 8 KB in 64: the wide tile leaves shared-memory
// bandwidth for the TMA fill and halves the A traffic per flop.
//
// Roles (320 threads, one CTA per SM, grid = min(units, SMs)): warp 0 issues
// the TMA loads of a 32-k stage — the three A planes (128 x 32 each) as one
// box and the three B planes (N x 32 each) as one box, 64-byte swizzle —
// into a ring of 3 (N = 256) or 4 (N = 128) stages; warp 1 owns 2N TMEM
// columns (two 128 x N FP32 accumulators, alternating between units) and
// issues the six plane MMAs per 16-k step; warps 2-9 run the epilogue of unit
// c while the MMAs of unit c+1 proceed: two warps per TMEM lane quarter, each
// thread one output row and N/2 columns in 64-column chunks, each chunk's
// read-modify-write loads issued before its TMEM reads.  Waits are bounded
// (see tc_common.cuh); a timeout sets the device error word and the CTA
// leaves without touching its outputs.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>

#include "split_bf16.cuh"
#include "gp_internal.cuh"
#include "se_common.cuh"
#include "tc_common.cuh"

namespace gpk {
namespace {

constexpr int TG_THREADS = 320;
constexpr int TG_EPI_WARPS = 8;
constexpr int TG_KS = 32;                          // k per stage
constexpr int TG_APLANE = 128 * TG_KS * 2;         // bytes of one 128-row A plane tile

// P = operand planes used (3: the six plane products a + b <= 2, FP32
// accuracy; 2: the three with a + b <= 1, about 2^-16 relative; 1: the
// leading planes only, about 2^-8): a stage holds P planes of A and of B.
template <int N, int P = 3>
struct TgCfg {
    static_assert(P >= 1 && P <= 3, "one to three planes");
    static constexpr int BPLANE = N * TG_KS * 2;                 // bytes of one N-row B plane tile
    static constexpr int STAGE = P * TG_APLANE + P * BPLANE;     // P = 3: 48 KB (N = 128) or 72 KB (N = 256)
    static constexpr int STAGES = (216 * 1024 / STAGE) < 12 ? (216 * 1024 / STAGE) : 12;
    static constexpr int BAR_OFF = STAGES * STAGE;
    static constexpr int SMEM = 1024 + BAR_OFF + 256;
    static constexpr uint32_t IDESC = tc::idesc_bf16(128, N);
    static constexpr uint32_t IDESC_BMN = tc::idesc_bf16_bmn(128, N);
};

// Operand coordinates of one k-segment: the A planes are the 128-row box at
// plane-0 row a_row, k-columns a_x + [k0, k1); likewise the N-row B box when
// B is K-major.  An Op with kBMN set gives B as K x N with n contiguous (the
// NN form): its planes hold k rows b_row + [k0, k1), n columns b_x + [0, N).
// k0 and k1 are multiples of 32.
struct Seg {
    int a_row, a_x, b_row, b_x, k0, k1;
};

__device__ __forceinline__ bool seg_wait_drain(uint32_t mbar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!tc::mbar_try(mbar, parity))
        if (clock64() - t0 > tc::WAIT_CYCLES) return false;
    return true;
}

template <class Op>
__global__ __launch_bounds__(TG_THREADS, 1) void k_tgemm(const __grid_constant__ CUtensorMap mapA,
                                                         const __grid_constant__ CUtensorMap mapB, const Op op,
                                                         int* err)
{
    using C = TgCfg<Op::kN, Op::kP>;
    extern __shared__ unsigned char dyn[];
    if (op.skip_all()) return;
    unsigned char* base = dyn + ((1024 - (tc::su32(dyn) & 1023)) & 1023);
    const uint32_t sbase = tc::su32(base);
    const uint32_t bar = sbase + C::BAR_OFF;   // full[S], empty[S], accf[2], acce[2], drain
    auto full = [&](int s) { return bar + 8 * s; };
    auto empty = [&](int s) { return bar + 8 * (C::STAGES + s); };
    auto accf = [&](int a) { return bar + 8 * (2 * C::STAGES + a); };
    auto acce = [&](int a) { return bar + 8 * (2 * C::STAGES + 2 + a); };
    const uint32_t drain = bar + 8 * (2 * C::STAGES + 4);
    uint32_t* tmem_slot = (uint32_t*)(base + C::BAR_OFF + 8 * (2 * C::STAGES + 5));
    volatile int* abort = (volatile int*)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            tc::mbar_init(full(s), 1);
            tc::mbar_init(empty(s), 1);
        }
        tc::mbar_init(accf(0), 1);
        tc::mbar_init(accf(1), 1);
        tc::mbar_init(acce(0), TG_EPI_WARPS);
        tc::mbar_init(acce(1), TG_EPI_WARPS);
        tc::mbar_init(drain, 1);
        *abort = 0;
        tc::mbar_init_fence();
    }
    if (warp == 1) tc::tmem_alloc(tc::su32(tmem_slot), 2 * Op::kN);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nunits = op.units();

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            const uint64_t pol = tc::policy_evict_last();
            for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
                if (!op.active(u)) continue;
                const int ns = op.nseg(u);
                for (int q = 0; q < ns && ok; ++q) {
                    const Seg sg = op.seg(u, q);
                    for (int k = sg.k0; k < sg.k1; k += TG_KS, ++it) {
                        const int st = it % C::STAGES, use = it / C::STAGES;
                        if (use > 0 && !tc::mbar_wait(empty(st), (uint32_t)((use - 1) & 1), abort, err)) {
                            ok = false;
                            break;
                        }
                        const uint32_t dst = sbase + st * C::STAGE;
                        tc::mbar_expect_tx(full(st), C::STAGE);
                        // one box per operand: the P planes are the box's last dimension
                        tc::tma_load_3d_hint(dst, &mapA, sg.a_x + k, sg.a_row, 0, full(st), pol);
                        if (Op::kBMN)
                            tc::tma_load_4d_hint(dst + Op::kP * TG_APLANE, &mapB, 0, sg.b_row + k, sg.b_x / 64, 0,
                                                 full(st), pol);
                        else
                            tc::tma_load_3d_hint(dst + Op::kP * TG_APLANE, &mapB, sg.b_x + k, sg.b_row, 0, full(st),
                                                 pol);
                    }
                }
            }
            if (!ok)
                for (int q = it - 1; q >= 0 && q >= it - C::STAGES; --q)
                    seg_wait_drain(full(q % C::STAGES), (uint32_t)((q / C::STAGES) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, c = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
                if (!op.active(u)) continue;
                const int a = c & 1;
                if (c >= 2 && !tc::mbar_wait(acce(a), (uint32_t)(((c >> 1) - 1) & 1), abort, err)) {
                    ok = false;
                    break;
                }
                tc::fence_after();
                const uint32_t d = tmem + (uint32_t)(a * Op::kN);
                bool first = true;
                const int ns = op.nseg(u);
                for (int q = 0; q < ns && ok; ++q) {
                    const Seg sg = op.seg(u, q);
                    for (int k = sg.k0; k < sg.k1; k += TG_KS, ++it) {
                        const int st = it % C::STAGES;
                        if (!tc::mbar_wait(full(st), (uint32_t)((it / C::STAGES) & 1), abort, err)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after();
                        // stage descriptors once; plane tiles follow each other, a 16-k step adds 32
                        // bytes (K-major) or 2048 bytes (MN-major B)
                        const uint32_t s0 = sbase + st * C::STAGE;
                        const uint64_t da = tc::desc_sw64(s0);
                        const uint64_t db = Op::kBMN ? tc::desc_mn32_sw128(s0 + Op::kP * TG_APLANE)
                                                     : tc::desc_sw64(s0 + Op::kP * TG_APLANE);
                        constexpr uint64_t apl = (uint64_t)(TG_APLANE >> 4);
                        constexpr uint64_t bpl = (uint64_t)(C::BPLANE >> 4);
                        constexpr uint64_t bstep = Op::kBMN ? (2048 >> 4) : 2;
                        constexpr uint32_t idesc = Op::kBMN ? C::IDESC_BMN : C::IDESC;
                        if (first) tc::mma_bf16(d, da, db, idesc, 0u);
                        else tc::mma_bf16_acc(d, da, db, idesc);
                        first = false;
#pragma unroll
                        for (int kk = 0; kk < TG_KS / 16; ++kk)
#pragma unroll
                            for (int qa = 0; qa < Op::kP; ++qa)
#pragma unroll
                                for (int qb = 0; qa + qb < Op::kP; ++qb) {
                                    if (kk == 0 && qa == 0 && qb == 0) continue;
                                    tc::mma_bf16_acc(d, da + qa * apl + 2 * kk, db + qb * bpl + bstep * kk, idesc);
                                }
                        tc::mma_commit(empty(st));
                    }
                }
                if (!ok) break;
                tc::mma_commit(accf(a));
                ++c;
            }
            if (!ok) {
                tc::mma_commit(drain);
                seg_wait_drain(drain, 0);
            }
        }
    } else {
        const int wq = warp & 3, row = wq * 32 + lane, c0 = ((warp - 2) >> 2) * (Op::kN / 2);
        const uint32_t lrow = (uint32_t)(wq * 32) << 16;
        int c = 0;
        for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
            if (!op.active(u)) continue;
            const int a = c & 1;
            auto wait = [&]() {
                const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(accf(a), (uint32_t)((c >> 1) & 1), abort, err));
                if (ok) tc::fence_after();
                return ok;
            };
            if (!op.epilogue(u, row, c0, tmem + lrow + (uint32_t)(a * Op::kN), wait)) break;
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(acce(a));
            ++c;
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc::fence_after();
        tc::tmem_dealloc(tmem, 2 * Op::kN);
    }
}

// ---------------------------------------------------------------- epilogue helpers
// 64 FP32 values of one row: p must be 16-byte aligned.
struct Row64 {
    float4 x[16];
};

// Epilogue traffic is read or written once: streaming (evict-first) accesses
// keep it from displacing the operand tiles in L2.
__device__ __forceinline__ void row_load(Row64& r, const float* p)
{
#pragma unroll
    for (int q = 0; q < 16; ++q) r.x[q] = __ldcs((const float4*)p + q);
}

__device__ __forceinline__ void row_store(float* p, const float (&v)[32], int h)
{
#pragma unroll
    for (int q = 0; q < 8; ++q)
        __stcs((float4*)p + 8 * h + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
}

// p[32h + e] = base[32h + e] + sign * v[e] for the 32 values of half h.
__device__ __forceinline__ void row_axpy(float* p, const Row64& base, const float (&v)[32], int h, float sign)
{
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        float4 x = base.x[8 * h + q];
        x.x += sign * v[4 * q];
        x.y += sign * v[4 * q + 1];
        x.z += sign * v[4 * q + 2];
        x.w += sign * v[4 * q + 3];
        __stcs((float4*)p + 8 * h + q, x);
    }
}

// Three BF16 planes of 32 values at p, p + ps, p + 2 ps (16-byte aligned).
__device__ __forceinline__ void planes32(__nv_bfloat16* p, int64_t ps, const float (&v)[32], float sign = 1.f)
{
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        __align__(16) __nv_bfloat16 hb[3][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) split3(sign * v[8 * g + q], hb[0][q], hb[1][q], hb[2][q]);
#pragma unroll
        for (int pl = 0; pl < 3; ++pl) *(uint4*)(p + pl * ps + 8 * g) = *(const uint4*)&hb[pl][0];
    }
}

// This thread's ncols accumulator columns c0 .. c0 + ncols of one row,
// folded into the FP32 row dst (column 0 of the unit): dst[col] += sign * v
// (store = false) or dst[col] = v (store = true), in 64-column chunks whose
// loads are issued before the chunk's TMEM reads.  Chunks that start at or
// beyond column limit are left untouched.  Calls wait() once, first.
template <class W>
__device__ __forceinline__ bool epi_rows(float* dst, uint32_t t, int c0, int ncols, float sign, bool store,
                                         int limit, W&& wait)
{
    bool waited = false;
#pragma unroll 1
    for (int h64 = 0; h64 < ncols; h64 += 64) {
        const int col = c0 + h64;
        const bool skip = col >= limit;
        Row64 cur;
        if (!store && !skip) row_load(cur, dst + col);
        if (!waited) {
            if (!wait()) return false;
            waited = true;
        }
        if (skip) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tc::tmem_ld32(t + col + 32 * h, v);
            if (store) row_store(dst + col, v, h);
            else row_axpy(dst + col, cur, v, h, sign);
        }
    }
    return true;
}

// ---------------------------------------------------------------- operations
// All tile stores are b x b row-major; LP, ZP: three planes per lower tile
// (tile t at rows 3 t b of the plane array); LinvP: three planes per diagonal
// tile; PA: three planes per panel slot.  Q = b / 128 row blocks per tile,
// Qn = b / N column units per tile.

// Cholesky panel: L_ik = A_ik Linv_kk^T, k-range of Linv_kk's lower rows of
// the column unit; FP32 L_ik over A_ik and its planes into LP.
template <int N>
struct OpPanel {
    static constexpr bool kBMN = false;
    static constexpr int kN = N;
    static constexpr int kP = 3;
    float* A32;
    __nv_bfloat16* LP;
    int b, k, tt, Q, Qn;
    const unsigned long long* info;
    __device__ bool skip_all() const { return failed(info); }
    __device__ int units() const { return tt * Q * Qn; }
    __device__ bool active(int) const { return true; }
    __device__ int nseg(int) const { return 1; }
    __device__ Seg seg(int u, int) const
    {
        const int y = u / (Q * Qn), r = u % (Q * Qn), rb = r / Qn, cn = r % Qn;
        return Seg{y * 3 * b + rb * 128, 0, k * 3 * b + cn * N, 0, 0, (cn + 1) * N};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t t, W&& wait) const
    {
        const int y = u / (Q * Qn), r = u % (Q * Qn), rb = r / Qn, cn = r % Qn;
        const int64_t i = k + 1 + y, bb = (int64_t)b * b;
        const int64_t off = (int64_t)(rb * 128 + row) * b + cn * N;
        float* dst = A32 + tri_index(i, k) * bb + off;
        __nv_bfloat16* lp = LP + 3 * tri_index(i, k) * bb + off;
        if (!wait()) return false;
#pragma unroll 1
        for (int h = 0; h < N / 2; h += 32) {
            float v[32];
            tc::tmem_ld32(t + c0 + h, v);
            row_store(dst + c0 + h, v, 0);
            planes32(lp + c0 + h, bb, v);
        }
        return true;
    }
};

// Trailing update: A_ij -= sum_{k in [k0, k0 + nsrc)} L_ik L_jk^T over the
// target tiles of a band of w columns j in [j0, j0 + w) and all rows i in
// [j, T) (one k-segment per source column).  w = T - j0 is the whole
// trailing triangle.  Units: the rows j0 .. j0+w-2 hold 1 .. w-1 tiles of the
// band (the triangle part, row j0 + r holding r + 1), every later row w tiles.  In diagonal tiles only
// the column blocks up to the row's own diagonal 128-block are written.
template <int N>
struct OpUpdate {
    static constexpr bool kBMN = false;
    static constexpr int kN = N;
    static constexpr int kP = 3;
    float* A32;
    int b, k0, nsrc, j0, w, T, Q, Qn;
    const unsigned long long* info;
    __device__ bool skip_all() const { return failed(info); }
    __device__ int units() const { return (w * (w - 1) / 2 + w * (T - j0 - w + 1)) * Q * Qn; }
    __device__ void decode(int u, int64_t& i, int64_t& j, int& rb, int& cn) const
    {
        const int64_t p = u / (Q * Qn), tp = (int64_t)w * (w - 1) / 2;
        if (p < tp) {
            int64_t r, c;
            tri_decode(p, r, c);
            i = j0 + r;
            j = j0 + c;
        } else {
            const int64_t v = p - tp;
            i = j0 + w - 1 + v / w;
            j = j0 + v % w;
        }
        rb = (u % (Q * Qn)) / Qn;
        cn = u % Qn;
    }
    __device__ bool active(int u) const
    {
        int64_t i, j;
        int rb, cn;
        decode(u, i, j, rb, cn);
        return !(i == j && cn * N > rb * 128);
    }
    __device__ int nseg(int) const { return nsrc; }
    __device__ Seg seg(int u, int q) const
    {
        int64_t i, j;
        int rb, cn;
        decode(u, i, j, rb, cn);
        const int64_t k = k0 + q;
        return Seg{(int)(tri_index(i, k) * 3 * b) + rb * 128, 0, (int)(tri_index(j, k) * 3 * b) + cn * N, 0, 0, b};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t t, W&& wait) const
    {
        int64_t i, j;
        int rb, cn;
        decode(u, i, j, rb, cn);
        float* dst = A32 + tri_index(i, j) * (int64_t)b * b + (int64_t)(rb * 128 + row) * b + cn * N;
        const int limit = (i == j) ? (rb + 1) * 128 - cn * N : N;
        return epi_rows(dst, t, c0, N / 2, -1.f, false, limit, wait);
    }
};

// Forward multi-RHS solve, super-block step: W_I = R_I X_I^T, X_I the
// inverse of the super-block's diagonal block (R_I planes in RP, row stride
// B = GP_SOLVE_SB b; X_I planes K-major, rows xrow0 ..); planes of W_I into
// WP, FP32 W_I over R, FP64 row sums of W_I^2 into vpart (one slot per 64
// columns).  X_I is lower triangular: column unit cn needs k < (cn + 1) N.
template <int N, int P = 3>
struct OpDiagWSB {
    static constexpr bool kBMN = false;
    static constexpr int kN = N;
    static constexpr int kP = P;
    __nv_bfloat16* WP;
    float* Wout;
    double* vpart;
    int64_t ldw, ldm;
    int col0, xrow0, Qn, nmb;
    __device__ bool skip_all() const { return false; }
    __device__ int units() const { return Qn * nmb; }
    __device__ bool active(int) const { return true; }
    __device__ int nseg(int) const { return 1; }
    __device__ Seg seg(int u, int) const
    {
        const int cn = u % Qn, mb = u / Qn;
        return Seg{mb * 128, 0, xrow0 + cn * N, 0, 0, (cn + 1) * N};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t t, W&& wait) const
    {
        const int cn = u % Qn, mb = u / Qn;
        const int64_t r = (int64_t)mb * 128 + row;
        const int64_t o = r * ldw + col0 + cn * N;
        if (!wait()) return false;
#pragma unroll 1
        for (int h64 = 0; h64 < N / 2; h64 += 64) {
            double sq = 0.0;
#pragma unroll 1
            for (int h = 0; h < 64; h += 32) {
                float v[32];
                tc::tmem_ld32(t + c0 + h64 + h, v);
                planes32(WP + o + c0 + h64 + h, ldm * ldw, v);
                row_store(Wout + o + c0 + h64 + h, v, 0);
#pragma unroll
                for (int q = 0; q < 32; ++q) sq += (double)v[q] * v[q];
            }
            vpart[(((int64_t)col0 + cn * N + c0 + h64) / 64) * ldm + r] = sq;
        }
        return true;
    }
};

// Forward multi-RHS solve, diagonal step: W_j = R_j Linv_jj^T; planes of W_j
// into WP, FP32 W_j over R_j, FP64 row sums of W_j^2 into vpart (one slot per
// 64 columns).
template <int N, int P = 3>
struct OpDiagW {
    static constexpr bool kBMN = false;
    static constexpr int kN = N;
    static constexpr int kP = P;
    __nv_bfloat16* WP;
    float* Wout;
    double* vpart;
    int64_t ldw, ldm;
    int b, j, Qn, nmb;
    __device__ bool skip_all() const { return false; }
    __device__ int units() const { return Qn * nmb; }
    __device__ bool active(int) const { return true; }
    __device__ int nseg(int) const { return 1; }
    __device__ Seg seg(int u, int) const
    {
        const int cn = u % Qn, mb = u / Qn;
        return Seg{mb * 128, 0, j * 3 * b + cn * N, 0, 0, (cn + 1) * N};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t t, W&& wait) const
    {
        const int cn = u % Qn, mb = u / Qn;
        const int64_t r = (int64_t)mb * 128 + row;
        const int64_t o = r * ldw + (int64_t)j * b + cn * N;
        if (!wait()) return false;
#pragma unroll 1
        for (int h64 = 0; h64 < N / 2; h64 += 64) {
            double sq = 0.0;
#pragma unroll 1
            for (int h = 0; h < 64; h += 32) {
                float v[32];
                tc::tmem_ld32(t + c0 + h64 + h, v);
                planes32(WP + o + c0 + h64 + h, ldm * ldw, v);
                row_store(Wout + o + c0 + h64 + h, v, 0);
#pragma unroll
                for (int q = 0; q < 32; ++q) sq += (double)v[q] * v[q];
            }
            vpart[(((int64_t)j * b + cn * N + c0 + h64) / 64) * ldm + r] = sq;
        }
        return true;
    }
};

// Forward multi-RHS solve, update: R_i -= sum_{j in [j0, j0 + nsrc)} W_j L_ij^T
// for the target tiles i in [i0, i0 + ni), one k-segment per source column
// (the block step of the sweep: R_i is read and written once per block).
template <int N, int P = 3>
struct OpUpdW {
    static constexpr bool kBMN = false;
    static constexpr int kN = N;
    static constexpr int kP = P;
    float* R32;
    int64_t ldr;
    int b, j0, nsrc, i0, ni, Qn, nmb;
    __device__ bool skip_all() const { return false; }
    __device__ int units() const { return ni * Qn * nmb; }
    __device__ bool active(int) const { return true; }
    __device__ int nseg(int) const { return nsrc; }
    __device__ void decode(int u, int64_t& i, int& cn, int& mb) const
    {
        const int nx = ni * Qn, x = u % nx;
        mb = u / nx;
        i = i0 + x / Qn;
        cn = x % Qn;
    }
    __device__ Seg seg(int u, int q) const
    {
        int64_t i;
        int cn, mb;
        decode(u, i, cn, mb);
        const int64_t j = j0 + q;
        return Seg{mb * 128, (int)(j * b), (int)(tri_index(i, j) * 3 * b) + cn * N, 0, 0, b};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t t, W&& wait) const
    {
        int64_t i;
        int cn, mb;
        decode(u, i, cn, mb);
        float* dst = R32 + ((int64_t)mb * 128 + row) * ldr + i * b + cn * N;
        return epi_rows(dst, t, c0, N / 2, -1.f, false, N, wait);
    }
};

// Full covariance: cov (m x m, FP64, holding K_{Z*,Z*}) -= W W^T on lower
// 128-blocks, mirrored (128-wide units).
struct OpSyrkCov {
    static constexpr bool kBMN = false;
    static constexpr int kN = 128;
    static constexpr int kP = 3;
    double* cov;
    int64_t m;
    int kdim, nb;
    __device__ bool skip_all() const { return false; }
    __device__ int units() const { return nb * (nb + 1) / 2; }
    __device__ bool active(int) const { return true; }
    __device__ int nseg(int) const { return 1; }
    __device__ Seg seg(int u, int) const
    {
        int64_t a, c;
        tri_decode(u, a, c);
        return Seg{(int)a * 128, 0, (int)c * 128, 0, 0, kdim};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t t, W&& wait) const
    {
        int64_t a, c;
        tri_decode(u, a, c);
        const int64_t R = a * 128 + row;
        if (!wait()) return false;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tc::tmem_ld32(t + c0 + 32 * h, v);
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int cc = c0 + 32 * h + q;
                const int64_t Cg = c * 128 + cc;
                if (R >= m || Cg >= m || (a == c && cc > row)) continue;
                const double x = cov[R * m + Cg] - (double)v[q];
                cov[R * m + Cg] = x;
                cov[Cg * m + R] = x;
            }
        }
        return true;
    }
};

// Inverse for the gradient, finishing step: Z_tj = -U_tj Linv_tt^T (j < t), planes into ZP.
template <int N>
struct OpTrtriFin {
    static constexpr bool kBMN = false;
    static constexpr int kN = N;
    static constexpr int kP = 3;
    __nv_bfloat16* ZP;
    int b, t, Q, Qn;
    __device__ bool skip_all() const { return false; }
    __device__ int units() const { return t * Q * Qn; }
    __device__ bool active(int) const { return true; }
    __device__ int nseg(int) const { return 1; }
    __device__ Seg seg(int u, int) const
    {
        const int j = u / (Q * Qn), r = u % (Q * Qn), rb = r / Qn, cn = r % Qn;
        return Seg{j * 3 * b + rb * 128, 0, t * 3 * b + cn * N, 0, 0, (cn + 1) * N};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t tm, W&& wait) const
    {
        const int j = u / (Q * Qn), r = u % (Q * Qn), rb = r / Qn, cn = r % Qn;
        const int64_t bb = (int64_t)b * b;
        __nv_bfloat16* zp = ZP + tri_index(t, j) * 3 * bb + (int64_t)(rb * 128 + row) * b + cn * N;
        if (!wait()) return false;
#pragma unroll 1
        for (int h = 0; h < N / 2; h += 32) {
            float v[32];
            tc::tmem_ld32(tm + c0 + h, v);
            planes32(zp + c0 + h, bb, v, -1.f);
        }
        return true;
    }
};

// Inverse, accumulation: U_ij (+)= sum_{t in [max(t0, j), t1)} Z_tj L_it^T for
// the target tiles i in [i0, i0 + ni) (all >= t1), j in [0, nj), one
// k-segment per t.  A tile's first contribution (t == j, inside the range
// exactly when j >= t0) overwrites, later ones add.
template <int N>
struct OpTrtriAcc {
    static constexpr bool kBMN = false;
    static constexpr int kN = N;
    static constexpr int kP = 3;
    float* U32;
    int b, t0, t1, i0, ni, nj, Q, Qn;
    __device__ bool skip_all() const { return false; }
    __device__ int units() const { return ni * nj * Q * Qn; }
    __device__ bool active(int) const { return true; }
    __device__ void decode(int u, int64_t& i, int64_t& j, int& rb, int& cn) const
    {
        const int x = u / (Q * Qn);
        i = i0 + x / nj;
        j = x % nj;
        rb = (u % (Q * Qn)) / Qn;
        cn = u % Qn;
    }
    __device__ int nseg(int u) const
    {
        int64_t i, j;
        int rb, cn;
        decode(u, i, j, rb, cn);
        return t1 - (int)(j > t0 ? j : t0);
    }
    __device__ Seg seg(int u, int q) const
    {
        int64_t i, j;
        int rb, cn;
        decode(u, i, j, rb, cn);
        const int64_t t = (j > t0 ? j : t0) + q;
        return Seg{(int)(tri_index(t, j) * 3 * b) + rb * 128, 0, (int)(tri_index(i, t) * 3 * b) + cn * N, 0, 0, b};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t tm, W&& wait) const
    {
        int64_t i, j;
        int rb, cn;
        decode(u, i, j, rb, cn);
        float* dst = U32 + tri_index(i, j) * (int64_t)b * b + (int64_t)(rb * 128 + row) * b + cn * N;
        return epi_rows(dst, tm, c0, N / 2, 1.f, j >= t0, N, wait);
    }
};

// Inverse, K^{-1}_ij = sum_{t >= i} Z_ti Z_tj^T on lower tiles (FP32 out);
// in diagonal tiles only the column blocks up to the row's diagonal block.
template <int N>
struct OpLauum {
    static constexpr bool kBMN = false;
    static constexpr int kN = N;
    static constexpr int kP = 3;
    float* Kinv32;
    int b, T, Q, Qn;
    __device__ bool skip_all() const { return false; }
    __device__ int units() const { return T * (T + 1) / 2 * Q * Qn; }
    __device__ void decode(int u, int64_t& i, int64_t& j, int& rb, int& cn) const
    {
        tri_decode(u / (Q * Qn), i, j);
        rb = (u % (Q * Qn)) / Qn;
        cn = u % Qn;
    }
    __device__ bool active(int u) const
    {
        int64_t i, j;
        int rb, cn;
        decode(u, i, j, rb, cn);
        return !(i == j && cn * N > rb * 128);
    }
    __device__ int nseg(int u) const
    {
        int64_t i, j;
        int rb, cn;
        decode(u, i, j, rb, cn);
        return (int)(T - i);
    }
    __device__ Seg seg(int u, int q) const
    {
        int64_t i, j;
        int rb, cn;
        decode(u, i, j, rb, cn);
        const int64_t t = i + q;
        return Seg{(int)(tri_index(t, i) * 3 * b) + rb * 128, 0, (int)(tri_index(t, j) * 3 * b) + cn * N, 0,
                   q == 0 ? rb * 128 : 0, b};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t tm, W&& wait) const
    {
        int64_t i, j;
        int rb, cn;
        decode(u, i, j, rb, cn);
        float* dst = Kinv32 + tri_index(i, j) * (int64_t)b * b + (int64_t)(rb * 128 + row) * b + cn * N;
        const int limit = (i == j) ? (rb + 1) * 128 - cn * N : N;
        return epi_rows(dst, tm, c0, N / 2, 1.f, true, limit, wait);
    }
};

// Backward multi-RHS solve of the variance correction (x0^T = W L~^{-1}, NN
// form), super-block step: Y_I = S_I X_I with X_I[k][n] nonzero for k >= n,
// so the k range of a column unit starts at its first column.  FP32 Y_I over
// S_I (column block col0 .. of R32) and its planes into the same columns of
// planes (three planes of ldm x ldr: the W plane buffer).
template <int N, int P = 3>
struct OpBDiagSB {
    static constexpr bool kBMN = true;
    static constexpr int kN = N;
    static constexpr int kP = P;
    float* R32;
    __nv_bfloat16* planes;
    int64_t ldr, ldm;
    int col0, xrow0, B, Qn, nmb;
    __device__ bool skip_all() const { return false; }
    __device__ int units() const { return Qn * nmb; }
    __device__ bool active(int) const { return true; }
    __device__ int nseg(int) const { return 1; }
    __device__ Seg seg(int u, int) const
    {
        const int cn = u % Qn, mb = u / Qn;
        return Seg{mb * 128, 0, xrow0, cn * N, cn * N, B};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t t, W&& wait) const
    {
        const int cn = u % Qn, mb = u / Qn;
        const int64_t r = (int64_t)mb * 128 + row;
        float* dst = R32 + r * ldr + col0 + cn * N;
        __nv_bfloat16* yp = planes + r * ldr + col0 + cn * N;
        if (!wait()) return false;
#pragma unroll 1
        for (int h = 0; h < N / 2; h += 32) {
            float v[32];
            tc::tmem_ld32(t + c0 + h, v);
            row_store(dst + c0 + h, v, 0);
            planes32(yp + c0 + h, ldm * ldr, v);
        }
        return true;
    }
};

// Backward solve, update: S_j -= sum_{i in [i0, i0 + nsrc)} Y_i L_ij for the
// target tiles j in [j0, j0 + nj), all below i0 (NN form, L_ij[t][c]), one
// k-segment per source column.
template <int N, int P = 3>
struct OpBUpd {
    static constexpr bool kBMN = true;
    static constexpr int kN = N;
    static constexpr int kP = P;
    float* R32;
    int64_t ldr;
    int b, i0, nsrc, j0, nj, Qn, nmb;
    __device__ bool skip_all() const { return false; }
    __device__ int units() const { return nj * Qn * nmb; }
    __device__ bool active(int) const { return true; }
    __device__ int nseg(int) const { return nsrc; }
    __device__ void decode(int u, int64_t& j, int& cn, int& mb) const
    {
        const int nx = nj * Qn, x = u % nx;
        mb = u / nx;
        j = j0 + x / Qn;
        cn = x % Qn;
    }
    __device__ Seg seg(int u, int q) const
    {
        int64_t j;
        int cn, mb;
        decode(u, j, cn, mb);
        const int64_t i = i0 + q;
        return Seg{mb * 128, (int)(i * b), (int)(tri_index(i, j) * 3 * b), cn * N, 0, b};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t t, W&& wait) const
    {
        int64_t j;
        int cn, mb;
        decode(u, j, cn, mb);
        float* dst = R32 + ((int64_t)mb * 128 + row) * ldr + j * b + cn * N;
        return epi_rows(dst, t, c0, N / 2, -1.f, false, N, wait);
    }
};

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn_tg()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
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

// Three-plane BF16 operand (plane p of row r at row r + p * plane_rows of a
// rows x cols row-major array) as one TMA box per stage.  K-major (mn =
// false): dims {cols, rows - 2 plane_rows, 3}, box {32 k, box_rows, 3
// planes}, 64-byte swizzle.  MN-major B (mn = true, rows are k, n
// contiguous): dims {64 n, rows - 2 plane_rows, cols / 64, 3}, box {64 n,
// 32 k, box_rows / 64 column groups, 3 planes}, 128-byte swizzle, which lands
// as [plane][group][k][n].  The row extent stops two planes short of the
// array's end, so the plane offset of any in-range coordinate stays inside
// the allocation.  planes < 3 loads only the leading planes of each box.
bool map_tiles(CUtensorMap* map, const void* p, int64_t rows, int64_t cols, int64_t plane_rows, int box_rows,
               bool mn = false, int planes = 3)
{
    auto enc = encode_fn_tg();
    const int64_t ext = rows - 2 * plane_rows;
    if (!enc || ((uintptr_t)p & 15) || (cols * 2) % 16 || ext <= 0 || rows >= (1ll << 31) || (mn && cols % 64) ||
        planes < 1 || planes > 3)
        return false;
    cuuint32_t es[4] = {1, 1, 1, 1};
    if (!mn) {
        cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)ext, 3};
        cuuint64_t strides[2] = {(cuuint64_t)cols * 2, (cuuint64_t)(plane_rows * cols * 2)};
        cuuint32_t box[3] = {(cuuint32_t)TG_KS, (cuuint32_t)box_rows, (cuuint32_t)planes};
        return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(p), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    cuuint64_t dims[4] = {64, (cuuint64_t)ext, (cuuint64_t)(cols / 64), 3};
    cuuint64_t strides[3] = {(cuuint64_t)cols * 2, 128, (cuuint64_t)(plane_rows * cols * 2)};
    cuuint32_t box[4] = {64u, (cuuint32_t)TG_KS, (cuuint32_t)(box_rows / 64), (cuuint32_t)planes};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(p), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int g_num_sms = 0;

template <class Op>
bool launch(gp_t h, int phase, const CUtensorMap& mA, const CUtensorMap& mB, const Op& op, int units)
{
    static int done_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (done_dev != dev) {
        cudaFuncSetAttribute(k_tgemm<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TgCfg<Op::kN, Op::kP>::SMEM);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        done_dev = dev;
    }
    if (units <= 0) return true;
    int* err = tc_error_dev();
    if (!err) return false;
    const int grid = units < g_num_sms ? units : g_num_sms;
    constexpr int smem = TgCfg<Op::kN, Op::kP>::SMEM;
    GPK_LAUNCH(h, phase, k_tgemm<Op>, (unsigned)grid, TG_THREADS, smem, mA, mB, op, err);
    h->tc_pending = true;
    return true;
}

// Column units of the tile edge b: 256 wide where b allows it.
bool wide(gp_t h) { return h->b % 256 == 0; }

int64_t lp_rows(gp_t h) { return 3 * h->T * (h->T + 1) / 2 * h->b; }

template <int N>
bool panel_n(gp_t h, int64_t k)
{
    const int b = (int)h->b, T = (int)h->T;
    CUtensorMap mA, mB;
    if (!map_tiles(&mA, h->PA, 3 * (int64_t)(T > 1 ? T - 1 : 1) * b, b, b, 128) ||
        !map_tiles(&mB, h->LinvP, 3 * (int64_t)T * b, b, b, N))
        return false;
    const int tt = T - (int)k - 1;
    OpPanel<N> op{h->A32, h->LP, b, (int)k, tt, b / 128, b / N, (const unsigned long long*)h->info};
    return launch(h, GP_PH_TRSM, mA, mB, op, tt * (b / 128) * (b / N));
}

template <int N>
bool update_n(gp_t h, int k0, int nsrc, int j0, int w)
{
    const int b = (int)h->b, T = (int)h->T;
    CUtensorMap mA, mB;
    if (!map_tiles(&mA, h->LP, lp_rows(h), b, b, 128) || !map_tiles(&mB, h->LP, lp_rows(h), b, b, N)) return false;
    OpUpdate<N> op{h->A32, b, k0, nsrc, j0, w, T, b / 128, b / N, (const unsigned long long*)h->info};
    return launch(h, GP_PH_UPDATE, mA, mB, op, (w * (w - 1) / 2 + w * (T - j0 - w + 1)) * (b / 128) * (b / N));
}

// The super-block inverses' planes as a B operand: rows are X_I rows (I B ..),
// k (or n, MN-major) along X_I's columns.
bool map_sbx(gp_t h, CUtensorMap* m, int box_rows, bool mn, int planes)
{
    const int64_t SBb = GP_SOLVE_SB * h->b, TS = (h->T + GP_SOLVE_SB - 1) / GP_SOLVE_SB;
    return map_tiles(m, h->XsbP, 3 * TS * SBb, SBb, TS * SBb, box_rows, mn, planes);
}

template <int N, int P>
bool diag_w_sb_n(gp_t h, int phase, float* R, int64_t ldm, double* vpart, int64_t I)
{
    const int64_t b = h->b, SBb = GP_SOLVE_SB * b, t0 = I * GP_SOLVE_SB;
    const int64_t st = h->T - t0 < GP_SOLVE_SB ? h->T - t0 : GP_SOLVE_SB;
    CUtensorMap mA, mB;
    if (!map_tiles(&mA, h->RP, 3 * ldm, SBb, ldm, 128, false, P) || !map_sbx(h, &mB, N, false, P)) return false;
    OpDiagWSB<N, P> op{h->WP, R, vpart, h->Np, ldm, (int)(t0 * b), (int)(I * SBb), (int)(st * b / N), (int)(ldm / 128)};
    return launch(h, phase, mA, mB, op, op.Qn * op.nmb);
}

template <int N, int P>
bool diag_w_n(gp_t h, int phase, float* R, int64_t ldm, double* vpart, int64_t j)
{
    const int b = (int)h->b, T = (int)h->T;
    CUtensorMap mA, mB;
    if (!map_tiles(&mA, h->RP, 3 * ldm, b, ldm, 128, false, P) ||
        !map_tiles(&mB, h->LinvP, 3 * (int64_t)T * b, b, b, N, false, P))
        return false;
    OpDiagW<N, P> op{h->WP, R, vpart, h->Np, ldm, b, (int)j, b / N, (int)(ldm / 128)};
    return launch(h, phase, mA, mB, op, (b / N) * (int)(ldm / 128));
}

template <int N, int P>
bool upd_w_n(gp_t h, int phase, float* R, int64_t ldm, int j0, int nsrc, int i0, int ni)
{
    const int b = (int)h->b;
    CUtensorMap mA, mB;
    if (!map_tiles(&mA, h->WP, 3 * ldm, h->Np, ldm, 128, false, P) ||
        !map_tiles(&mB, h->LP, lp_rows(h), b, b, N, false, P))
        return false;
    OpUpdW<N, P> op{R, h->Np, b, j0, nsrc, i0, ni, b / N, (int)(ldm / 128)};
    return launch(h, phase, mA, mB, op, ni * (b / N) * (int)(ldm / 128));
}

template <int N>
bool trtri_fin_n(gp_t h, int64_t t)
{
    const int b = (int)h->b, T = (int)h->T;
    CUtensorMap mA, mB;
    if (!map_tiles(&mA, h->PA, 3 * (int64_t)(T > 1 ? T - 1 : 1) * b, b, b, 128) ||
        !map_tiles(&mB, h->LinvP, 3 * (int64_t)T * b, b, b, N))
        return false;
    OpTrtriFin<N> op{h->ZP, b, (int)t, b / 128, b / N};
    return launch(h, GP_PH_TRTRI, mA, mB, op, (int)t * (b / 128) * (b / N));
}

template <int N>
bool trtri_acc_n(gp_t h, int t0, int t1, int i0, int ni, int nj)
{
    const int b = (int)h->b;
    CUtensorMap mA, mB;
    if (!map_tiles(&mA, h->ZP, lp_rows(h), b, b, 128) || !map_tiles(&mB, h->LP, lp_rows(h), b, b, N)) return false;
    OpTrtriAcc<N> op{h->U32, b, t0, t1, i0, ni, nj, b / 128, b / N};
    return launch(h, GP_PH_TRTRI, mA, mB, op, ni * nj * (b / 128) * (b / N));
}

template <int N>
bool lauum_n(gp_t h)
{
    const int b = (int)h->b, T = (int)h->T;
    CUtensorMap mA, mB;
    if (!map_tiles(&mA, h->ZP, lp_rows(h), b, b, 128) || !map_tiles(&mB, h->ZP, lp_rows(h), b, b, N)) return false;
    OpLauum<N> op{h->Kinv32, b, T, b / 128, b / N};
    return launch(h, GP_PH_LAUUM, mA, mB, op, T * (T + 1) / 2 * (b / 128) * (b / N));
}

template <int N, int P>
bool bdiag_sb_n(gp_t h, int64_t ldm, int64_t I)
{
    const int64_t b = h->b, SBb = GP_SOLVE_SB * b, t0 = I * GP_SOLVE_SB;
    const int64_t st = h->T - t0 < GP_SOLVE_SB ? h->T - t0 : GP_SOLVE_SB;
    CUtensorMap mA, mB;
    if (!map_tiles(&mA, h->RP, 3 * ldm, SBb, ldm, 128, false, P) || !map_sbx(h, &mB, N, true, P)) return false;
    OpBDiagSB<N, P> op{h->R32,         h->WP,           h->Np, ldm, (int)(t0 * b), (int)(I * SBb), (int)(st * b),
                     (int)(st * b / N), (int)(ldm / 128)};
    return launch(h, GP_PH_BSOLVE, mA, mB, op, op.Qn * op.nmb);
}

template <int N, int P>
bool bupd_n(gp_t h, int64_t ldm, int i0, int nsrc, int j0, int nj)
{
    const int b = (int)h->b;
    CUtensorMap mA, mB;
    if (!map_tiles(&mA, h->WP, 3 * ldm, h->Np, ldm, 128, false, P) ||
        !map_tiles(&mB, h->LP, lp_rows(h), b, b, N, true, P))
        return false;
    OpBUpd<N, P> op{h->R32, h->Np, b, i0, nsrc, j0, nj, b / N, (int)(ldm / 128)};
    return launch(h, GP_PH_BSOLVE, mA, mB, op, nj * (b / N) * (int)(ldm / 128));
}

}  // namespace

bool tg_panel(gp_t h, int64_t k) { return wide(h) ? panel_n<256>(h, k) : panel_n<128>(h, k); }
bool tg_update(gp_t h, int k0, int nsrc, int j0, int w)
{
    return wide(h) ? update_n<256>(h, k0, nsrc, j0, w) : update_n<128>(h, k0, nsrc, j0, w);
}

// Sweep products with P operand planes: the 128- or 256-wide instantiation.
template <int P>
bool diag_w_sb_p(gp_t h, int phase, float* R, int64_t ldm, double* vpart, int64_t I)
{
    return wide(h) ? diag_w_sb_n<256, P>(h, phase, R, ldm, vpart, I) : diag_w_sb_n<128, P>(h, phase, R, ldm, vpart, I);
}
template <int P>
bool diag_w_p(gp_t h, int phase, float* R, int64_t ldm, double* vpart, int64_t j)
{
    return wide(h) ? diag_w_n<256, P>(h, phase, R, ldm, vpart, j) : diag_w_n<128, P>(h, phase, R, ldm, vpart, j);
}
template <int P>
bool upd_w_p(gp_t h, int phase, float* R, int64_t ldm, int j0, int nsrc, int i0, int ni)
{
    return wide(h) ? upd_w_n<256, P>(h, phase, R, ldm, j0, nsrc, i0, ni)
                   : upd_w_n<128, P>(h, phase, R, ldm, j0, nsrc, i0, ni);
}
template <int P>
bool bdiag_sb_p(gp_t h, int64_t ldm, int64_t I)
{
    return wide(h) ? bdiag_sb_n<256, P>(h, ldm, I) : bdiag_sb_n<128, P>(h, ldm, I);
}

template <int P>
bool bupd_p(gp_t h, int64_t ldm, int i0, int nsrc, int j0, int nj)
{
    return wide(h) ? bupd_n<256, P>(h, ldm, i0, nsrc, j0, nj) : bupd_n<128, P>(h, ldm, i0, nsrc, j0, nj);
}

bool tg_syrk_cov(gp_t h, int64_t m, int64_t ldm, double* cov)
{
    CUtensorMap mA;
    if (!map_tiles(&mA, h->WP, 3 * ldm, h->Np, ldm, 128)) return false;
    const int nb = (int)((m + 127) / 128);
    OpSyrkCov op{cov, m, (int)h->Np, nb};
    return launch(h, GP_PH_COV, mA, mA, op, nb * (nb + 1) / 2);
}

bool tg_trtri_fin(gp_t h, int64_t t) { return wide(h) ? trtri_fin_n<256>(h, t) : trtri_fin_n<128>(h, t); }
bool tg_trtri_acc(gp_t h, int t0, int t1, int i0, int ni, int nj)
{
    return wide(h) ? trtri_acc_n<256>(h, t0, t1, i0, ni, nj) : trtri_acc_n<128>(h, t0, t1, i0, ni, nj);
}
bool tg_lauum(gp_t h) { return wide(h) ? lauum_n<256>(h) : lauum_n<128>(h); }
bool tg_diag_w_sb(gp_t h, int phase, float* R, int64_t ldm, double* vpart, int64_t I, int planes)
{
    return planes == 2 ? diag_w_sb_p<2>(h, phase, R, ldm, vpart, I) : diag_w_sb_p<3>(h, phase, R, ldm, vpart, I);
}
bool tg_diag_w(gp_t h, int phase, float* R, int64_t ldm, double* vpart, int64_t j, int planes)
{
    return planes == 2 ? diag_w_p<2>(h, phase, R, ldm, vpart, j) : diag_w_p<3>(h, phase, R, ldm, vpart, j);
}
bool tg_upd_w(gp_t h, int phase, float* R, int64_t ldm, int j0, int nsrc, int i0, int ni, int planes)
{
    return planes == 2 ? upd_w_p<2>(h, phase, R, ldm, j0, nsrc, i0, ni)
                       : upd_w_p<3>(h, phase, R, ldm, j0, nsrc, i0, ni);
}
bool tg_bdiag_sb(gp_t h, int64_t ldm, int64_t I, int planes)
{
    return planes == 2 ? bdiag_sb_p<2>(h, ldm, I) : bdiag_sb_p<3>(h, ldm, I);
}

bool tg_bupd(gp_t h, int64_t ldm, int i0, int nsrc, int j0, int nj, int planes)
{
    return planes == 2 ? bupd_p<2>(h, ldm, i0, nsrc, j0, nj) : bupd_p<3>(h, ldm, i0, nsrc, j0, nj);
}

}  // namespace gpk
