// Split-BF16 ("bf16x6") block products of the mixed path on tcgen05.
//
// Every FP32 operand X is held as three BF16 planes X = X0 + X1 + X2 (round
// to nearest at each step); a product A B^T is taken as the six plane
// products Aa Bb^T with a + b <= 2, accumulated in FP32, which reproduces the
// FP32 product to about FP32 rounding.  One persistent kernel template,
// k_tgemm<Op>, runs all of them: a work unit is a 128 x 128 output block with
// one or more k-segments; Op names the operand tiles, the units and the
// epilogue.
//
// Roles (320 threads, one CTA per SM, grid = min(units, SMs)): warp 0 issues
// the TMA loads of a 32-k stage (three A planes and three B planes, six
// 128 x 32 tiles with 64-byte swizzle, 48 KB) into a four-stage ring; warp 1
// owns 256 TMEM columns
// (two 128-column accumulators, alternating between units) and issues the
// six plane MMAs per 16-k step; warps 2-9 run the epilogue of unit c while
// the MMAs of unit c+1 proceed: two warps per TMEM lane quarter, each thread
// one output row and 64 columns, its read-modify-write loads issued before it
// waits for the accumulator.  Waits are bounded
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
constexpr int TG_STAGES = 4;
constexpr int TG_KS = 32;                          // k per stage
constexpr int TG_PLANE = 128 * TG_KS * 2;          // bytes of one 128-row plane tile
constexpr int TG_STAGE_BYTES = 6 * TG_PLANE;
constexpr int TG_BAR_OFF = TG_STAGES * TG_STAGE_BYTES;
constexpr int TG_SMEM = 1024 + TG_BAR_OFF + 256;
constexpr uint32_t TG_IDESC = tc::idesc_bf16(128, 128);
constexpr uint32_t TG_IDESC_BMN = tc::idesc_bf16_bmn(128, 128);

// Operand coordinates of one k-segment: plane p of A is the 128-row box at
// map row a_row + p * a_ps, k-columns a_x + [k0, k1); likewise B when B is
// K-major.  An Op with kBMN set gives B as K x N with n contiguous (the NN
// form): plane p holds k rows b_row + p * b_ps + [k0, k1), n columns b_x +
// [0, 128), loaded as two 64-column boxes per stage.  k0 and k1 are
// multiples of 32.
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
    extern __shared__ unsigned char dyn[];
    if (op.skip_all()) return;
    unsigned char* base = dyn + ((1024 - (tc::su32(dyn) & 1023)) & 1023);
    const uint32_t sbase = tc::su32(base);
    const uint32_t bar = sbase + TG_BAR_OFF;   // full[2], empty[2], accf[2], acce[2], drain
    auto full = [&](int s) { return bar + 8 * s; };
    auto empty = [&](int s) { return bar + 8 * (TG_STAGES + s); };
    auto accf = [&](int a) { return bar + 8 * (2 * TG_STAGES + a); };
    auto acce = [&](int a) { return bar + 8 * (2 * TG_STAGES + 2 + a); };
    const uint32_t drain = bar + 8 * (2 * TG_STAGES + 4);
    uint32_t* tmem_slot = (uint32_t*)(base + TG_BAR_OFF + 8 * (2 * TG_STAGES + 5));
    volatile int* abort = (volatile int*)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TG_STAGES; ++s) {
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
    if (warp == 1) tc::tmem_alloc(tc::su32(tmem_slot), 256);
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
                        const int st = it % TG_STAGES, use = it / TG_STAGES;
                        if (use > 0 && !tc::mbar_wait(empty(st), (uint32_t)((use - 1) & 1), abort, err)) {
                            ok = false;
                            break;
                        }
                        const uint32_t dst = sbase + st * TG_STAGE_BYTES;
                        tc::mbar_expect_tx(full(st), TG_STAGE_BYTES);
#pragma unroll
                        for (int p = 0; p < 3; ++p) {
                            tc::tma_load_2d_hint(dst + p * TG_PLANE, &mapA, sg.a_x + k, sg.a_row + p * op.a_ps, full(st),
                                                 pol);
                            if (Op::kBMN) {
                                const uint32_t db = dst + (3 + p) * TG_PLANE;
                                tc::tma_load_2d_hint(db, &mapB, sg.b_x, sg.b_row + p * op.b_ps + k, full(st), pol);
                                tc::tma_load_2d_hint(db + TG_PLANE / 2, &mapB, sg.b_x + 64, sg.b_row + p * op.b_ps + k,
                                                     full(st), pol);
                            } else {
                                tc::tma_load_2d_hint(dst + (3 + p) * TG_PLANE, &mapB, sg.b_x + k,
                                                     sg.b_row + p * op.b_ps, full(st), pol);
                            }
                        }
                    }
                }
            }
            if (!ok)
                for (int q = it - 1; q >= 0 && q >= it - TG_STAGES; --q)
                    seg_wait_drain(full(q % TG_STAGES), (uint32_t)((q / TG_STAGES) & 1));
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
                const uint32_t d = tmem + (uint32_t)(a * 128);
                bool first = true;
                const int ns = op.nseg(u);
                for (int q = 0; q < ns && ok; ++q) {
                    const Seg sg = op.seg(u, q);
                    for (int k = sg.k0; k < sg.k1; k += TG_KS, ++it) {
                        const int st = it % TG_STAGES;
                        if (!tc::mbar_wait(full(st), (uint32_t)((it / TG_STAGES) & 1), abort, err)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after();
                        // stage descriptors once; planes are TG_PLANE apart (TG_PLANE >> 4 in the address
                        // field), a 16-k step adds 32 bytes (K-major) or 2048 bytes (MN-major B)
                        const uint32_t s0 = sbase + st * TG_STAGE_BYTES;
                        const uint64_t da = tc::desc_sw64(s0);
                        const uint64_t db = Op::kBMN ? tc::desc_mn32_sw128(s0 + 3 * TG_PLANE)
                                                     : tc::desc_sw64(s0 + 3 * TG_PLANE);
                        constexpr uint64_t pl = (uint64_t)(TG_PLANE >> 4);
                        constexpr uint64_t bstep = Op::kBMN ? (2048 >> 4) : 2;
                        constexpr uint32_t idesc = Op::kBMN ? TG_IDESC_BMN : TG_IDESC;
                        if (first) tc::mma_bf16(d, da, db, idesc, 0u);
                        else tc::mma_bf16_acc(d, da, db, idesc);
                        first = false;
#pragma unroll
                        for (int kk = 0; kk < TG_KS / 16; ++kk)
#pragma unroll
                            for (int qa = 0; qa < 3; ++qa)
#pragma unroll
                                for (int qb = 0; qa + qb < 3; ++qb) {
                                    if (kk == 0 && qa == 0 && qb == 0) continue;
                                    tc::mma_bf16_acc(d, da + qa * pl + 2 * kk, db + qb * pl + bstep * kk, idesc);
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
        const int wq = warp & 3, row = wq * 32 + lane, c0 = ((warp - 2) >> 2) * 64;
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
            if (!op.epilogue(u, row, c0, tmem + lrow + (uint32_t)(a * 128), wait)) break;
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
        tc::tmem_dealloc(tmem, 256);
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

// ---------------------------------------------------------------- operations
// All tile stores are b x b row-major; LP, ZP: three planes per lower tile
// (tile t at rows 3 t b of the plane map); LinvP: three planes per diagonal
// tile; PA: three planes per panel slot.

// Cholesky panel: L_ik = A_ik Linv_kk^T, k-range of Linv_kk's lower 128-block
// column; FP32 L_ik over A_ik and its planes into LP.
struct OpPanel {
    static constexpr bool kBMN = false;
    float* A32;
    __nv_bfloat16* LP;
    int b, k, tt, Q;
    int a_ps, b_ps;
    const unsigned long long* info;
    __device__ bool skip_all() const { return failed(info); }
    __device__ int units() const { return tt * Q * Q; }
    __device__ bool active(int) const { return true; }
    __device__ int nseg(int) const { return 1; }
    __device__ Seg seg(int u, int) const
    {
        const int y = u / (Q * Q), r = u % (Q * Q), rb = r / Q, cb = r % Q;
        return Seg{y * 3 * b + rb * 128, 0, k * 3 * b + cb * 128, 0, 0, (cb + 1) * 128};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t t, W&& wait) const
    {
        const int y = u / (Q * Q), r = u % (Q * Q), rb = r / Q, cb = r % Q;
        const int64_t i = k + 1 + y, bb = (int64_t)b * b;
        const int64_t off = (int64_t)(rb * 128 + row) * b + cb * 128 + c0;
        float* dst = A32 + tri_index(i, k) * bb + off;
        __nv_bfloat16* lp = LP + 3 * tri_index(i, k) * bb + off;
        if (!wait()) return false;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tc::tmem_ld32(t + c0 + 32 * h, v);
            row_store(dst, v, h);
            planes32(lp + 32 * h, bb, v);
        }
        return true;
    }
};

// Trailing update: A_ij -= L_ik L_jk^T for k < j <= i (lower 128-blocks of diagonal tiles).
struct OpUpdate {
    static constexpr bool kBMN = false;
    float* A32;
    int b, k, tt, Q;
    int a_ps, b_ps;
    const unsigned long long* info;
    __device__ bool skip_all() const { return failed(info); }
    __device__ int units() const { return tt * (tt + 1) / 2 * Q * Q; }
    __device__ void decode(int u, int64_t& i, int64_t& j, int& rb, int& cb) const
    {
        int64_t ii, jj;
        tri_decode(u / (Q * Q), ii, jj);
        i = k + 1 + ii;
        j = k + 1 + jj;
        rb = (u % (Q * Q)) / Q;
        cb = u % Q;
    }
    __device__ bool active(int u) const
    {
        int64_t i, j;
        int rb, cb;
        decode(u, i, j, rb, cb);
        return !(i == j && cb > rb);
    }
    __device__ int nseg(int) const { return 1; }
    __device__ Seg seg(int u, int) const
    {
        int64_t i, j;
        int rb, cb;
        decode(u, i, j, rb, cb);
        return Seg{(int)(tri_index(i, k) * 3 * b) + rb * 128, 0, (int)(tri_index(j, k) * 3 * b) + cb * 128, 0, 0, b};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t t, W&& wait) const
    {
        int64_t i, j;
        int rb, cb;
        decode(u, i, j, rb, cb);
        float* dst = A32 + tri_index(i, j) * (int64_t)b * b + (int64_t)(rb * 128 + row) * b + cb * 128 + c0;
        Row64 cur;
        row_load(cur, dst);
        if (!wait()) return false;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tc::tmem_ld32(t + c0 + 32 * h, v);
            row_axpy(dst, cur, v, h, -1.f);
        }
        return true;
    }
};

// Forward multi-RHS solve, diagonal step: W_j = R_j Linv_jj^T; planes of W_j
// into WP, FP32 W_j over R_j, FP64 row sums of W_j^2 into vpart.
struct OpDiagW {
    static constexpr bool kBMN = false;
    __nv_bfloat16* WP;
    float* Wout;
    double* vpart;
    int64_t ldw, ldm;
    int b, j, Q, nmb;
    int a_ps, b_ps;
    __device__ bool skip_all() const { return false; }
    __device__ int units() const { return Q * nmb; }
    __device__ bool active(int) const { return true; }
    __device__ int nseg(int) const { return 1; }
    __device__ Seg seg(int u, int) const
    {
        const int cb = u % Q, mb = u / Q;
        return Seg{mb * 128, 0, j * 3 * b + cb * 128, 0, 0, (cb + 1) * 128};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t t, W&& wait) const
    {
        const int cb = u % Q, mb = u / Q;
        const int64_t r = (int64_t)mb * 128 + row;
        const int64_t o = r * ldw + (int64_t)j * b + cb * 128 + c0;
        if (!wait()) return false;
        double sq = 0.0;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tc::tmem_ld32(t + c0 + 32 * h, v);
            planes32(WP + o + 32 * h, ldm * ldw, v);
            row_store(Wout + o, v, h);
#pragma unroll
            for (int q = 0; q < 32; ++q) sq += (double)v[q] * v[q];
        }
        vpart[(((int64_t)j * b + cb * 128 + c0) / 64) * ldm + r] = sq;   // one slot per 64 columns
        return true;
    }
};

// Forward multi-RHS solve, update: R_i -= W_j L_ij^T for all tiles i > j.
struct OpUpdW {
    static constexpr bool kBMN = false;
    float* R32;
    int64_t ldr;
    int b, j, T, Q, nmb;
    int a_ps, b_ps;
    __device__ bool skip_all() const { return false; }
    __device__ int units() const { return (T - j - 1) * Q * nmb; }
    __device__ bool active(int) const { return true; }
    __device__ int nseg(int) const { return 1; }
    __device__ Seg seg(int u, int) const
    {
        const int nx = (T - j - 1) * Q, x = u % nx, mb = u / nx;
        const int64_t i = j + 1 + x / Q;
        const int cb = x % Q;
        return Seg{mb * 128, j * b, (int)(tri_index(i, j) * 3 * b) + cb * 128, 0, 0, b};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t t, W&& wait) const
    {
        const int nx = (T - j - 1) * Q, x = u % nx, mb = u / nx;
        const int64_t i = j + 1 + x / Q;
        const int cb = x % Q;
        float* dst = R32 + ((int64_t)mb * 128 + row) * ldr + i * b + cb * 128 + c0;
        Row64 cur;
        row_load(cur, dst);
        if (!wait()) return false;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tc::tmem_ld32(t + c0 + 32 * h, v);
            row_axpy(dst, cur, v, h, -1.f);
        }
        return true;
    }
};

// Full covariance: cov (m x m, FP64, holding K_{Z*,Z*}) -= W W^T on lower 128-blocks, mirrored.
struct OpSyrkCov {
    static constexpr bool kBMN = false;
    double* cov;
    int64_t m;
    int kdim, nb;
    int a_ps, b_ps;
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
                const int64_t C = c * 128 + cc;
                if (R >= m || C >= m || (a == c && cc > row)) continue;
                const double x = cov[R * m + C] - (double)v[q];
                cov[R * m + C] = x;
                cov[C * m + R] = x;
            }
        }
        return true;
    }
};

// Inverse for the gradient, finishing step: Z_tj = -U_tj Linv_tt^T (j < t), planes into ZP.
struct OpTrtriFin {
    static constexpr bool kBMN = false;
    __nv_bfloat16* ZP;
    int b, t, Q;
    int a_ps, b_ps;
    __device__ bool skip_all() const { return false; }
    __device__ int units() const { return t * Q * Q; }
    __device__ bool active(int) const { return true; }
    __device__ int nseg(int) const { return 1; }
    __device__ Seg seg(int u, int) const
    {
        const int j = u / (Q * Q), r = u % (Q * Q), rb = r / Q, cb = r % Q;
        return Seg{j * 3 * b + rb * 128, 0, t * 3 * b + cb * 128, 0, 0, (cb + 1) * 128};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t tm, W&& wait) const
    {
        const int j = u / (Q * Q), r = u % (Q * Q), rb = r / Q, cb = r % Q;
        const int64_t bb = (int64_t)b * b;
        __nv_bfloat16* zp = ZP + tri_index(t, j) * 3 * bb + (int64_t)(rb * 128 + row) * b + cb * 128 + c0;
        if (!wait()) return false;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tc::tmem_ld32(tm + c0 + 32 * h, v);
            planes32(zp + 32 * h, bb, v, -1.f);
        }
        return true;
    }
};

// Inverse, accumulation step: U_ij (+)= Z_tj L_it^T for i > t >= j; t == j overwrites.
struct OpTrtriAcc {
    static constexpr bool kBMN = false;
    float* U32;
    int b, t, T, Q;
    int a_ps, b_ps;
    __device__ bool skip_all() const { return false; }
    __device__ int units() const { return (T - t - 1) * (t + 1) * Q * Q; }
    __device__ bool active(int) const { return true; }
    __device__ int nseg(int) const { return 1; }
    __device__ void decode(int u, int64_t& i, int64_t& j, int& rb, int& cb) const
    {
        const int x = u / (Q * Q);
        i = t + 1 + x / (t + 1);
        j = x % (t + 1);
        rb = (u % (Q * Q)) / Q;
        cb = u % Q;
    }
    __device__ Seg seg(int u, int) const
    {
        int64_t i, j;
        int rb, cb;
        decode(u, i, j, rb, cb);
        return Seg{(int)(tri_index(t, j) * 3 * b) + rb * 128, 0, (int)(tri_index(i, t) * 3 * b) + cb * 128, 0, 0, b};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t tm, W&& wait) const
    {
        int64_t i, j;
        int rb, cb;
        decode(u, i, j, rb, cb);
        float* dst = U32 + tri_index(i, j) * (int64_t)b * b + (int64_t)(rb * 128 + row) * b + cb * 128 + c0;
        const bool first = (t == j);
        Row64 cur;
        if (!first) row_load(cur, dst);
        if (!wait()) return false;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tc::tmem_ld32(tm + c0 + 32 * h, v);
            if (first) row_store(dst, v, h);
            else row_axpy(dst, cur, v, h, 1.f);
        }
        return true;
    }
};

// Inverse, K^{-1}_ij = sum_{t >= i} Z_ti Z_tj^T on lower tiles (FP32 out).
struct OpLauum {
    static constexpr bool kBMN = false;
    float* Kinv32;
    int b, T, Q;
    int a_ps, b_ps;
    __device__ bool skip_all() const { return false; }
    __device__ int units() const { return T * (T + 1) / 2 * Q * Q; }
    __device__ void decode(int u, int64_t& i, int64_t& j, int& rb, int& cb) const
    {
        tri_decode(u / (Q * Q), i, j);
        rb = (u % (Q * Q)) / Q;
        cb = u % Q;
    }
    __device__ bool active(int u) const
    {
        int64_t i, j;
        int rb, cb;
        decode(u, i, j, rb, cb);
        return !(i == j && cb > rb);
    }
    __device__ int nseg(int u) const
    {
        int64_t i, j;
        int rb, cb;
        decode(u, i, j, rb, cb);
        return (int)(T - i);
    }
    __device__ Seg seg(int u, int q) const
    {
        int64_t i, j;
        int rb, cb;
        decode(u, i, j, rb, cb);
        const int64_t t = i + q;
        return Seg{(int)(tri_index(t, i) * 3 * b) + rb * 128, 0, (int)(tri_index(t, j) * 3 * b) + cb * 128, 0,
                   q == 0 ? rb * 128 : 0, b};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t tm, W&& wait) const
    {
        int64_t i, j;
        int rb, cb;
        decode(u, i, j, rb, cb);
        float* dst = Kinv32 + tri_index(i, j) * (int64_t)b * b + (int64_t)(rb * 128 + row) * b + cb * 128 + c0;
        if (!wait()) return false;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tc::tmem_ld32(tm + c0 + 32 * h, v);
            row_store(dst, v, h);
        }
        return true;
    }
};

// Backward multi-RHS solve of the variance correction (x0^T = W L~^{-1}, NN form).
// Diagonal step: Y_i = S_i Linv_ii, Linv_ii[t][c] nonzero for t >= c, so the
// k-range of output column block cb starts at cb * 128.  FP32 Y_i over S_i
// (column block i of R32) and its planes into YP (3 x ldm x b).
struct OpBDiag {
    static constexpr bool kBMN = true;
    float* R32;
    __nv_bfloat16* YP;
    int64_t ldr, ldm;
    int b, i, Q, nmb;
    int a_ps, b_ps;
    __device__ bool skip_all() const { return false; }
    __device__ int units() const { return Q * nmb; }
    __device__ bool active(int) const { return true; }
    __device__ int nseg(int) const { return 1; }
    __device__ Seg seg(int u, int) const
    {
        const int cb = u % Q, mb = u / Q;
        return Seg{mb * 128, 0, i * 3 * b, cb * 128, cb * 128, b};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t t, W&& wait) const
    {
        const int cb = u % Q, mb = u / Q;
        const int64_t r = (int64_t)mb * 128 + row;
        float* dst = R32 + r * ldr + (int64_t)i * b + cb * 128 + c0;
        __nv_bfloat16* yp = YP + r * b + cb * 128 + c0;
        if (!wait()) return false;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tc::tmem_ld32(t + c0 + 32 * h, v);
            row_store(dst, v, h);
            planes32(yp + 32 * h, ldm * b, v);
        }
        return true;
    }
};

// Backward solve, update: S_j -= Y_i L_ij for all j < i (NN form, L_ij[t][c]).
struct OpBUpd {
    static constexpr bool kBMN = true;
    float* R32;
    int64_t ldr;
    int b, i, Q, nmb;
    int a_ps, b_ps;
    __device__ bool skip_all() const { return false; }
    __device__ int units() const { return i * Q * nmb; }
    __device__ bool active(int) const { return true; }
    __device__ int nseg(int) const { return 1; }
    __device__ Seg seg(int u, int) const
    {
        const int nx = i * Q, x = u % nx, mb = u / nx;
        const int64_t j = x / Q;
        const int cb = x % Q;
        return Seg{mb * 128, 0, (int)(tri_index(i, j) * 3 * b), cb * 128, 0, b};
    }
    template <class W>
    __device__ bool epilogue(int u, int row, int c0, uint32_t t, W&& wait) const
    {
        const int nx = i * Q, x = u % nx, mb = u / nx;
        const int64_t j = x / Q;
        const int cb = x % Q;
        float* dst = R32 + ((int64_t)mb * 128 + row) * ldr + j * b + cb * 128 + c0;
        Row64 cur;
        row_load(cur, dst);
        if (!wait()) return false;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tc::tmem_ld32(t + c0 + 32 * h, v);
            row_axpy(dst, cur, v, h, -1.f);
        }
        return true;
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

// Row-major BF16 matrix (rows x cols, row stride cols) as TMA boxes: K-major
// operands as {32 k, 128 rows} with 64-byte swizzle (mn = false), an MN-major
// B as {64 n, 32 k rows} with 128-byte swizzle (mn = true).
bool map_tiles(CUtensorMap* map, const void* p, int64_t rows, int64_t cols, bool mn = false)
{
    auto enc = encode_fn_tg();
    if (!enc || ((uintptr_t)p & 15) || (cols * 2) % 16 || rows >= (1ll << 31)) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {mn ? 64u : (cuuint32_t)TG_KS, mn ? (cuuint32_t)TG_KS : 128u}, es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(p), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, mn ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int g_num_sms = 0;

template <class Op>
bool launch(gp_t h, int phase, const CUtensorMap& mA, const CUtensorMap& mB, const Op& op, int units)
{
    static int done_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (done_dev != dev) {
        cudaFuncSetAttribute(k_tgemm<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, TG_SMEM);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        done_dev = dev;
    }
    if (units <= 0) return true;
    int* err = tc_error_dev();
    if (!err) return false;
    const int grid = units < g_num_sms ? units : g_num_sms;
    GPK_LAUNCH(h, phase, k_tgemm<Op>, (unsigned)grid, TG_THREADS, TG_SMEM, mA, mB, op, err);
    h->tc_pending = true;
    return true;
}

}  // namespace

bool tg_panel(gp_t h, int64_t k)
{
    const int b = (int)h->b, T = (int)h->T, Q = b / 128;
    CUtensorMap mA, mB;
    if (!map_tiles(&mA, h->PA, 3 * (int64_t)(T > 1 ? T - 1 : 1) * b, b) || !map_tiles(&mB, h->LinvP, 3 * (int64_t)T * b, b))
        return false;
    const int tt = T - (int)k - 1;
    OpPanel op{h->A32, h->LP, b, (int)k, tt, Q, b, b, (const unsigned long long*)h->info};
    return launch(h, GP_PH_TRSM, mA, mB, op, tt * Q * Q);
}

bool tg_update(gp_t h, int64_t k)
{
    const int b = (int)h->b, T = (int)h->T, Q = b / 128;
    CUtensorMap mA;
    if (!map_tiles(&mA, h->LP, 3 * (int64_t)T * (T + 1) / 2 * b, b)) return false;
    const int tt = T - (int)k - 1;
    OpUpdate op{h->A32, b, (int)k, tt, Q, b, b, (const unsigned long long*)h->info};
    return launch(h, GP_PH_UPDATE, mA, mA, op, tt * (tt + 1) / 2 * Q * Q);
}

bool tg_diag_w(gp_t h, int phase, float* R, int64_t ldm, double* vpart, int64_t j)
{
    const int b = (int)h->b, T = (int)h->T, Q = b / 128;
    CUtensorMap mA, mB;
    if (!map_tiles(&mA, h->RP, 3 * ldm, b) || !map_tiles(&mB, h->LinvP, 3 * (int64_t)T * b, b)) return false;
    OpDiagW op{h->WP, R, vpart, h->Np, ldm, b, (int)j, Q, (int)(ldm / 128), (int)ldm, b};
    return launch(h, phase, mA, mB, op, Q * (int)(ldm / 128));
}

bool tg_upd_w(gp_t h, int phase, float* R, int64_t ldm, int64_t j)
{
    const int b = (int)h->b, T = (int)h->T, Q = b / 128;
    CUtensorMap mA, mB;
    if (!map_tiles(&mA, h->WP, 3 * ldm, h->Np) || !map_tiles(&mB, h->LP, 3 * (int64_t)T * (T + 1) / 2 * b, b))
        return false;
    OpUpdW op{R, h->Np, b, (int)j, T, Q, (int)(ldm / 128), (int)ldm, b};
    return launch(h, phase, mA, mB, op, (T - (int)j - 1) * Q * (int)(ldm / 128));
}

bool tg_syrk_cov(gp_t h, int64_t m, int64_t ldm, double* cov)
{
    CUtensorMap mA;
    if (!map_tiles(&mA, h->WP, 3 * ldm, h->Np)) return false;
    const int nb = (int)((m + 127) / 128);
    OpSyrkCov op{cov, m, (int)h->Np, nb, (int)ldm, (int)ldm};
    return launch(h, GP_PH_COV, mA, mA, op, nb * (nb + 1) / 2);
}

bool tg_trtri_fin(gp_t h, int64_t t)
{
    const int b = (int)h->b, T = (int)h->T, Q = b / 128;
    CUtensorMap mA, mB;
    if (!map_tiles(&mA, h->PA, 3 * (int64_t)(T > 1 ? T - 1 : 1) * b, b) || !map_tiles(&mB, h->LinvP, 3 * (int64_t)T * b, b))
        return false;
    OpTrtriFin op{h->ZP, b, (int)t, Q, b, b};
    return launch(h, GP_PH_TRTRI, mA, mB, op, (int)t * Q * Q);
}

bool tg_trtri_acc(gp_t h, int64_t t)
{
    const int b = (int)h->b, T = (int)h->T, Q = b / 128;
    CUtensorMap mA, mB;
    const int64_t rows = 3 * (int64_t)T * (T + 1) / 2 * b;
    if (!map_tiles(&mA, h->ZP, rows, b) || !map_tiles(&mB, h->LP, rows, b)) return false;
    OpTrtriAcc op{h->U32, b, (int)t, T, Q, b, b};
    return launch(h, GP_PH_TRTRI, mA, mB, op, (T - (int)t - 1) * ((int)t + 1) * Q * Q);
}

bool tg_lauum(gp_t h)
{
    const int b = (int)h->b, T = (int)h->T, Q = b / 128;
    CUtensorMap mA;
    if (!map_tiles(&mA, h->ZP, 3 * (int64_t)T * (T + 1) / 2 * b, b)) return false;
    OpLauum op{h->Kinv32, b, T, Q, b, b};
    return launch(h, GP_PH_LAUUM, mA, mA, op, T * (T + 1) / 2 * Q * Q);
}

bool tg_bdiag(gp_t h, int64_t ldm, int64_t i)
{
    const int b = (int)h->b, T = (int)h->T, Q = b / 128;
    CUtensorMap mA, mB;
    if (!map_tiles(&mA, h->RP, 3 * ldm, b) || !map_tiles(&mB, h->LinvP, 3 * (int64_t)T * b, b, true)) return false;
    OpBDiag op{h->R32, h->YP, h->Np, ldm, b, (int)i, Q, (int)(ldm / 128), (int)ldm, b};
    return launch(h, GP_PH_BSOLVE, mA, mB, op, Q * (int)(ldm / 128));
}

bool tg_bupd(gp_t h, int64_t ldm, int64_t i)
{
    const int b = (int)h->b, T = (int)h->T, Q = b / 128;
    CUtensorMap mA, mB;
    if (!map_tiles(&mA, h->YP, 3 * ldm, b) || !map_tiles(&mB, h->LP, 3 * (int64_t)T * (T + 1) / 2 * b, b, true))
        return false;
    OpBUpd op{h->R32, h->Np, b, (int)i, Q, (int)(ldm / 128), (int)ldm, b};
    return launch(h, GP_PH_BSOLVE, mA, mB, op, (int)i * Q * (int)(ldm / 128));
}

}  // namespace gpk
