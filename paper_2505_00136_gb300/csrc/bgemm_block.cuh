// FP32-accurate 128x128 block product from split-BF16 operands on the BF16
// tensor pipe (mma.sync.m16n8k16, FP32 accumulation).
//
// Each FP32 operand value v is stored as three BF16 "planes" hi, mid, lo with
// hi = bf16(v), mid = bf16(v - hi), lo = bf16(v - hi - mid), so that
// hi + mid + lo carries v's 24-bit significand.  The block product keeps the
// six plane products whose order is at most 2^-16 below the leading one,
//
//   acc += A_hi B_hi^T + A_hi B_mid^T + A_mid B_hi^T
//        + A_hi B_lo^T + A_mid B_mid^T + A_lo B_hi^T,
//
// which matches an FP32 product to about 2^-24 relative per term.
//
// Operands are K-contiguous ("NT" form): element (row, k) of plane q is at
// p[q * ps + row * ld + k], ld and k multiples of 8.  Rows at or beyond
// `rows` read as zero.  (ke - kb) must be a multiple of 32.
//
// One CTA of 256 threads (8 warps, 2 x 4) owns a 128 x 128 block; warp
// (wm, wn) computes rows wm*64..+64, columns wn*32..+32.  Stages of 32 k are
// double-buffered in shared memory through cp.async; rows are padded to 40
// BF16 (80 bytes) so ldmatrix reads are free of bank conflicts.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace gpk {

struct BView {
    const __nv_bfloat16* p;
    int64_t ld, ps;
    int rows;
};

struct BAcc {
    float c[4][4][4];   // [m16 tile][n8 tile][fragment]
};

constexpr int BG_KS = 32;                     // k per stage
constexpr int BG_LD = 40;                     // padded row length (bf16)
constexpr int BG_ROWS = 128;
constexpr int BG_PLANE = BG_ROWS * BG_LD;     // bf16 per plane per operand per stage
constexpr int BG_STAGE = 2 * 3 * BG_PLANE;    // A and B, 3 planes
constexpr int BG_SMEM_BYTES = 2 * BG_STAGE * 2;

__device__ __forceinline__ void bacc_zero(BAcc& a)
{
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) a.c[i][j][e] = 0.f;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid)
{
    const int bytes = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Issues the cp.async copies of one 128 x 32 stage (3 planes) of view v.
__device__ __forceinline__ void bg_stage_load(const BView& v, int64_t k0, __nv_bfloat16* s)
{
    // 3 planes x 128 rows x 4 chunks of 8 bf16 = 1536 chunks; 6 per thread
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        int idx = threadIdx.x + q * 256;
        int plane = idx >> 9, rem = idx & 511;
        int r = rem >> 2, ch = rem & 3;
        bool ok = r < v.rows;
        const __nv_bfloat16* src = v.p + plane * v.ps + (int64_t)(ok ? r : 0) * v.ld + k0 + ch * 8;
        cp_async16(s + plane * BG_PLANE + r * BG_LD + ch * 8, src, ok);
    }
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&d)[4], const __nv_bfloat16* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// acc += sum of the six plane products over k in [kb, ke).  smem: BG_SMEM_BYTES.
// Starts and ends with a CTA barrier.
static __device__ __forceinline__ void bgemm_acc(BAcc& acc, const BView& A, const BView& B, int64_t kb, int64_t ke,
                          __nv_bfloat16* smem)
{
    __syncthreads();
    const int nst = (int)((ke - kb) / BG_KS);
    if (nst <= 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp >> 2, wn = warp & 3;
    const int lq = lane >> 3, lr = lane & 7;
    bg_stage_load(A, kb, smem);
    bg_stage_load(B, kb, smem + 3 * BG_PLANE);
    cp_async_commit();
    for (int s = 0; s < nst; ++s) {
        __nv_bfloat16* cur = smem + (s & 1) * BG_STAGE;
        cp_async_wait_all();
        __syncthreads();
        if (s + 1 < nst) {
            __nv_bfloat16* nxt = smem + ((s + 1) & 1) * BG_STAGE;
            bg_stage_load(A, kb + (int64_t)(s + 1) * BG_KS, nxt);
            bg_stage_load(B, kb + (int64_t)(s + 1) * BG_KS, nxt + 3 * BG_PLANE);
            cp_async_commit();
        }
        const __nv_bfloat16* As = cur;
        const __nv_bfloat16* Bs = cur + 3 * BG_PLANE;
#pragma unroll
        for (int kk = 0; kk < BG_KS; kk += 16) {
            uint32_t bf[3][4][2];
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int np = 0; np < 2; ++np) {
                    uint32_t d[4];
                    const int n0 = wn * 32 + np * 16;
                    ldsm_x4(d, Bs + q * BG_PLANE + (n0 + lr + (lq >> 1) * 8) * BG_LD + kk + (lq & 1) * 8);
                    bf[q][np * 2][0] = d[0];
                    bf[q][np * 2][1] = d[1];
                    bf[q][np * 2 + 1][0] = d[2];
                    bf[q][np * 2 + 1][1] = d[3];
                }
#pragma unroll
            for (int qa = 0; qa < 3; ++qa) {
#pragma unroll
                for (int mt = 0; mt < 4; ++mt) {
                    uint32_t af[4];
                    const int m0 = wm * 64 + mt * 16;
                    ldsm_x4(af, As + qa * BG_PLANE + (m0 + lr + (lq & 1) * 8) * BG_LD + kk + (lq >> 1) * 8);
#pragma unroll
                    for (int qb = 0; qb + qa < 3; ++qb)
#pragma unroll
                        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc.c[mt][nt], af, bf[qb][nt][0], bf[qb][nt][1]);
                }
            }
        }
    }
    __syncthreads();
}

// "NN" form: B is stored k-major, element (k, col) of plane q at
// p[q * ps + k * ld + col]; `rows` bounds the columns.  Fragments come from
// ldmatrix.trans on a [k][col] shared-memory layout (rows of 136 BF16).
constexpr int BN_LD = 136;
constexpr int BN_PLANE = BG_KS * BN_LD;            // bf16 per plane per stage (B, NN form)
constexpr int BN_STAGE = 3 * BG_PLANE + 3 * BN_PLANE;
constexpr int BN_SMEM_BYTES = 2 * BN_STAGE * 2;

__device__ __forceinline__ void bn_stage_load(const BView& v, int64_t k0, __nv_bfloat16* s)
{
    // 3 planes x 32 k-rows x 16 chunks of 8 columns = 1536 chunks; 6 per thread
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        int idx = threadIdx.x + q * 256;
        int plane = idx >> 9, rem = idx & 511;
        int kr = rem >> 4, ch = rem & 15;
        bool ok = ch * 8 < v.rows;
        const __nv_bfloat16* src = v.p + plane * v.ps + (k0 + kr) * v.ld + (ok ? ch * 8 : 0);
        cp_async16(s + plane * BN_PLANE + kr * BN_LD + ch * 8, src, ok);
    }
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&d)[4], const __nv_bfloat16* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3])
                 : "r"(smem_u32(p)));
}

// acc += A B over k in [kb, ke), A in NT form (rows x k), B in NN form (k x cols).
// smem: BN_SMEM_BYTES.  Starts and ends with a CTA barrier.
static __device__ __forceinline__ void bgemm_acc_nn(BAcc& acc, const BView& A, const BView& B, int64_t kb,
                                                     int64_t ke, __nv_bfloat16* smem)
{
    __syncthreads();
    const int nst = (int)((ke - kb) / BG_KS);
    if (nst <= 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp >> 2, wn = warp & 3;
    const int lq = lane >> 3, lr = lane & 7;
    bg_stage_load(A, kb, smem);
    bn_stage_load(B, kb, smem + 3 * BG_PLANE);
    cp_async_commit();
    for (int s = 0; s < nst; ++s) {
        __nv_bfloat16* cur = smem + (s & 1) * BN_STAGE;
        cp_async_wait_all();
        __syncthreads();
        if (s + 1 < nst) {
            __nv_bfloat16* nxt = smem + ((s + 1) & 1) * BN_STAGE;
            bg_stage_load(A, kb + (int64_t)(s + 1) * BG_KS, nxt);
            bn_stage_load(B, kb + (int64_t)(s + 1) * BG_KS, nxt + 3 * BG_PLANE);
            cp_async_commit();
        }
        const __nv_bfloat16* As = cur;
        const __nv_bfloat16* Bs = cur + 3 * BG_PLANE;
#pragma unroll
        for (int kk = 0; kk < BG_KS; kk += 16) {
            uint32_t bf[3][4][2];
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int np = 0; np < 2; ++np) {
                    uint32_t d[4];
                    const int n0 = wn * 32 + np * 16;
                    ldsm_x4_t(d, Bs + q * BN_PLANE + (kk + (lq & 1) * 8 + lr) * BN_LD + n0 + (lq >> 1) * 8);
                    bf[q][np * 2][0] = d[0];
                    bf[q][np * 2][1] = d[1];
                    bf[q][np * 2 + 1][0] = d[2];
                    bf[q][np * 2 + 1][1] = d[3];
                }
#pragma unroll
            for (int qa = 0; qa < 3; ++qa) {
#pragma unroll
                for (int mt = 0; mt < 4; ++mt) {
                    uint32_t af[4];
                    const int m0 = wm * 64 + mt * 16;
                    ldsm_x4(af, As + qa * BG_PLANE + (m0 + lr + (lq & 1) * 8) * BG_LD + kk + (lq >> 1) * 8);
#pragma unroll
                    for (int qb = 0; qb + qa < 3; ++qb)
#pragma unroll
                        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc.c[mt][nt], af, bf[qb][nt][0], bf[qb][nt][1]);
                }
            }
        }
    }
    __syncthreads();
}

// Visits (row, col, value) of this thread's accumulator entries, rows and
// columns in [0, 128).
template <class F>
__device__ __forceinline__ void bacc_for_each(const BAcc& acc, F&& f)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp >> 2, wn = warp & 3;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int r = wm * 64 + mt * 16 + g, c = wn * 32 + nt * 8 + 2 * t;
            f(r, c, acc.c[mt][nt][0]);
            f(r, c + 1, acc.c[mt][nt][1]);
            f(r + 8, c, acc.c[mt][nt][2]);
            f(r + 8, c + 1, acc.c[mt][nt][3]);
        }
}

// Three-plane split of an FP32 value (round to nearest at each step).
__device__ __forceinline__ void split3(float v, __nv_bfloat16& hi, __nv_bfloat16& mid, __nv_bfloat16& lo)
{
    hi = __float2bfloat16_rn(v);
    float r1 = v - __bfloat162float(hi);
    mid = __float2bfloat16_rn(r1);
    float r2 = r1 - __bfloat162float(mid);
    lo = __float2bfloat16_rn(r2);
}

}  // namespace gpk
