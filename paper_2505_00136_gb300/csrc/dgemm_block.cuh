// FP64 64x64 block product on the FP64 tensor pipe (mma.sync.m8n8k4.f64),
// the building block of every FP64 tile operation (POTRF/TRSM/SYRK/GEMM of
// Fig. 1, the multi-right-hand-side solve, the inverse and the covariance).
//
//   acc(r, c) += sum_{k in [kb, ke)} A(r, k) * Bt(c, k),   0 <= r, c < 64
//
// Each operand is a strided view: element (row, k) lives at p[row*sr + k*sk],
// which covers row-major, column-major and transposed tiles without copies.
// Rows at or beyond `rows` read as zero.  (ke - kb) must be a multiple of 16.
//
// One CTA of 256 threads (8 warps) owns the block.  Warp w computes rows
// (w>>1)*16 .. +16 and columns (w&1)*32 .. +32 as 2 x 4 8x8 fragments.  K is
// staged 16 at a time through double-buffered shared memory, global loads
// for stage s+1 in flight while stage s is multiplied.
#pragma once
#include <stdint.h>

namespace gpk {

struct DView {
    const double* p;
    int64_t sr, sk;
    int rows;
};

struct DAcc {
    double c[2][4][2];
};

constexpr int DG_KS = 16;       // k per stage
constexpr int DG_LD = 72;       // padded row length in shared memory (doubles)
constexpr int DG_SMEM_DOUBLES = 2 * 2 * DG_KS * DG_LD;  // 2 stages x {A, B}
constexpr int DG_SMEM_BYTES = DG_SMEM_DOUBLES * 8;

__device__ __forceinline__ void dacc_zero(DAcc& a)
{
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) a.c[i][j][0] = a.c[i][j][1] = 0.0;
}

// Loads this thread's 4 elements of a 64 x 16 stage of view v into regs.
__device__ __forceinline__ void dg_load(const DView& v, int64_t k0, double (&reg)[4])
{
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int idx = tid + q * 256;
        int r, kk;
        if (v.sk == 1) { r = idx >> 4; kk = idx & 15; }   // contiguous along k
        else           { kk = idx >> 6; r = idx & 63; }   // contiguous along rows
        reg[q] = (r < v.rows) ? __ldcg(v.p + (int64_t)r * v.sr + (k0 + kk) * v.sk) : 0.0;
    }
}

__device__ __forceinline__ void dg_store(const DView& v, double* s, const double (&reg)[4])
{
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int idx = tid + q * 256;
        int r, kk;
        if (v.sk == 1) { r = idx >> 4; kk = idx & 15; }
        else           { kk = idx >> 6; r = idx & 63; }
        s[kk * DG_LD + r] = reg[q];
    }
}

__device__ __forceinline__ void dmma(double (&c)[2], double a, double b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c[0]), "+d"(c[1])
                 : "d"(a), "d"(b));
}

// acc += A[:, kb:ke] * Bt[:, kb:ke]^T.  smem must hold DG_SMEM_DOUBLES.
// Starts and ends with a CTA barrier, so callers may overwrite the operands
// (in place) right after it returns.
static __device__ __forceinline__ void dgemm_acc(DAcc& acc, const DView& A, const DView& B, int64_t kb, int64_t ke,
                          double* smem)
{
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int g = lane >> 2, t = lane & 3;
    const int nst = (int)((ke - kb) / DG_KS);
    if (nst <= 0) return;
    double ra[4], rb[4];
    dg_load(A, kb, ra);
    dg_load(B, kb, rb);
    dg_store(A, smem, ra);
    dg_store(B, smem + DG_KS * DG_LD, rb);
    __syncthreads();
    for (int s = 0; s < nst; ++s) {
        const int cur = s & 1;
        const double* As = smem + cur * (2 * DG_KS * DG_LD);
        const double* Bs = As + DG_KS * DG_LD;
        if (s + 1 < nst) {
            dg_load(A, kb + (int64_t)(s + 1) * DG_KS, ra);
            dg_load(B, kb + (int64_t)(s + 1) * DG_KS, rb);
        }
#pragma unroll
        for (int kq = 0; kq < DG_KS; kq += 4) {
            const double* ap = As + (kq + t) * DG_LD + wm * 16 + g;
            const double* bp = Bs + (kq + t) * DG_LD + wn * 32 + g;
            double a0 = ap[0], a1 = ap[8];
            double b0 = bp[0], b1 = bp[8], b2 = bp[16], b3 = bp[24];
            dmma(acc.c[0][0], a0, b0); dmma(acc.c[0][1], a0, b1);
            dmma(acc.c[0][2], a0, b2); dmma(acc.c[0][3], a0, b3);
            dmma(acc.c[1][0], a1, b0); dmma(acc.c[1][1], a1, b1);
            dmma(acc.c[1][2], a1, b2); dmma(acc.c[1][3], a1, b3);
        }
        if (s + 1 < nst) {
            double* An = smem + (cur ^ 1) * (2 * DG_KS * DG_LD);
            dg_store(A, An, ra);
            dg_store(B, An + DG_KS * DG_LD, rb);
        }
        __syncthreads();
    }
}

// Visits this thread's accumulator entries as (row, col, value), rows and
// columns in [0, 64).
template <class F>
__device__ __forceinline__ void dacc_for_each(const DAcc& acc, F&& f)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int i = 0; i < 2; ++i)
                f(wm * 16 + mt * 8 + g, wn * 32 + nt * 8 + t * 2 + i, acc.c[mt][nt][i]);
}

}  // namespace gpk
