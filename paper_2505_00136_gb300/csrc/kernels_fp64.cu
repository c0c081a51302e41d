// FP64 hot path of exact GP regression on GB300 (sm_103a).
//
// Tile storage and the step order follow the tiled right-looking Cholesky of
// GPRat Section 4.2 / Fig. 1 (POTRF on the diagonal tile, TRSM on the panel,
// SYRK/GEMM on the trailing tiles).  Every tile product runs on the FP64
// tensor pipe through dgemm_acc; the diagonal-tile factor uses a 64x64
// shared-memory Cholesky with per-column barriers.
#include <float.h>
#include <math.h>

#include "dgemm_block.cuh"
#include "gp_internal.cuh"
#include "se_common.cuh"
#include "kfun.cuh"

namespace gpk {

constexpr int TB = GP_TB;
constexpr int NT = GP_THREADS;

// ---------------------------------------------------------------- assembly (Eq. 2)
enum SeMode { SE_TRAIN = 0, SE_CROSS = 1, SE_PRIOR = 2 };

// SE_TRAIN : lower tiles of K = K_f + sigma^2 I, identity on padding rows.
// SE_CROSS : B (Np x ldm) = K_{Z*,Z}^T, zero outside n x m.
// SE_PRIOR : out (m x m, ld m) = K_{Z*,Z*} (+ sigma^2 I when noisy).
__global__ __launch_bounds__(NT) void k_se_block(int mode, double* out, float* out32, int64_t ldo,
                                                 const double* X, int64_t n, const double* Xs,
                                                 int64_t m, int64_t d, int64_t b, int P,
                                                 const GpHyperDev* hyp, int noisy)
{
    __shared__ double sm[2 * 64 * 17];
    int64_t r0, c0;          // global row / column of the block's first element
    double* dst;             // block origin
    float* dst32 = nullptr;  // optional FP32 copy (SE_TRAIN, mixed precision)
    int64_t ld;
    const double *Pp = X, *Qp = X;
    int64_t np = n, nq = n;
    if (mode == SE_TRAIN) {
        int64_t ti, tj;
        tri_decode(blockIdx.x, ti, tj);
        int rb = blockIdx.y / P, cb = blockIdx.y % P;
        if (ti == tj && cb > rb) return;
        r0 = ti * b + rb * TB;
        c0 = tj * b + cb * TB;
        ld = b;
        dst = out + tri_index(ti, tj) * b * b + (int64_t)rb * TB * b + cb * TB;
        if (out32) dst32 = out32 + tri_index(ti, tj) * b * b + (int64_t)rb * TB * b + cb * TB;
    } else if (mode == SE_CROSS) {
        r0 = (int64_t)blockIdx.x * TB;
        c0 = (int64_t)blockIdx.y * TB;
        ld = ldo;
        dst = out + r0 * ldo + c0;
        Qp = Xs;
        nq = m;
    } else {
        r0 = (int64_t)blockIdx.x * TB;
        c0 = (int64_t)blockIdx.y * TB;
        ld = ldo;
        dst = out + r0 * ldo + c0;
        Pp = Xs;
        Qp = Xs;
        np = m;
        nq = m;
    }
    double r2[4][4];
    dist_block(r2, Pp, r0, np, Qp, c0, nq, d, sm);
    const double s2 = hyp->s2;
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int rr = ty + 16 * a, cc = tx + 16 * c;
            int64_t gi = r0 + rr, gj = c0 + cc;
            double v;
            if (mode == SE_TRAIN) {
                if (gi < n && gj < n) v = kval(r2[a][c], hyp) + (gi == gj ? s2 : 0.0);
                else v = (gi == gj) ? 1.0 : 0.0;
            } else if (mode == SE_CROSS) {
                v = (gi < n && gj < m) ? kval(r2[a][c], hyp) : 0.0;
            } else {
                if (gi >= m || gj >= m) continue;
                v = kval(r2[a][c], hyp) + ((noisy && gi == gj) ? s2 : 0.0);
            }
            dst[(int64_t)rr * ld + cc] = v;
            if (dst32) dst32[(int64_t)rr * ld + cc] = (float)v;
        }
}

// ---------------------------------------------------------------- POTRF + TRTRI of one diagonal tile
// Left-looking blocked Cholesky of the b x b diagonal tile k (64-wide
// panels), then the blocked inverse of its factor into Linv[k].  Adds
// sum log L_ii of the tile to logdet_part[k]; on a non-positive pivot records
// the global row in *info and stops.
// Operands that other CTAs of a persistent launch may have written are read
// through L2 (ld.global.cg), never from a possibly stale L1 line.
__device__ __forceinline__ double ldl2(const double* p) { return __ldcg(p); }

// Returns false (after recording the row) on a non-positive pivot.
__device__ bool potrf_tile(double* A, double* Xk, int64_t b, int64_t row0, double* logdet_slot,
                           unsigned long long* info, double* smem)
{
    double* gsm = smem;                              // dgemm staging
    double* S = smem + DG_SMEM_DOUBLES;              // 64 x 65 factor block
    double* Iv = S + 64 * 65;                        // 64 x 65 inverse block
    __shared__ double logacc, rcp;
    __shared__ int fail;
    const int tid = threadIdx.x;
    const int P = (int)(b / TB);
    if (tid == 0) { logacc = 0.0; fail = 0; }

    for (int p = 0; p < P; ++p) {
        double* App = A + (int64_t)p * TB * b + p * TB;
        if (p > 0) {  // A_pp -= A_p,<p A_p,<p^T
            DAcc acc;
            dacc_zero(acc);
            DView va{A + (int64_t)p * TB * b, b, 1, TB};
            dgemm_acc(acc, va, va, 0, (int64_t)p * TB, gsm);
            dacc_for_each(acc, [&](int r, int c, double v) {
                double* q = App + (int64_t)r * b + c;
                *q = ldl2(q) - v;
            });
        }
        __syncthreads();
        for (int e = tid; e < 64 * 64; e += NT) {
            int r = e >> 6, c = e & 63;
            S[r * 65 + c] = (c <= r) ? ldl2(App + (int64_t)r * b + c) : 0.0;
            Iv[r * 65 + c] = 0.0;
        }
        __syncthreads();
        // unblocked right-looking Cholesky of the 64 x 64 block
        for (int j = 0; j < 64; ++j) {
            if (tid == 0) {
                double piv = S[j * 65 + j];
                if (piv > 0.0) {
                    double s = sqrt(piv);
                    S[j * 65 + j] = s;
                    rcp = 1.0 / s;
                } else {
                    fail = 1;
                    atomicMin(info, (unsigned long long)(row0 + p * TB + j));
                }
            }
            __syncthreads();
            if (fail) return false;
            const double djj_inv = rcp;
            for (int r = j + 1 + tid; r < 64; r += NT) S[r * 65 + j] *= djj_inv;
            __syncthreads();
            const int ty = tid >> 4, tx = tid & 15;
            for (int r = j + 1 + ty; r < 64; r += 16) {
                const double lr = S[r * 65 + j];
                for (int c = j + 1 + tx; c <= r; c += 16) S[r * 65 + c] -= lr * S[c * 65 + j];
            }
            __syncthreads();
        }
        if (tid < 32) {  // sum log L_jj of the block
            double lg = log(S[tid * 65 + tid]) + log(S[(tid + 32) * 65 + tid + 32]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) lg += __shfl_xor_sync(0xffffffffu, lg, o);
            if (tid == 0) logacc += lg;
        }
        // inverse of the 64 x 64 factor, row by row; 4 threads per column
        {
            const int c = tid >> 2, q = tid & 3;
            for (int r = 0; r < 64; ++r) {
                double s = 0.0;
                if (c < r)
                    for (int t = c + q; t < r; t += 4) s = fma(S[r * 65 + t], Iv[t * 65 + c], s);
                s += __shfl_xor_sync(0xffffffffu, s, 1);
                s += __shfl_xor_sync(0xffffffffu, s, 2);
                if (q == 0 && c <= r) Iv[r * 65 + c] = ((r == c) ? 1.0 : -s) / S[r * 65 + r];
                __syncthreads();
            }
        }
        double* Xpp = Xk + (int64_t)p * TB * b + p * TB;
        for (int e = tid; e < 64 * 64; e += NT) {
            int r = e >> 6, c = e & 63;
            App[(int64_t)r * b + c] = S[r * 65 + c];
            Xpp[(int64_t)r * b + c] = Iv[r * 65 + c];
        }
        __syncthreads();
        // panel below the block inside the tile: A_rp = (A_rp - A_r,<p A_p,<p^T) L_pp^{-T}
        for (int r = p + 1; r < P; ++r) {
            double* Arp = A + (int64_t)r * TB * b + p * TB;
            if (p > 0) {
                DAcc acc;
                dacc_zero(acc);
                DView va{A + (int64_t)r * TB * b, b, 1, TB};
                DView vb{A + (int64_t)p * TB * b, b, 1, TB};
                dgemm_acc(acc, va, vb, 0, (int64_t)p * TB, gsm);
                dacc_for_each(acc, [&](int rr, int c, double v) {
                    double* q = Arp + (int64_t)rr * b + c;
                    *q = ldl2(q) - v;
                });
            }
            DAcc acc;
            dacc_zero(acc);
            DView va{Arp, b, 1, TB};
            DView vx{Xpp, b, 1, TB};
            dgemm_acc(acc, va, vx, 0, TB, gsm);
            dacc_for_each(acc, [&](int rr, int c, double v) { Arp[(int64_t)rr * b + c] = v; });
        }
    }
    // zero the strict upper triangle of the tile
    __syncthreads();
    for (int64_t e = tid; e < b * b; e += NT) {
        int64_t r = e / b, c = e % b;
        if (c > r) { A[e] = 0.0; Xk[e] = 0.0; }
    }
    // TRTRI: X_rq = -X_rr * sum_{t=q}^{r-1} L_rt X_tq  (64-blocks inside the tile)
    for (int r = 1; r < P; ++r) {
        for (int q = 0; q < r; ++q) {
            double* Xrq = Xk + (int64_t)r * TB * b + q * TB;
            DAcc acc;
            dacc_zero(acc);
            DView vl{A + (int64_t)r * TB * b, b, 1, TB};       // L_r,(.)
            DView vx{Xk + q * TB, 1, b, TB};                    // Bt(c, t) = X[t][q*64 + c]
            dgemm_acc(acc, vl, vx, (int64_t)q * TB, (int64_t)r * TB, gsm);
            dacc_for_each(acc, [&](int rr, int c, double v) { Xrq[(int64_t)rr * b + c] = v; });
            dacc_zero(acc);
            DView vrr{Xk + (int64_t)r * TB * b + r * TB, b, 1, TB};
            DView vs{Xrq, 1, b, TB};
            dgemm_acc(acc, vrr, vs, 0, TB, gsm);
            dacc_for_each(acc, [&](int rr, int c, double v) { Xrq[(int64_t)rr * b + c] = -v; });
        }
    }
    __syncthreads();
    if (tid == 0) *logdet_slot = logacc;
    return true;
}

__global__ __launch_bounds__(NT) void k_potrf_diag(double* A, double* Xk, int64_t b, int64_t row0,
                                                   double* logdet_slot, unsigned long long* info)
{
    extern __shared__ double smem[];
    if (failed(info)) return;
    potrf_tile(A, Xk, b, row0, logdet_slot, info, smem);
}

// Panel TRSM of step k: L_ik = A_ik L_kk^{-T} = A_ik Linv_kk^T for i > k.
// One CTA per (64-row block, tile); column blocks right to left keep it in place.
__device__ void panel_rows(double* tile, const double* Xk, int64_t b, int rb, double* smem)
{
    const int P = (int)(b / TB);
    double* Arow = tile + (int64_t)rb * TB * b;
    for (int cb = P - 1; cb >= 0; --cb) {
        DAcc acc;
        dacc_zero(acc);
        DView va{Arow, b, 1, TB};
        DView vx{Xk + (int64_t)cb * TB * b, b, 1, TB};
        dgemm_acc(acc, va, vx, 0, (int64_t)(cb + 1) * TB, smem);
        double* dst = Arow + cb * TB;
        dacc_for_each(acc, [&](int r, int c, double v) { dst[(int64_t)r * b + c] = v; });
    }
}

__global__ __launch_bounds__(NT) void k_panel(double* Lt, const double* Linv, int64_t b, int64_t k,
                                              const unsigned long long* info)
{
    extern __shared__ double smem[];
    if (failed(info)) return;
    const int64_t i = k + 1 + blockIdx.y;
    panel_rows(Lt + tri_index(i, k) * b * b, Linv + k * b * b, b, blockIdx.x, smem);
}

// Trailing update of step k: A_ij -= L_ik L_jk^T for k < j <= i (SYRK on
// diagonal tiles, GEMM elsewhere).  grid.x: trailing lower tile, grid.y: 64-block.
__device__ void update_block(double* Lt, int64_t b, int64_t i, int64_t j, int64_t k, int rb, int cb,
                             double* smem)
{
    DAcc acc;
    dacc_zero(acc);
    DView va{Lt + tri_index(i, k) * b * b + (int64_t)rb * TB * b, b, 1, TB};
    DView vb{Lt + tri_index(j, k) * b * b + (int64_t)cb * TB * b, b, 1, TB};
    dgemm_acc(acc, va, vb, 0, b, smem);
    double* dst = Lt + tri_index(i, j) * b * b + (int64_t)rb * TB * b + cb * TB;
    dacc_for_each(acc, [&](int r, int c, double v) {
        double* q = dst + (int64_t)r * b + c;
        *q = ldl2(q) - v;
    });
}

__global__ __launch_bounds__(NT) void k_update(double* Lt, int64_t b, int64_t k,
                                               const unsigned long long* info)
{
    extern __shared__ double smem[];
    if (failed(info)) return;
    const int P = (int)(b / TB);
    int64_t ii, jj;
    tri_decode(blockIdx.x, ii, jj);
    const int64_t i = k + 1 + ii, j = k + 1 + jj;
    const int rb = blockIdx.y / P, cb = blockIdx.y % P;
    if (i == j && cb > rb) return;
    update_block(Lt, b, i, j, k, rb, cb, smem);
}

// ---------------------------------------------------------------- persistent tile-DAG Cholesky
// One launch walks the whole task graph of Fig. 1: POTRF(k), TRSM(i, k) and
// UPDATE(i, j, k) tasks, queued on the host in a topological order with
// one-step lookahead.  CTAs claim tasks with an atomic ticket; a task waits
// only on tasks with smaller tickets, which are already held by running CTAs,
// so the walk cannot deadlock.  Dependencies are per-tile counters:
//   upd[tri(i, j)] = number of trailing updates applied to tile (i, j),
//   fin[tri(i, j)] = 1 once tile (i, j) of L is final (POTRF or TRSM done).
// Every wait is bounded by a clock-cycle budget; on expiry the CTA sets
// ctl[1] = 1 (timeout), a failed pivot sets ctl[1] = 2, and all CTAs leave.
__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ bool dag_wait(const int* p, int need, int* ctl, long long budget)
{
    if (ld_acquire(p) >= need) return true;
    const long long t0 = clock64();
    for (;;) {
        __nanosleep(256);
        if (ld_acquire(p) >= need) return true;
        if (ld_acquire(ctl + 1) != 0) return false;
        if (clock64() - t0 > budget) {
            atomicCAS(ctl + 1, 0, 1);
            return false;
        }
    }
}

__global__ __launch_bounds__(NT) void k_chol_dag(double* Lt, double* Linv, int64_t b, const int4* tasks,
                                                 int64_t ntasks, int* ctl, int* upd, int* fin,
                                                 double* logdet_part, unsigned long long* info, long long budget)
{
    extern __shared__ double smem[];
    __shared__ int s_task, s_go;
    const int P = (int)(b / TB);
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(ctl, 1);
            int go = (t < ntasks) && ld_acquire(ctl + 1) == 0;
            if (go) {
                const int4 tk = tasks[t];
                if (tk.x == 0)
                    go = dag_wait(upd + tri_index(tk.w, tk.w), tk.w, ctl, budget);
                else if (tk.x == 1)
                    go = dag_wait(fin + tri_index(tk.w, tk.w), 1, ctl, budget) &&
                         dag_wait(upd + tri_index(tk.y, tk.w), tk.w, ctl, budget);
                else
                    go = dag_wait(fin + tri_index(tk.y, tk.w), 1, ctl, budget) &&
                         dag_wait(fin + tri_index(tk.z, tk.w), 1, ctl, budget) &&
                         dag_wait(upd + tri_index(tk.y, tk.z), tk.w, ctl, budget);
            }
            s_task = t;
            s_go = go;
        }
        __syncthreads();
        if (!s_go) break;
        const int4 tk = tasks[s_task];   // (type, i, j, k)
        const int64_t i = tk.y, j = tk.z, k = tk.w;
        bool ok = true;
        if (tk.x == 0) {
            ok = potrf_tile(Lt + tri_index(k, k) * b * b, Linv + k * b * b, b, k * b, logdet_part + k, info, smem);
        } else if (tk.x == 1) {
            for (int rb = 0; rb < P; ++rb) panel_rows(Lt + tri_index(i, k) * b * b, Linv + k * b * b, b, rb, smem);
        } else {
            for (int rb = 0; rb < P; ++rb)
                for (int cb = 0; cb <= (i == j ? rb : P - 1); ++cb) update_block(Lt, b, i, j, k, rb, cb, smem);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (!ok) atomicExch(ctl + 1, 2);
            else if (tk.x == 0) atomicExch(fin + tri_index(k, k), 1);
            else if (tk.x == 1) atomicExch(fin + tri_index(i, k), 1);
            else atomicAdd(upd + tri_index(i, j), 1);
        }
    }
}

__global__ void k_dag_stall(int* upd, int64_t idx) { upd[idx] = -(1 << 30); }

// ---------------------------------------------------------------- single right-hand side solves
// out_j = Linv_jj w_j (lower: rows of the tile inverse) or Linv_jj^T w_j (upper).
__global__ __launch_bounds__(NT) void k_tri_apply(const double* Linv, int64_t b, int64_t j,
                                                  const double* w, double* out, int upper)
{
    const double* Xj = Linv + j * b * b;
    const double* wj = w + j * b;
    double* oj = out + j * b;
    if (!upper) {  // warp per row, lanes over columns t <= r
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int64_t r = (int64_t)blockIdx.x * 8 + warp; r < b; r += (int64_t)gridDim.x * 8) {
            double s = 0.0;
            for (int64_t t = lane; t <= r; t += 32) s = fma(Xj[r * b + t], wj[t], s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) oj[r] = s;
        }
    } else {       // thread per output column c: sum over rows t >= c of X[t][c] w[t]
        for (int64_t c = (int64_t)blockIdx.x * NT + threadIdx.x; c < b; c += (int64_t)gridDim.x * NT) {
            double s = 0.0;
            for (int64_t t = c; t < b; ++t) s = fma(Xj[t * b + c], wj[t], s);
            oj[c] = s;
        }
    }
}

// Forward sweep update: w_i -= L_ij x_j for all i > j.  Warp per row.
__global__ __launch_bounds__(NT) void k_gemv_lower(const double* Lt, int64_t b, int64_t j, int64_t T,
                                                   const double* x, double* w)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t rows = (T - j - 1) * b;
    const double* xj = x + j * b;
    for (int64_t R = (int64_t)blockIdx.x * 8 + warp; R < rows; R += (int64_t)gridDim.x * 8) {
        int64_t i = j + 1 + R / b, r = R % b;
        const double* row = Lt + tri_index(i, j) * b * b + r * b;
        double s = 0.0;
        for (int64_t t = lane; t < b; t += 32) s = fma(row[t], xj[t], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) w[i * b + r] -= s;
    }
}

// Backward sweep update: w_i -= L_ji^T x_j for all i < j.  64 columns per CTA,
// 4 row phases reduced through shared memory.
__global__ __launch_bounds__(NT) void k_gemv_upper(const double* Lt, int64_t b, int64_t j,
                                                   const double* x, double* w)
{
    __shared__ double red[4][64];
    const int c = threadIdx.x & 63, q = threadIdx.x >> 6;
    const int64_t cols = j * b;
    const int64_t C = (int64_t)blockIdx.x * 64 + c;
    const double* xj = x + j * b;
    double s = 0.0;
    if (C < cols) {
        int64_t i = C / b, cc = C % b;
        const double* tile = Lt + tri_index(j, i) * b * b;
        for (int64_t r = q; r < b; r += 4) s = fma(tile[r * b + cc], xj[r], s);
    }
    red[q][c] = s;
    __syncthreads();
    if (q == 0 && C < cols) w[C] -= red[0][c] + red[1][c] + red[2][c] + red[3][c];
}

// ---------------------------------------------------------------- multi right-hand side forward solve
// V_j = Linv_jj B_j for a 64 x 64 block of V (rows of tile j, test columns),
// with fused per-column partial sums of V^2 (variance) and V * beta (mean).
__global__ __launch_bounds__(NT) void k_diagV(const double* Linv, const double* B, double* V,
                                              const double* beta, double* part, int64_t b,
                                              int64_t j, int64_t ldm, int64_t nq)
{
    extern __shared__ double smem[];
    __shared__ double cs[2][4][64];
    const int P = (int)(b / TB);
    const int rb = blockIdx.x, cb = blockIdx.y;
    const int64_t row0 = j * b + (int64_t)rb * TB, col0 = (int64_t)cb * TB;
    DAcc acc;
    dacc_zero(acc);
    DView va{Linv + j * b * b + (int64_t)rb * TB * b, b, 1, TB};
    DView vb{B + j * b * ldm + col0, 1, ldm, TB};
    dgemm_acc(acc, va, vb, 0, (int64_t)(rb + 1) * TB, smem);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wm = warp >> 1;
    double sq[4][2], sb[4][2];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) sq[nt][0] = sq[nt][1] = sb[nt][0] = sb[nt][1] = 0.0;
    const int g = lane >> 2;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const double bt = beta[row0 + wm * 16 + mt * 8 + g];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                double v = acc.c[mt][nt][e];
                sq[nt][e] = fma(v, v, sq[nt][e]);
                sb[nt][e] = fma(v, bt, sb[nt][e]);
            }
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                sq[nt][e] += __shfl_xor_sync(0xffffffffu, sq[nt][e], o);
                sb[nt][e] += __shfl_xor_sync(0xffffffffu, sb[nt][e], o);
            }
    const int wn = warp & 1, t = lane & 3;
    if (g == 0) {
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                int c = wn * 32 + nt * 8 + t * 2 + e;
                cs[0][wm][c] = sq[nt][e];
                cs[1][wm][c] = sb[nt][e];
            }
    }
    dacc_for_each(acc, [&](int r, int c, double v) { V[(row0 + r) * ldm + col0 + c] = v; });
    __syncthreads();
    if (threadIdx.x < 128) {
        int w = threadIdx.x >> 6, c = threadIdx.x & 63;
        double s = cs[w][0][c] + cs[w][1][c] + cs[w][2][c] + cs[w][3][c];
        int64_t q = j * P + rb;
        part[((int64_t)w * nq + q) * ldm + col0 + c] = s;
    }
}

// B_i -= L_ij V_j for all tiles i > j (64 x 64 blocks over test columns).
__global__ __launch_bounds__(NT) void k_updV(const double* Lt, double* B, const double* V, int64_t b,
                                             int64_t j, int64_t ldm)
{
    extern __shared__ double smem[];
    const int P = (int)(b / TB);
    const int64_t i = j + 1 + blockIdx.x / P;
    const int rb = blockIdx.x % P;
    const int64_t col0 = (int64_t)blockIdx.y * TB;
    DAcc acc;
    dacc_zero(acc);
    DView va{Lt + tri_index(i, j) * b * b + (int64_t)rb * TB * b, b, 1, TB};
    DView vb{V + j * b * ldm + col0, 1, ldm, TB};
    dgemm_acc(acc, va, vb, 0, b, smem);
    double* dst = B + (i * b + (int64_t)rb * TB) * ldm + col0;
    dacc_for_each(acc, [&](int r, int c, double v) { dst[(int64_t)r * ldm + c] -= v; });
}

// mean_c = sum_q part[1][q][c], var_c = prior - sum_q part[0][q][c].
__global__ void k_predict_finish(const double* part, int64_t nq, int64_t ldm, int64_t m,
                                 const GpHyperDev* hyp, int noisy, double* mean, double* var)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    double sv = 0.0, sm = 0.0;
    for (int64_t q = 0; q < nq; ++q) {
        sv += part[q * ldm + c];
        sm += part[(nq + q) * ldm + c];
    }
    if (mean) mean[c] = sm;
    if (var) var[c] = hyp->nu + (noisy ? hyp->s2 : 0.0) - sv;
}

// mean only: part[q][c] = sum over rows of chunk q of B[r][c] alpha[r].
__global__ void k_mean_gemv(const double* B, const double* alpha, int64_t rows_per, int64_t Np,
                            int64_t ldm, double* part)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ldm) return;
    int64_t q = blockIdx.y, r0 = q * rows_per, r1 = r0 + rows_per < Np ? r0 + rows_per : Np;
    double s = 0.0;
    for (int64_t r = r0; r < r1; ++r) s = fma(B[r * ldm + c], alpha[r], s);
    part[q * ldm + c] = s;
}

__global__ void k_sum_rows(const double* part, int64_t nq, int64_t ldm, int64_t m, double* out)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    double s = 0.0;
    for (int64_t q = 0; q < nq; ++q) s += part[q * ldm + c];
    out[c] = s;
}

// ---------------------------------------------------------------- full covariance (Eq. 4)
// cov (m x m) -= V^T V on lower 64-blocks, mirrored to the upper triangle.
__global__ __launch_bounds__(NT) void k_syrk_cov(const double* V, int64_t Np, int64_t ldm, int64_t m,
                                                 double* cov)
{
    extern __shared__ double smem[];
    int64_t a, c;
    tri_decode(blockIdx.x, a, c);
    DAcc acc;
    dacc_zero(acc);
    DView va{V + a * TB, 1, ldm, TB};
    DView vb{V + c * TB, 1, ldm, TB};
    dgemm_acc(acc, va, vb, 0, Np, smem);
    dacc_for_each(acc, [&](int r, int cc, double v) {
        int64_t R = a * TB + r, C = c * TB + cc;
        if (R >= m || C >= m || (a == c && cc > r)) return;
        double x = cov[R * m + C] - v;
        cov[R * m + C] = x;
        cov[C * m + R] = x;
    });
}

// ---------------------------------------------------------------- NLML (Eq. 5)
__global__ void k_nlml(const double* beta, int64_t n, const double* logdet_part, int64_t T,
                       double* scal)
{
    __shared__ double red[NT];
    double s = 0.0, ld = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += NT) s = fma(beta[i], beta[i], s);
    for (int64_t i = threadIdx.x; i < T; i += NT) ld += logdet_part[i];
    red[threadIdx.x] = 0.5 * s + ld;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) scal[0] = red[0] + 0.5 * (double)n * log(2.0 * M_PI);
}

// ---------------------------------------------------------------- K^{-1} for the gradient
// Xinv_jj = Linv_jj.
__global__ void k_copy_diag(const double* Linv, double* Xinv, int64_t b, int64_t T)
{
    int64_t total = T * b * b;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = e / (b * b), off = e % (b * b);
        Xinv[tri_index(j, j) * b * b + off] = Linv[e];
    }
}

// X_tj = -Linv_tt S_tj (S_tj accumulated in place) for j < t; row blocks
// bottom-up keep the product in place.  grid: (column block, j).
__global__ __launch_bounds__(NT) void k_trtri_scale(const double* Linv, double* Xinv, int64_t b, int64_t t)
{
    extern __shared__ double smem[];
    const int P = (int)(b / TB);
    const int cb = blockIdx.x;
    const int64_t j = blockIdx.y;
    double* S = Xinv + tri_index(t, j) * b * b;
    const double* Lt_ = Linv + t * b * b;
    for (int rb = P - 1; rb >= 0; --rb) {
        DAcc acc;
        dacc_zero(acc);
        DView va{Lt_ + (int64_t)rb * TB * b, b, 1, TB};
        DView vb{S + cb * TB, 1, b, TB};
        dgemm_acc(acc, va, vb, 0, (int64_t)(rb + 1) * TB, smem);
        double* dst = S + (int64_t)rb * TB * b + cb * TB;
        dacc_for_each(acc, [&](int r, int c, double v) { dst[(int64_t)r * b + c] = -v; });
    }
}

// S_ij (+)= L_it X_tj for i > t >= j; the first contribution (t == j) overwrites.
// grid.x: (i - t - 1) * (t + 1) + j, grid.y: 64-block.
__global__ __launch_bounds__(NT) void k_trtri_accum(const double* Lt, double* Xinv, int64_t b, int64_t t)
{
    extern __shared__ double smem[];
    const int P = (int)(b / TB);
    const int64_t i = t + 1 + blockIdx.x / (t + 1), j = blockIdx.x % (t + 1);
    const int rb = blockIdx.y / P, cb = blockIdx.y % P;
    DAcc acc;
    dacc_zero(acc);
    DView va{Lt + tri_index(i, t) * b * b + (int64_t)rb * TB * b, b, 1, TB};
    DView vb{Xinv + tri_index(t, j) * b * b + cb * TB, 1, b, TB};
    dgemm_acc(acc, va, vb, 0, b, smem);
    double* dst = Xinv + tri_index(i, j) * b * b + (int64_t)rb * TB * b + cb * TB;
    const bool first = (t == j);
    dacc_for_each(acc, [&](int r, int c, double v) {
        double* p = dst + (int64_t)r * b + c;
        *p = first ? v : *p + v;
    });
}

// K^{-1}_ij = sum_{t >= i} X_ti^T X_tj on lower tiles (LAUUM).
__global__ __launch_bounds__(NT) void k_lauum(const double* Xinv, double* Kinv, int64_t b, int64_t T)
{
    extern __shared__ double smem[];
    const int P = (int)(b / TB);
    int64_t i, j;
    tri_decode(blockIdx.x, i, j);
    const int rb = blockIdx.y / P, cb = blockIdx.y % P;
    if (i == j && cb > rb) return;
    DAcc acc;
    dacc_zero(acc);
    for (int64_t t = i; t < T; ++t) {
        DView va{Xinv + tri_index(t, i) * b * b + rb * TB, 1, b, TB};
        DView vb{Xinv + tri_index(t, j) * b * b + cb * TB, 1, b, TB};
        dgemm_acc(acc, va, vb, (t == i) ? (int64_t)rb * TB : 0, b, smem);
    }
    double* dst = Kinv + tri_index(i, j) * b * b + (int64_t)rb * TB * b + cb * TB;
    dacc_for_each(acc, [&](int r, int c, double v) { dst[(int64_t)r * b + c] = v; });
}

// ---------------------------------------------------------------- adjoint gradient
// Partial sums over one 64 x 64 block of a lower tile of
//   sum W_ij K_f,ij r2_ij,  sum W_ij K_f,ij,  sum_i W_ii
// with W = K^{-1} - alpha alpha^T, weight 2 off the diagonal; dK/dtheta is
// regenerated from X here and never stored.
template <class KT>
__global__ __launch_bounds__(NT) void k_adjoint(const KT* Kinv, const double* alpha, const double* X,
                                                int64_t n, int64_t d, int64_t b,
                                                const GpHyperDev* hyp, double* gpart)
{
    __shared__ double sm[2 * 64 * 17];
    __shared__ double red[3][NT];
    const int P = (int)(b / TB);
    int64_t i, j;
    tri_decode(blockIdx.x, i, j);
    const int rb = blockIdx.y / P, cb = blockIdx.y % P;
    double s_l = 0.0, s_nu = 0.0, s_s2 = 0.0;
    if (!(i == j && cb > rb)) {
        const int64_t r0 = i * b + (int64_t)rb * TB, c0 = j * b + (int64_t)cb * TB;
        double r2[4][4];
        dist_block(r2, X, r0, n, X, c0, n, d, sm);
        const KT* tile = Kinv + tri_index(i, j) * b * b + (int64_t)rb * TB * b + cb * TB;
        const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int rr = ty + 16 * a, cc = tx + 16 * c;
                int64_t gi = r0 + rr, gj = c0 + cc;
                if (gi >= n || gj >= n || gj > gi) continue;
                double w = (double)tile[(int64_t)rr * b + cc] - alpha[gi] * alpha[gj];
                double kf = kval(r2[a][c], hyp);
                double wt = (gi == gj) ? 1.0 : 2.0;
                s_l = fma(wt * w, kdl_term(r2[a][c], kf, hyp), s_l);
                s_nu = fma(wt * w, kf, s_nu);
                if (gi == gj) s_s2 += w;
            }
    }
    red[0][threadIdx.x] = s_l;
    red[1][threadIdx.x] = s_nu;
    red[2][threadIdx.x] = s_s2;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int p = 0; p < 3; ++p) red[p][threadIdx.x] += red[p][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 3) {
        int64_t blk = (int64_t)blockIdx.x * gridDim.y + blockIdx.y;
        gpart[blk * 3 + threadIdx.x] = red[threadIdx.x][0];
    }
}

// Mixed path: the same partial sums with K_f,ij read from the FP64 K of the
// factorisation (same hyperparameters; K_f = K - sigma^2 on the diagonal)
// instead of regenerated with an FP64 exponential, and r2_ij and the sums of
// one thread's 16 elements in FP32: the FP32 inverse in W bounds the accuracy
// of this path.  Coordinates are taken relative to the block's first row (in
// FP64) before rounding to FP32, so differences of nearby points keep their
// digits.
__global__ __launch_bounds__(NT) void k_adjoint_k(const float* Kinv, const double* K64, const double* alpha,
                                                  const double* X, int64_t n, int64_t d, int64_t b,
                                                  const GpHyperDev* hyp, double* gpart)
{
    __shared__ float sp[64 * 17], sq[64 * 17];
    __shared__ float sa[2][64];
    __shared__ double red[3][NT];
    const int P = (int)(b / TB);
    int64_t i, j;
    tri_decode(blockIdx.x, i, j);
    const int rb = blockIdx.y / P, cb = blockIdx.y % P;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const bool live = !(i == j && cb > rb);
    const int64_t r0 = i * b + (int64_t)rb * TB, c0 = j * b + (int64_t)cb * TB;
    float r2[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) r2[a][c] = 0.f;
    if (live) {
        if (tid < 128) {
            const int q = tid & 63;
            const int64_t g = (tid < 64 ? r0 : c0) + q;
            sa[tid >> 6][q] = g < n ? (float)alpha[g] : 0.f;
        }
        for (int64_t d0 = 0; d0 < d; d0 += 16) {
            __syncthreads();
            for (int idx = tid; idx < 1024; idx += NT) {
                const int r = idx >> 4, k = idx & 15;
                const int64_t gp = r0 + r, gq = c0 + r;
                const bool kin = d0 + k < d;
                const double ref = (kin && r0 < n) ? X[r0 * d + d0 + k] : 0.0;
                sp[r * 17 + k] = (gp < n && kin) ? (float)(X[gp * d + d0 + k] - ref) : 0.f;
                sq[r * 17 + k] = (gq < n && kin) ? (float)(X[gq * d + d0 + k] - ref) : 0.f;
            }
            __syncthreads();
            const int kmax = (int)((d - d0) < 16 ? (d - d0) : 16);
            for (int k = 0; k < kmax; ++k) {
                float pa[4], qc[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) pa[a] = sp[(ty + 16 * a) * 17 + k];
#pragma unroll
                for (int c = 0; c < 4; ++c) qc[c] = sq[(tx + 16 * c) * 17 + k];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float t = pa[a] - qc[c];
                        r2[a][c] = fmaf(t, t, r2[a][c]);
                    }
            }
        }
    }
    float s_l = 0.f, s_nu = 0.f, s_s2 = 0.f;
    if (live) {
        const double s2 = hyp->s2;
        const int kind = hyp->kernel;
        const float lf = (float)hyp->l;
        const int64_t off = tri_index(i, j) * b * b + (int64_t)rb * TB * b + cb * TB;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int rr = ty + 16 * a, cc = tx + 16 * c;
                const int64_t gi = r0 + rr, gj = c0 + cc;
                if (gi >= n || gj >= n || gj > gi) continue;
                const int64_t e = off + (int64_t)rr * b + cc;
                const float w = __ldcs(Kinv + e) - sa[0][rr] * sa[1][cc];
                const float kf = (float)(gi == gj ? __ldcs(K64 + e) - s2 : __ldcs(K64 + e));
                const float wt = (gi == gj) ? 1.f : 2.f;
                s_l = fmaf(wt * w, kdl_term_f(r2[a][c], kf, kind, lf), s_l);
                s_nu = fmaf(wt * w, kf, s_nu);
                if (gi == gj) s_s2 += w;
            }
    }
    red[0][tid] = s_l;
    red[1][tid] = s_nu;
    red[2][tid] = s_s2;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (tid < o)
            for (int p = 0; p < 3; ++p) red[p][tid] += red[p][tid + o];
        __syncthreads();
    }
    if (tid < 3) {
        const int64_t blk = (int64_t)blockIdx.x * gridDim.y + blockIdx.y;
        gpart[blk * 3 + tid] = red[tid][0];
    }
}

// grad = 1/2 (sum_l kdl_scale, sum_nu, sigma^2 sum_s2), deterministic single-CTA reduction.
__global__ void k_grad_finish(const double* gpart, int64_t nblk, const GpHyperDev* hyp, double* scal)
{
    __shared__ double red[3][NT];
    double s[3] = {0.0, 0.0, 0.0};
    for (int64_t q = threadIdx.x; q < nblk; q += NT)
        for (int p = 0; p < 3; ++p) s[p] += gpart[q * 3 + p];
    for (int p = 0; p < 3; ++p) red[p][threadIdx.x] = s[p];
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int p = 0; p < 3; ++p) red[p][threadIdx.x] += red[p][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scal[1] = 0.5 * red[0][0] * kdl_scale(hyp);
        scal[2] = 0.5 * red[1][0];
        scal[3] = 0.5 * hyp->s2 * red[2][0];
    }
}

// ---------------------------------------------------------------- Adam (Kingma & Ba 2015)
__global__ void k_adam(GpHyperDev* hyp, GpAdamDev* st, const double* scal, double lr, double b1,
                       double b2, double eps, int tr0, int tr1, int tr2, double* hist_slot,
                       const unsigned long long* info)
{
    if (threadIdx.x != 0 || blockIdx.x != 0 || failed(info)) return;
    if (hist_slot) *hist_slot = scal[0];
    const int tr[3] = {tr0, tr1, tr2};
    st->t += 1.0;
    for (int p = 0; p < 3; ++p) {
        if (!tr[p]) continue;
        double g = scal[1 + p];
        st->m[p] = b1 * st->m[p] + (1.0 - b1) * g;
        st->v[p] = b2 * st->v[p] + (1.0 - b2) * g * g;
        double mh = st->m[p] / (1.0 - pow(b1, st->t));
        double vh = st->v[p] / (1.0 - pow(b2, st->t));
        hyp->log_theta[p] -= lr * mh / (sqrt(vh) + eps);
    }
    hyp->l = exp(hyp->log_theta[0]);
    hyp->nu = exp(hyp->log_theta[1]);
    hyp->s2 = exp(hyp->log_theta[2]);
    hyp->inv2l2 = 1.0 / (2.0 * hyp->l * hyp->l);
}

// Dense copy of L (n x n row-major, zero upper triangle).
__global__ void k_factor_dense(const double* Lt, int64_t b, int64_t n, double* out)
{
    int64_t total = n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e / n, c = e % n;
        out[e] = (c <= r) ? Lt[tri_index(r / b, c / b) * b * b + (r % b) * b + (c % b)] : 0.0;
    }
}

__global__ void k_set_u64(unsigned long long* p, unsigned long long v) { *p = v; }

// ================================================================ host launchers
static int grid_for(int64_t work, int per = NT)
{
    int64_t g = (work + per - 1) / per;
    if (g < 1) g = 1;
    if (g > 152 * 64) g = 152 * 64;
    return (int)g;
}

constexpr int POTRF_SMEM = DG_SMEM_BYTES + 2 * 64 * 65 * 8;

static void ensure_attrs()
{
    static int done_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (done_dev == dev) return;
    cudaFuncSetAttribute(k_potrf_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, POTRF_SMEM);
    done_dev = dev;
}

void assemble_train(gp_t h)
{
    const int P = (int)(h->b / TB);
    dim3 grid((unsigned)(h->T * (h->T + 1) / 2), (unsigned)(P * P));
    GPK_LAUNCH(h, GP_PH_ASSEMBLE, k_se_block, grid, NT, 0, SE_TRAIN, h->L, h->A32, h->b, h->X, h->n,
               (const double*)nullptr, (int64_t)0, h->d, h->b, P, h->hyp, 0);
}

void assemble_cross(gp_t h, int64_t m, int64_t ldm)
{
    dim3 grid((unsigned)(h->Np / TB), (unsigned)(ldm / TB));
    GPK_LAUNCH(h, GP_PH_CROSS, k_se_block, grid, NT, 0, SE_CROSS, h->B, (float*)nullptr, ldm, h->X, h->n, h->Xs, m,
               h->d, h->b, 1, h->hyp, 0);
}

void assemble_test_prior(gp_t h, int64_t m, double* out)
{
    unsigned g = (unsigned)((m + TB - 1) / TB);
    GPK_LAUNCH(h, GP_PH_COV, k_se_block, dim3(g, g), NT, 0, SE_PRIOR, out, (float*)nullptr, m, (const double*)nullptr,
               (int64_t)0, h->Xs, m, h->d, h->b, 1, h->hyp, h->opt.noisy_test_var);
}

void set_info_none(gp_t h) { GPK_LAUNCH(h, GP_PH_OTHER, k_set_u64, 1, 1, 0, h->info, ~0ull); }

// Persistent tile-DAG factorisation (GP_SCHED_PERSISTENT).  reset_err = false
// keeps an earlier abort code, so a failure inside an optimisation loop stays
// visible until the host reads it.
void factor_dag(gp_t h, bool reset_err)
{
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaFuncSetAttribute(k_chol_dag, cudaFuncAttributeMaxDynamicSharedMemorySize, POTRF_SMEM);
        attr_dev = dev;
    }
    ensure_attrs();
    const int64_t nt = h->T * (h->T + 1) / 2;
    cudaMemsetAsync(h->dag_ctl, 0, sizeof(int) * (reset_err ? 2 : 1), h->st);
    cudaMemsetAsync(h->dag_upd, 0, sizeof(int) * nt, h->st);
    cudaMemsetAsync(h->dag_fin, 0, sizeof(int) * nt, h->st);
    if (h->dag_stall >= 0) GPK_LAUNCH(h, GP_PH_OTHER, k_dag_stall, 1, 1, 0, h->dag_upd, h->dag_stall);
    int per_sm = 1, sms = 1, khz = 1000000;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chol_dag, NT, POTRF_SMEM);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    const long long budget = (long long)h->opt.dag_timeout_ms * (long long)khz;
    const int grid = (per_sm > 0 ? per_sm : 1) * sms;
    GPK_LAUNCH(h, GP_PH_UPDATE, k_chol_dag, grid, NT, POTRF_SMEM, h->L, h->Linv, h->b, (const int4*)h->dag_tasks,
               h->dag_ntasks, h->dag_ctl, h->dag_upd, h->dag_fin, h->logdet_part, h->info, budget);
}

void potrf_diag_launch(gp_t h, double* A, double* X, int64_t b, int64_t row0, double* logdet_slot)
{
    ensure_attrs();
    GPK_LAUNCH(h, GP_PH_POTRF, k_potrf_diag, 1, NT, POTRF_SMEM, A, X, b, row0, logdet_slot, h->info);
}

// GP_FP64_OZAKI: right-looking in super-panels of GP_OG_SP tile columns (as
// the mixed path), each diagonal tile factored and inverted by the whole GPU
// (kernels_potrf_grid.cu): each column of a super-panel is factored, solved and
// applied to the super-panel's later columns; one update with a k range of
// the whole super-panel then reaches the trailing triangle, so each trailing
// tile is read and written once per super-panel instead of once per column.
static bool factor_fp64_ozaki(gp_t h)
{
    const int64_t T = h->T, b = h->b;
    for (int64_t K0 = 0; K0 < T; K0 += GP_OG_SP) {
        const int64_t e = K0 + GP_OG_SP < T ? K0 + GP_OG_SP : T;
        for (int64_t k = K0; k < e; ++k) {
            if (!potrf_diag_grid(h, h->L + tri_index(k, k) * b * b, h->Linv + k * b * b, b, k * b,
                                 h->logdet_part + k))
                return false;
            if (k + 1 < T && (!og_panel(h, k) || !og_chol_update_cols(h, k, e))) return false;
        }
        if (e < T && !og_chol_update_sp(h, K0, e)) return false;
    }
    return true;
}

bool factor_fp64(gp_t h)
{
    ensure_attrs();
    if (h->opt.prec == GP_FP64_OZAKI) return factor_fp64_ozaki(h);
    const int64_t T = h->T, b = h->b;
    const int P = (int)(b / TB);
    for (int64_t k = 0; k < T; ++k) {
        potrf_diag_launch(h, h->L + tri_index(k, k) * b * b, h->Linv + k * b * b, b, k * b,
                          h->logdet_part + k);
        if (k + 1 < T) {
            const int64_t tt = T - k - 1;
            {
                GPK_LAUNCH(h, GP_PH_TRSM, k_panel, dim3((unsigned)P, (unsigned)(T - k - 1)), NT,
                           DG_SMEM_BYTES, h->L, (const double*)h->Linv, b, k, (const unsigned long long*)h->info);
                GPK_LAUNCH(h, GP_PH_UPDATE, k_update, dim3((unsigned)(tt * (tt + 1) / 2), (unsigned)(P * P)),
                           NT, DG_SMEM_BYTES, h->L, b, k, (const unsigned long long*)h->info);
            }
        }
    }
    return true;
}

void solve_lower(gp_t h, const double* rhs, double* out)
{
    const int64_t T = h->T, b = h->b;
    cudaMemcpyAsync(h->work, rhs, h->Np * sizeof(double), cudaMemcpyDeviceToDevice, h->st);
    const unsigned g_apply = (unsigned)((b + 7) / 8 < 64 ? (b + 7) / 8 : 64);
    for (int64_t j = 0; j < T; ++j) {
        GPK_LAUNCH(h, GP_PH_SOLVE, k_tri_apply, g_apply, NT, 0, (const double*)h->Linv, b, j,
                   (const double*)h->work, out, 0);
        if (j + 1 < T)
            GPK_LAUNCH(h, GP_PH_SOLVE, k_gemv_lower, grid_for((T - j - 1) * b, 8), NT, 0,
                       (const double*)h->L, b, j, T, (const double*)out, h->work);
    }
}

void solve_upper(gp_t h, const double* rhs, double* out)
{
    const int64_t T = h->T, b = h->b;
    cudaMemcpyAsync(h->work, rhs, h->Np * sizeof(double), cudaMemcpyDeviceToDevice, h->st);
    for (int64_t j = T - 1; j >= 0; --j) {
        GPK_LAUNCH(h, GP_PH_SOLVE, k_tri_apply, (unsigned)((b + NT - 1) / NT), NT, 0,
                   (const double*)h->Linv, b, j, (const double*)h->work, out, 1);
        if (j > 0)
            GPK_LAUNCH(h, GP_PH_SOLVE, k_gemv_upper, (unsigned)((j * b + 63) / 64), NT, 0,
                       (const double*)h->L, b, j, (const double*)out, h->work);
    }
}

void nlml_reduce(gp_t h)
{
    GPK_LAUNCH(h, GP_PH_REDUCE, k_nlml, 1, NT, 0, (const double*)h->beta, h->n,
               (const double*)h->logdet_part, h->T, h->scal);
}

bool predict_solve(gp_t h, int64_t m, int64_t ldm)
{
    (void)m;
    const int64_t T = h->T, b = h->b;
    const int P = (int)(b / TB);
    const int64_t nq = h->Np / TB;
    if (h->opt.prec == GP_FP64_OZAKI) {   // blocks of GP_OG_SP tile columns, as the factorisation
        for (int64_t J0 = 0; J0 < T; J0 += GP_OG_SP) {
            const int64_t e = J0 + GP_OG_SP < T ? J0 + GP_OG_SP : T;
            for (int64_t j = J0; j < e; ++j)
                if (!og_vsolve_diag(h, j, ldm) || !og_vsolve_update(h, j, e, ldm)) return false;
            if (!og_vsolve_update_sp(h, J0, e, ldm)) return false;
        }
        return true;
    }
    for (int64_t j = 0; j < T; ++j) {
        GPK_LAUNCH(h, GP_PH_VSOLVE, k_diagV, dim3((unsigned)P, (unsigned)(ldm / TB)), NT, DG_SMEM_BYTES,
                   (const double*)h->Linv, (const double*)h->B, h->V, (const double*)h->beta, h->part,
                   b, j, ldm, nq);
        if (j + 1 < T)
            GPK_LAUNCH(h, GP_PH_VSOLVE, k_updV, dim3((unsigned)((T - j - 1) * P), (unsigned)(ldm / TB)),
                       NT, DG_SMEM_BYTES, (const double*)h->L, h->B, (const double*)h->V, b, j, ldm);
    }
    return true;
}

void predict_finish(gp_t h, int64_t m, int64_t ldm, bool want_var)
{
    const int64_t nq = h->Np / TB;
    GPK_LAUNCH(h, GP_PH_REDUCE, k_predict_finish, (unsigned)((m + 255) / 256), 256, 0,
               (const double*)h->part, nq, ldm, m, (const GpHyperDev*)h->hyp, h->opt.noisy_test_var,
               h->outm, want_var ? h->outv : (double*)nullptr);
}

void predict_mean_only(gp_t h, int64_t m, int64_t ldm)
{
    const int64_t chunks = 64, rows_per = (h->Np + chunks - 1) / chunks;
    GPK_LAUNCH(h, GP_PH_REDUCE, k_mean_gemv, dim3((unsigned)((ldm + 255) / 256), (unsigned)chunks), 256,
               0, (const double*)h->B, (const double*)h->alpha, rows_per, h->Np, ldm, h->part);
    GPK_LAUNCH(h, GP_PH_REDUCE, k_sum_rows, (unsigned)((m + 255) / 256), 256, 0,
               (const double*)h->part, chunks, ldm, m, h->outm);
}

bool full_cov(gp_t h, int64_t m, int64_t ldm, double* cov)
{
    assemble_test_prior(h, m, cov);
    if (h->opt.prec == GP_FP64_OZAKI) return og_full_cov(h, m, ldm, cov);
    const int64_t nb = (m + TB - 1) / TB;
    GPK_LAUNCH(h, GP_PH_COV, k_syrk_cov, (unsigned)(nb * (nb + 1) / 2), NT, DG_SMEM_BYTES,
               (const double*)h->V, h->Np, ldm, m, cov);
    return true;
}

bool inverse_tiles(gp_t h)
{
    const int64_t T = h->T, b = h->b;
    const int P = (int)(b / TB);
    GPK_LAUNCH(h, GP_PH_TRTRI, k_copy_diag, grid_for(T * b * b), NT, 0, (const double*)h->Linv,
               h->Xinv, b, T);
    if (h->opt.prec == GP_FP64_OZAKI) {   // exact digit products, blocks of GP_OG_SP row blocks of X
        for (int64_t T0 = 0; T0 < T; T0 += GP_OG_SP) {
            const int64_t e = T0 + GP_OG_SP < T ? T0 + GP_OG_SP : T;
            for (int64_t t = T0; t < e; ++t)
                if ((t > 0 && !og_trtri_scale(h, t)) || !og_trtri_accum(h, t, e)) return false;
            if (!og_trtri_accum_sp(h, T0, e)) return false;
        }
        return og_lauum(h);
    }
    for (int64_t t = 0; t < T; ++t) {
        if (t > 0)
            GPK_LAUNCH(h, GP_PH_TRTRI, k_trtri_scale, dim3((unsigned)P, (unsigned)t), NT, DG_SMEM_BYTES,
                       (const double*)h->Linv, h->Xinv, b, t);
        if (t + 1 < T)
            GPK_LAUNCH(h, GP_PH_TRTRI, k_trtri_accum, dim3((unsigned)((T - t - 1) * (t + 1)), (unsigned)(P * P)),
                       NT, DG_SMEM_BYTES, (const double*)h->L, h->Xinv, b, t);
    }
    GPK_LAUNCH(h, GP_PH_LAUUM, k_lauum, dim3((unsigned)(T * (T + 1) / 2), (unsigned)(P * P)), NT,
               DG_SMEM_BYTES, (const double*)h->Xinv, h->Kinv, b, T);
    return true;
}

void adjoint_grad(gp_t h)
{
    const int64_t T = h->T;
    const int P = (int)(h->b / TB);
    dim3 grid((unsigned)(T * (T + 1) / 2), (unsigned)(P * P));
    if (h->opt.prec == GP_MIXED)
        GPK_LAUNCH(h, GP_PH_ADJOINT, k_adjoint_k, grid, NT, 0, (const float*)h->Kinv32, (const double*)h->L,
                   (const double*)h->alpha, (const double*)h->X, h->n, h->d, h->b, (const GpHyperDev*)h->hyp,
                   h->gpart);
    else
        GPK_LAUNCH(h, GP_PH_ADJOINT, k_adjoint<double>, grid, NT, 0, (const double*)h->Kinv,
                   (const double*)h->alpha, (const double*)h->X, h->n, h->d, h->b, (const GpHyperDev*)h->hyp,
                   h->gpart);
    GPK_LAUNCH(h, GP_PH_REDUCE, k_grad_finish, 1, NT, 0, (const double*)h->gpart,
               (int64_t)grid.x * grid.y, (const GpHyperDev*)h->hyp, h->scal);
}

void adam_step(gp_t h, double lr, double* hist_slot)
{
    GPK_LAUNCH(h, GP_PH_ADAM, k_adam, 1, 32, 0, h->hyp, h->adam, (const double*)h->scal, lr,
               h->opt.adam_beta1, h->opt.adam_beta2, h->opt.adam_eps, h->trainable[0], h->trainable[1],
               h->trainable[2], hist_slot, (const unsigned long long*)h->info);
}

void copy_factor_dense(gp_t h, double* out)
{
    GPK_LAUNCH(h, GP_PH_OTHER, k_factor_dense, grid_for(h->n * h->n), NT, 0, (const double*)h->L,
               h->b, h->n, out);
}

}  // namespace gpk
