// Squared distances on the tensor cores for many regressors (mixed path).
//
// Eq. 2 needs r^2_ij = |z_i - z_j|^2 for every pair of training points (the
// K tiles), every (test, training) pair (K_{Z*,Z}) and every pair of test
// points (K_{Z*,Z*}).  With d regressors the direct differences cost 3d FP64
// operations per element, which bound the assembly at d = 128.  Written as
// r^2_ij = |z_i|^2 + |z_j|^2 - 2 z_i . z_j, the inner products form a matrix
// product of rank d, taken here as an exact digit product on the BF16 tensor
// cores (the scheme of the variance correction, kernels_tc.cu):
//
//  - each row, shifted by a common origin (the first training row for the K
//    tiles and K_{Z*,Z}, the first test row for K_{Z*,Z*}), is scaled by
//    mu = a power of two >= max_k |z_k| and rounded to
//    42 bits, zhat = q mu 2^-42 (k_zslices); q is split into six balanced
//    7-bit digits (|d| <= 2^7, exact in BF16) and |zhat|^2 is summed in FP64;
//  - zhat_i . zhat_j = mu_i mu_j sum over digit pairs (s, u), s + u <= 8, of
//    2^{-7(s+u)} (D_s D_u^T)_ij; the pairs of one level l = s + u share one
//    FP32 TMEM accumulator, at most six pairs x 128 k per exact chunk
//    (6 x 128 x 2^14 < 2^24), and the chunk sums are added into double-FP32
//    running sums in registers;
//  - the epilogue forms r^2 = |zhat_i|^2 + |zhat_j|^2 - 2 zhat_i . zhat_j
//    (clamped at 0, exactly 0 on the diagonal of K), the kernel value
//    (Eq. 2 or a Matern kernel, kfun.cuh) in FP64 and writes the output of
//    its mode.
//
// The rounding of z to 42 bits moves r^2 by about 2^-42 |z| |z_i - z_j| and
// the dropped digit pairs by about d 2^-56 mu_i mu_j: both far below the FP64
// rounding of K for the mixed path's 1e-8 target.
//
// Roles as in k_ozaki_tc (320 threads, one CTA per 128 x 128 output block):
// warp 0 loads, per 32-k stage, the A and B digit slices that the current
// level's pairs use (twelve 8 KB slots, 64-byte swizzle, two stages); warp 1
// issues the level's pair products into one of two 128-column accumulators;
// warps 2-9 flush each (level, chunk) sum into their registers and then run
// the epilogue.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "gp_internal.cuh"
#include "kfun.cuh"
#include "se_common.cuh"
#include "tc_common.cuh"

namespace gpk {
namespace {

constexpr int ZD_SLICES = 6;                                 // digits per quantised row (42 bits)
constexpr int ZD_LMIN = 2, ZD_LMAX = 8;                      // levels s + u kept
constexpr int ZD_KS = 32;                                    // k per stage
constexpr int ZD_SLOT = 128 * ZD_KS * 2;                     // one 128 x 32 BF16 tile (8 KB)
constexpr int ZD_STAGE_BYTES = 2 * ZD_SLICES * ZD_SLOT;      // A slices 1..6, B slices 1..6
constexpr int ZD_STAGES = 2;
constexpr int ZD_CHUNK = 128;                                // k per exact chunk
constexpr int ZD_THREADS = 320;
constexpr int ZD_EPI_WARPS = 8;
constexpr int ZD_BAR_OFF = ZD_STAGES * ZD_STAGE_BYTES;
constexpr int ZD_SMEM = 1024 + ZD_BAR_OFF + 256;
constexpr uint32_t ZD_IDESC = tc::idesc_bf16(128, 128);
static_assert(ZD_SMEM <= 227 * 1024, "shared memory");
static_assert(6 * ZD_CHUNK * (1 << 14) <= (1 << 24), "a level's chunk sum must stay exact in FP32");

// Digit pairs of level l: s from smin(l) to smax(l), u = l - s, 1 <= s, u <= 6.
__host__ __device__ constexpr int zd_smin(int l) { return l - ZD_SLICES > 1 ? l - ZD_SLICES : 1; }
__host__ __device__ constexpr int zd_smax(int l) { return l - 1 < ZD_SLICES ? l - 1 : ZD_SLICES; }

enum { ZD_TRAIN = 0, ZD_CROSS = 1, ZD_PRIOR = 2 };

struct DistOp {
    int mode;
    int64_t a_ps, b_ps;            // rows between digit slices of the A / B arrays
    int64_t dp;                    // padded regressor count (multiple of 32)
    const double *muA, *muB;       // row scales
    const double *nA, *nB;         // |zhat|^2 of the rows
    int64_t na, nb;                // valid rows of A and B
    const GpHyperDev* hyp;
    // ZD_TRAIN: lower K tiles (FP64) and their FP32 copy
    double* L;
    float* A32;
    int64_t b;
    int P;                         // 128-row blocks per tile edge
    // ZD_CROSS: K_{Z*,Z} in FP32 and FP64 (row stride ldr) and mean partials
    float* R32;
    double* R64;
    int64_t ldr;
    double* mpart;
    int64_t ldp;
    const double* alpha;
    // ZD_PRIOR: K_{Z*,Z*} (+ sigma^2 I when noisy), row stride ldc
    double* cov;
    int64_t ldc;
    int noisy;
};

__device__ __forceinline__ bool zd_drain(uint32_t mbar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!tc::mbar_try(mbar, parity))
        if (clock64() - t0 > tc::WAIT_CYCLES) return false;
    return true;
}

__device__ __forceinline__ void zd_two_sum(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bv = s - hi;
    const float er = (hi - (s - bv)) + (x - bv);
    hi = s;
    lo += er;
}

__global__ __launch_bounds__(ZD_THREADS, 1) void k_dist_tc(const __grid_constant__ CUtensorMap mapA,
                                                          const __grid_constant__ CUtensorMap mapB, const DistOp op,
                                                          int* err)
{
    // output block: A rows r0 .. r0 + 127, B rows c0 .. c0 + 127
    int64_t r0, c0, ti = 0, tj = 0;
    int rb = 0, cb = 0;
    if (op.mode == ZD_TRAIN) {
        tri_decode(blockIdx.x, ti, tj);
        rb = (int)blockIdx.y / op.P;
        cb = (int)blockIdx.y % op.P;
        if (ti == tj && cb > rb) return;   // upper blocks of a diagonal tile are never read
        r0 = ti * op.b + rb * 128;
        c0 = tj * op.b + cb * 128;
    } else {
        r0 = (int64_t)blockIdx.y * 128;
        c0 = (int64_t)blockIdx.x * 128;
    }

    extern __shared__ unsigned char dyn[];
    unsigned char* base = dyn + ((1024 - (tc::su32(dyn) & 1023)) & 1023);
    const uint32_t sbase = tc::su32(base);
    const uint32_t bar = sbase + ZD_BAR_OFF;   // full[S], empty[S], accf[2], acce[2], drain
    auto full = [&](int s) { return bar + 8 * s; };
    auto empty = [&](int s) { return bar + 8 * (ZD_STAGES + s); };
    auto accf = [&](int a) { return bar + 8 * (2 * ZD_STAGES + a); };
    auto acce = [&](int a) { return bar + 8 * (2 * ZD_STAGES + 2 + a); };
    const uint32_t drain = bar + 8 * (2 * ZD_STAGES + 4);
    uint32_t* tmem_slot = (uint32_t*)(base + ZD_BAR_OFF + 8 * (2 * ZD_STAGES + 5));
    volatile int* abort = (volatile int*)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ZD_STAGES; ++s) {
            tc::mbar_init(full(s), 1);
            tc::mbar_init(empty(s), 1);
        }
        tc::mbar_init(accf(0), 1);
        tc::mbar_init(accf(1), 1);
        tc::mbar_init(acce(0), ZD_EPI_WARPS);
        tc::mbar_init(acce(1), ZD_EPI_WARPS);
        tc::mbar_init(drain, 1);
        *abort = 0;
        tc::mbar_init_fence();
    }
    if (warp == 1) tc::tmem_alloc(tc::su32(tmem_slot), 256);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    const int kst = (int)(op.dp / ZD_KS);                              // 32-k stages along the regressors
    const int spc = ZD_CHUNK / ZD_KS;                                  // stages per exact chunk
    const int nch = (kst + spc - 1) / spc;

    if (warp == 0) {
        if (lane == 0) {
            int gs = 0;
            bool ok = true;
            for (int l = ZD_LMIN; l <= ZD_LMAX && ok; ++l) {
                const int s0 = zd_smin(l), s1 = zd_smax(l);
                for (int c = 0; c < nch && ok; ++c)
                    for (int k = c * spc; k < min(kst, (c + 1) * spc); ++k, ++gs) {
                        const int st = gs % ZD_STAGES, use = gs / ZD_STAGES;
                        if (use > 0 && !tc::mbar_wait(empty(st), (uint32_t)((use - 1) & 1), abort, err)) {
                            ok = false;
                            break;
                        }
                        const uint32_t dst = sbase + st * ZD_STAGE_BYTES;
                        tc::mbar_expect_tx(full(st), (uint32_t)(2 * (s1 - s0 + 1) * ZD_SLOT));
                        for (int s = s0; s <= s1; ++s) {
                            const int u = l - s;
                            tc::tma_load_2d(dst + (s - 1) * ZD_SLOT, &mapA, k * ZD_KS, (int)((s - 1) * op.a_ps + r0),
                                            full(st));
                            tc::tma_load_2d(dst + (ZD_SLICES + u - 1) * ZD_SLOT, &mapB, k * ZD_KS,
                                            (int)((u - 1) * op.b_ps + c0), full(st));
                        }
                    }
            }
            if (!ok)   // let the copies in flight land before the CTA exits
                for (int q = gs - 1; q >= 0 && q >= gs - ZD_STAGES; --q)
                    zd_drain(full(q % ZD_STAGES), (uint32_t)((q / ZD_STAGES) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int gs = 0, un = 0;
            bool ok = true;
            constexpr uint64_t slot16 = (uint64_t)(ZD_SLOT >> 4);
            for (int l = ZD_LMIN; l <= ZD_LMAX && ok; ++l) {
                const int s0 = zd_smin(l), s1 = zd_smax(l);
                for (int c = 0; c < nch && ok; ++c, ++un) {
                    const int a = un & 1;
                    if (un >= 2 && !tc::mbar_wait(acce(a), (uint32_t)(((un >> 1) - 1) & 1), abort, err)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const uint32_t d = tmem + (uint32_t)(a * 128);
                    bool first = true;
                    for (int k = c * spc; k < min(kst, (c + 1) * spc); ++k, ++gs) {
                        const int st = gs % ZD_STAGES;
                        if (!tc::mbar_wait(full(st), (uint32_t)((gs / ZD_STAGES) & 1), abort, err)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after();
                        const uint64_t d0 = tc::desc_sw64(sbase + st * ZD_STAGE_BYTES);
#pragma unroll
                        for (int kk = 0; kk < ZD_KS / 16; ++kk)
                            for (int s = s0; s <= s1; ++s) {
                                const uint64_t da = d0 + (uint64_t)(s - 1) * slot16 + 2 * kk;
                                const uint64_t db = d0 + (uint64_t)(ZD_SLICES + l - s - 1) * slot16 + 2 * kk;
                                if (first) tc::mma_bf16(d, da, db, ZD_IDESC, 0u);
                                else tc::mma_bf16_acc(d, da, db, ZD_IDESC);
                                first = false;
                            }
                        tc::mma_commit(empty(st));
                    }
                    if (ok) tc::mma_commit(accf(a));
                }
            }
            if (!ok) {   // MMAs in flight finish before TMEM is released
                tc::mma_commit(drain);
                zd_drain(drain, 0);
            }
        }
    } else {
        const int wq = warp & 3, row = wq * 32 + lane, cq = ((warp - 2) >> 2) * 64;
        const uint32_t tl = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)cq;
        float hi[64], lo[64];
#pragma unroll
        for (int q = 0; q < 64; ++q) hi[q] = lo[q] = 0.f;
        bool ok = true;
        int un = 0;
        for (int l = ZD_LMIN; l <= ZD_LMAX && ok; ++l) {
            const float sc = __int_as_float((127 - 7 * l) << 23);   // 2^{-7 l}
            for (int c = 0; c < nch; ++c, ++un) {
                const int a = un & 1;
                ok = __all_sync(0xffffffffu, tc::mbar_wait(accf(a), (uint32_t)((un >> 1) & 1), abort, err));
                if (!ok) break;
                tc::fence_after();
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    float v[16];
                    tc::tmem_ld16(tl + (uint32_t)(a * 128) + 16 * q4, v);
#pragma unroll
                    for (int e = 0; e < 16; ++e) zd_two_sum(hi[16 * q4 + e], lo[16 * q4 + e], v[e] * sc);
                }
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(acce(a));
            }
        }
        // every MMA has completed (the last unit's commit covers the earlier ones): the
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
        const double nu = op.hyp->nu, s2 = op.hyp->s2;
        const double nanv = __longlong_as_double(0x7ff8000000000000ll);
        const int64_t gi = r0 + row;
        const double mi = op.muA[gi], ni = op.nA[gi];
        double msum = 0.0;
#pragma unroll 1
        for (int q = 0; q < 8; ++q) {   // eight columns at a time
            float h[8], lw[8];
            if (ok) tc::tmem_ld8x2(tl + 8 * q, tl + 128 + 8 * q, h, lw);
            double v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int64_t gj = c0 + cq + 8 * q + e;
                const double G = ((double)h[e] + (double)lw[e]) * (mi * op.muB[gj]);
                const double r2 = fmax(ni + op.nB[gj] - 2.0 * G, 0.0);
                double kv;
                if (op.mode == ZD_TRAIN) {
                    if (gi < op.na && gj < op.na) kv = gi == gj ? nu + s2 : kval(r2, op.hyp);
                    else kv = gi == gj ? 1.0 : 0.0;
                } else if (op.mode == ZD_CROSS) {
                    kv = (gi < op.na && gj < op.nb) ? kval(r2, op.hyp) : 0.0;
                    if (gj < op.nb) msum = fma(kv, op.alpha[gj], msum);
                } else {
                    kv = gi == gj ? nu + (op.noisy ? s2 : 0.0) : kval(r2, op.hyp);
                }
                v[e] = ok ? kv : nanv;
            }
            if (op.mode == ZD_TRAIN) {
                const int64_t o = tri_index(ti, tj) * op.b * op.b + (int64_t)(rb * 128 + row) * op.b + cb * 128 + cq +
                                  8 * q;
#pragma unroll
                for (int e = 0; e < 4; ++e) __stcs((double2*)(op.L + o) + e, make_double2(v[2 * e], v[2 * e + 1]));
                if (op.A32)
#pragma unroll
                    for (int e = 0; e < 2; ++e)
                        __stcs((float4*)(op.A32 + o) + e, make_float4((float)v[4 * e], (float)v[4 * e + 1],
                                                                      (float)v[4 * e + 2], (float)v[4 * e + 3]));
            } else if (op.mode == ZD_CROSS) {
                const int64_t o = gi * op.ldr + c0 + cq + 8 * q;
                if (op.R64)
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        __stcs((double2*)(op.R64 + o) + e, make_double2(v[2 * e], v[2 * e + 1]));
#pragma unroll
                for (int e = 0; e < 2; ++e)
                    __stcs((float4*)(op.R32 + o) + e, make_float4((float)v[4 * e], (float)v[4 * e + 1],
                                                                  (float)v[4 * e + 2], (float)v[4 * e + 3]));
            } else if (gi < op.na) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int64_t gj = c0 + cq + 8 * q + e;
                    if (gj < op.nb) op.cov[gi * op.ldc + gj] = v[e];
                }
            }
        }
        if (op.mode == ZD_CROSS) op.mpart[((c0 + cq) / 64) * op.ldp + gi] = ok ? msum : nanv;
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc::fence_after();
        tc::tmem_dealloc(tmem, 256);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 zd_encode_fn()
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

// Digit slices (ZD_SLICES x rows x dp BF16, slice-major) as one 2-D map of
// 32-column x 128-row boxes, 64-byte swizzle.
bool zd_map(CUtensorMap* map, const void* p, int64_t rows, int64_t dp)
{
    auto enc = zd_encode_fn();
    const int64_t all = ZD_SLICES * rows;
    if (!enc || ((uintptr_t)p & 15) || dp % ZD_KS || rows % 128 || all >= (1ll << 31)) return false;
    cuuint64_t dims[2] = {(cuuint64_t)dp, (cuuint64_t)all};
    cuuint64_t strides[1] = {(cuuint64_t)dp * 2};
    cuuint32_t box[2] = {(cuuint32_t)ZD_KS, 128}, es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(p), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool zd_launch(gp_t h, int phase, const CUtensorMap& mA, const CUtensorMap& mB, const DistOp& op, dim3 grid)
{
    static int done_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (done_dev != dev) {
        cudaFuncSetAttribute(k_dist_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, ZD_SMEM);
        done_dev = dev;
    }
    int* err = tc_error_dev();
    if (!err) return false;
    GPK_LAUNCH(h, phase, k_dist_tc, grid, ZD_THREADS, ZD_SMEM, mA, mB, op, err);
    h->tc_pending = true;
    return true;
}

DistOp zd_base(gp_t h)
{
    DistOp op;
    memset(&op, 0, sizeof(op));
    op.dp = h->dp;
    op.hyp = (const GpHyperDev*)h->hyp;
    return op;
}

}  // namespace

bool use_tc_dist(gp_t h) { return h->opt.prec == GP_MIXED && h->d >= GP_TC_DIST_MIN_D; }

// K tiles (FP64 into h->L, FP32 copy into h->A32) from the training digits.
bool dist_train_tc(gp_t h)
{
    CUtensorMap mX;
    if (!zd_map(&mX, h->ZXS, h->Np, h->dp)) return false;
    DistOp op = zd_base(h);
    op.mode = ZD_TRAIN;
    op.a_ps = op.b_ps = h->Np;
    op.muA = op.muB = h->zx_mu;
    op.nA = op.nB = h->zx_nrm;
    op.na = op.nb = h->n;
    op.L = h->L;
    op.A32 = h->A32;
    op.b = h->b;
    op.P = (int)(h->b / 128);
    return zd_launch(h, GP_PH_ASSEMBLE, mX, mX, op, dim3((unsigned)(h->T * (h->T + 1) / 2), (unsigned)(op.P * op.P)));
}

// K_{Z*,Z} into R32 / R64 (row stride Np) and the mean partials from the test
// digits (h->ZSS, sliced by the caller) and the training digits.
bool dist_cross_tc(gp_t h, int64_t m, int64_t ldm)
{
    CUtensorMap mA, mB;
    if (!zd_map(&mA, h->ZSS, ldm, h->dp) || !zd_map(&mB, h->ZXS, h->Np, h->dp)) return false;
    DistOp op = zd_base(h);
    op.mode = ZD_CROSS;
    op.a_ps = ldm;
    op.b_ps = h->Np;
    op.muA = h->zs_mu;
    op.nA = h->zs_nrm;
    op.muB = h->zx_mu;
    op.nB = h->zx_nrm;
    op.na = m;
    op.nb = h->n;
    op.R32 = h->R32;
    op.R64 = h->R64;
    op.ldr = h->Np;
    op.mpart = h->mpart;
    op.ldp = ldm;
    op.alpha = h->alpha;
    return zd_launch(h, GP_PH_CROSS, mA, mB, op, dim3((unsigned)(h->Np / 128), (unsigned)(ldm / 128)));
}

// K_{Z*,Z*} (+ sigma^2 on the diagonal when noisy) into out (m x m) from the test digits.
bool dist_prior_tc(gp_t h, int64_t m, int64_t ldm, double* out)
{
    CUtensorMap mA;
    if (!zd_map(&mA, h->ZSS, ldm, h->dp)) return false;
    DistOp op = zd_base(h);
    op.mode = ZD_PRIOR;
    op.a_ps = op.b_ps = ldm;
    op.muA = op.muB = h->zs_mu;
    op.nA = op.nB = h->zs_nrm;
    op.na = op.nb = m;
    op.cov = out;
    op.ldc = m;
    op.noisy = h->opt.noisy_test_var;
    return zd_launch(h, GP_PH_COV, mA, mA, op, dim3((unsigned)(ldm / 128), (unsigned)(ldm / 128)));
}

}  // namespace gpk
