// tcgen05 kernels of the mixed-precision path (5th-generation tensor cores,
// accumulators in tensor memory, operands staged by TMA).
//
// k_ozaki_tc: C = Y K for the third-order variance correction.  Y (test rows
// x Np) holds x~0^T, the mixed-factor solution rounded, row by row, to
// GP_OZ_YSLICES signed GP_OZ_BITS-bit digits (k_yslices writes that rounded
// value back, so the correction uses the same x~0 everywhere and is exact
// for it); K (Np x Np, symmetric) is split into GP_OZ_SLICES digits.  Both are
// given as BF16 slices of integer digits (|d| <= 2^GP_OZ_BITS, exact in
// BF16), C = sum over digit pairs (s, u) with s + u <= GP_OZ_LMAX of
// 2^{-GP_OZ_BITS (s+u)} Y_s K_u.  Pairs of equal level l = s + u share one
// FP32 accumulator.  The leading digits are at most 2^GP_OZ_BITS in
// magnitude, the others at most 2^(GP_OZ_BITS-1), so the digit products of
// one level sum to at most 2^(2 GP_OZ_BITS) = 2^14 per k (level 2: d_1 e_1;
// level 3: two products of at most 2^13; higher levels: 2^13 + 2^12), and a
// chunk of OZT_CHUNK = 1024 k stays below 2^24, exact in FP32; each chunk sum
// is added into a double-FP32 (hi + lo) running sum, about 48 bits, held in
// registers.  The fused
// epilogue forms r0 = Kc - C and the partial row sums of Kc x~0 and x~0 r0
// (the terms k*^T x~0 and x~0^T r0 of the corrected variance).
//
// Operand reuse without any cross-CTA traffic: the six levels 2..7 run in
// three groups of two levels; a 32-k stage of a group holds the two Y slices
// and the two or three K slices its pairs need (five 8 KB slots), and all of
// the group's three or four pair products are issued from that one stage, so
// a 128 x 128 x 16 product needs about 5 KB of operands from L2 instead of 8.
//
// Roles (320 threads, one CTA per 128 x 128 output tile): warp 0 issues TMA
// loads into a 5-stage ring; warp 1 owns the 512 TMEM columns (two pairs of
// 128-column level accumulators, used alternately by successive group
// chunks) and issues the MMAs; warps 2-9 (two per TMEM lane quarter, one
// output row and 64 columns per thread) flush each group chunk's two level
// sums into their registers' running sums while the next chunk's MMAs run,
// then run the epilogue.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>
#include <mutex>

#include "gp_internal.cuh"
#include "tc_common.cuh"

namespace gpk {

__device__ int g_tc_error;

namespace {

static_assert(GP_OZ_YSLICES == 2 && GP_OZ_SLICES == 6 && GP_OZ_LMAX == 7 && GP_OZ_BITS == 7,
              "the level groups below are laid out for 2 x 6 slices of 7-bit digits and levels 2..7");

constexpr int OZT_STAGES = 5;
constexpr int OZT_KS = 32;                                 // k per stage
constexpr int OZT_SLOT = 128 * OZT_KS * 2;                 // one 128 x 32 BF16 tile, 64-byte swizzle
constexpr int OZT_STAGE_BYTES = 5 * OZT_SLOT;              // Y_1, Y_2 and up to three K slices
constexpr int OZT_CHUNK = 1024;                            // k per exact chunk
constexpr int OZT_STAGES_PER_CHUNK = OZT_CHUNK / OZT_KS;
constexpr int OZT_GROUPS = 3;                              // levels (2, 3), (4, 5), (6, 7)
constexpr int OZT_THREADS = 320;
constexpr int OZT_EPI_WARPS = 8;
constexpr int OZT_BAR_OFF = OZT_STAGES * OZT_STAGE_BYTES;
constexpr int OZT_SMEM = 1024 + OZT_BAR_OFF + 256;
constexpr int OZT_RASTER = 16;                             // row blocks that share a K column block in flight
constexpr uint32_t OZT_IDESC = tc::idesc_bf16(128, 128);
static_assert(OZT_CHUNK << (2 * GP_OZ_BITS) <= (1 << 24), "a level's chunk sum must stay exact in FP32");
static_assert(OZT_SMEM <= 227 * 1024, "shared memory");

// Lowest K slice (1-based) and number of K slices of group g (levels 2g + 2, 2g + 3):
// group 0 pairs (1,1) | (1,2) (2,1); group 1 (1,3) (2,2) | (1,4) (2,3); group 2 (1,5) (2,4) | (1,6) (2,5).
__host__ __device__ constexpr int grp_u0(int g) { return g == 0 ? 1 : 2 * g; }
__host__ __device__ constexpr int grp_nk(int g) { return g == 0 ? 2 : 3; }

__device__ __forceinline__ bool drain_wait(uint32_t mbar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!tc::mbar_try(mbar, parity))
        if (clock64() - t0 > tc::WAIT_CYCLES) return false;
    return true;
}

__device__ __forceinline__ void mma_first(uint32_t d, uint64_t da, uint64_t db, bool& first)
{
    if (first) tc::mma_bf16(d, da, db, OZT_IDESC, 0u);
    else tc::mma_bf16_acc(d, da, db, OZT_IDESC);
    first = false;
}

// TwoSum (Knuth): hi + lo += x with the rounding error of hi + x kept in lo.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bv = s - hi;
    const float er = (hi - (s - bv)) + (x - bv);
    hi = s;
    lo += er;
}

__global__ __launch_bounds__(OZT_THREADS, 1) void k_ozaki_tc(
    const __grid_constant__ CUtensorMap mapY, const __grid_constant__ CUtensorMap mapK, int64_t ldm, int64_t Np,
    const double* mu, const double* kappa_p, const double* R64, const float* Y, float* Rr32, double* qpart,
    int64_t m, int64_t n_valid, int* err)
{
    extern __shared__ unsigned char dyn[];
    unsigned char* base = dyn + ((1024 - (tc::su32(dyn) & 1023)) & 1023);
    const uint32_t sbase = tc::su32(base);
    const uint32_t bar = sbase + OZT_BAR_OFF;   // full[S], empty[S], accf[2], acce[2], drain
    auto full = [&](int s) { return bar + 8 * s; };
    auto empty = [&](int s) { return bar + 8 * (OZT_STAGES + s); };
    auto accf = [&](int a) { return bar + 8 * (2 * OZT_STAGES + a); };
    auto acce = [&](int a) { return bar + 8 * (2 * OZT_STAGES + 2 + a); };
    const uint32_t drain = bar + 8 * (2 * OZT_STAGES + 4);
    uint32_t* tmem_slot = (uint32_t*)(base + OZT_BAR_OFF + 8 * (2 * OZT_STAGES + 5));
    volatile int* abort = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // grouped raster: OZT_RASTER consecutive CTAs take consecutive row blocks of one column block,
    // so the CTAs in flight share each K column block and each Y row block through L2
    const int64_t nbn = Np / 128, nbm = ldm / 128;
    const int64_t t = blockIdx.x;
    const int64_t first_rb = (t / (OZT_RASTER * nbn)) * OZT_RASTER;
    const int64_t gsz = (nbm - first_rb) < OZT_RASTER ? (nbm - first_rb) : OZT_RASTER;
    const int64_t r_in = t % (OZT_RASTER * nbn);
    const int64_t m0 = (first_rb + r_in % gsz) * 128, n0 = (r_in / gsz) * 128;

    if (threadIdx.x == 0) {
        for (int s = 0; s < OZT_STAGES; ++s) {
            tc::mbar_init(full(s), 1);
            tc::mbar_init(empty(s), 1);
        }
        tc::mbar_init(accf(0), 1);
        tc::mbar_init(accf(1), 1);
        tc::mbar_init(acce(0), OZT_EPI_WARPS);
        tc::mbar_init(acce(1), OZT_EPI_WARPS);
        tc::mbar_init(drain, 1);
        *abort = 0;
        tc::mbar_init_fence();
    }
    if (warp == 1) tc::tmem_alloc(tc::su32(tmem_slot), 512);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    const int kst = (int)(Np / OZT_KS);
    const int nwin = (kst + OZT_STAGES_PER_CHUNK - 1) / OZT_STAGES_PER_CHUNK;   // exact chunks along k

    if (warp == 0) {
        if (lane == 0) {
            int gs = 0;
            bool ok = true;
            const uint64_t pol = tc::policy_evict_last();
            for (int w = 0; w < nwin && ok; ++w) {
                const int k_lo = w * OZT_STAGES_PER_CHUNK;
                const int k_hi = min(kst, k_lo + OZT_STAGES_PER_CHUNK);
                for (int g = 0; g < OZT_GROUPS && ok; ++g) {
                    const int u0 = grp_u0(g), nk = grp_nk(g);
                    for (int k = k_lo; k < k_hi; ++k, ++gs) {
                        const int st = gs % OZT_STAGES, use = gs / OZT_STAGES;
                        if (use > 0 && !tc::mbar_wait(empty(st), (uint32_t)((use - 1) & 1), abort, err)) {
                            ok = false;
                            break;
                        }
                        const uint32_t dst = sbase + st * OZT_STAGE_BYTES;
                        const int kx = k * OZT_KS;
                        tc::mbar_expect_tx(full(st), (uint32_t)((2 + nk) * OZT_SLOT));
                        tc::tma_load_2d_hint(dst, &mapY, kx, (int)m0, full(st), pol);
                        tc::tma_load_2d_hint(dst + OZT_SLOT, &mapY, kx, (int)(ldm + m0), full(st), pol);
                        for (int j = 0; j < nk; ++j)
                            tc::tma_load_2d_hint(dst + (2 + j) * OZT_SLOT, &mapK, kx,
                                                 (int)((u0 - 1 + j) * Np + n0), full(st), pol);
                    }
                }
            }
            if (!ok)   // let the copies in flight land before the CTA exits
                for (int q = gs - 1; q >= 0 && q >= gs - OZT_STAGES; --q)
                    drain_wait(full(q % OZT_STAGES), (uint32_t)((q / OZT_STAGES) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int gs = 0, c = 0;
            bool ok = true;
            constexpr uint64_t slot16 = (uint64_t)(OZT_SLOT >> 4);
            for (int w = 0; w < nwin && ok; ++w) {
                const int k_lo = w * OZT_STAGES_PER_CHUNK;
                const int k_hi = min(kst, k_lo + OZT_STAGES_PER_CHUNK);
                for (int g = 0; g < OZT_GROUPS && ok; ++g, ++c) {
                    const int a = c & 1;
                    if (c >= 2 && !tc::mbar_wait(acce(a), (uint32_t)(((c >> 1) - 1) & 1), abort, err)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const uint32_t d0 = tmem + (uint32_t)(a * 256), d1 = d0 + 128;
                    bool f0 = true, f1 = true;
                    for (int k = k_lo; k < k_hi; ++k, ++gs) {
                        const int st = gs % OZT_STAGES;
                        if (!tc::mbar_wait(full(st), (uint32_t)((gs / OZT_STAGES) & 1), abort, err)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after();
                        const uint64_t y1 = tc::desc_sw64(sbase + st * OZT_STAGE_BYTES);
                        const uint64_t y2 = y1 + slot16, k0 = y1 + 2 * slot16, k1 = k0 + slot16, k2 = k1 + slot16;
#pragma unroll
                        for (int kk = 0; kk < OZT_KS / 16; ++kk) {
                            const uint64_t o = (uint64_t)(2 * kk);   // a 16-k step is 32 bytes
                            if (g == 0) {   // level 2: (1,1); level 3: (1,2), (2,1)
                                mma_first(d0, y1 + o, k0 + o, f0);
                                mma_first(d1, y1 + o, k1 + o, f1);
                                tc::mma_bf16_acc(d1, y2 + o, k0 + o, OZT_IDESC);
                            } else {        // level 2g+2: (1, u0+1), (2, u0); level 2g+3: (1, u0+2), (2, u0+1)
                                mma_first(d0, y1 + o, k1 + o, f0);
                                tc::mma_bf16_acc(d0, y2 + o, k0 + o, OZT_IDESC);
                                mma_first(d1, y1 + o, k2 + o, f1);
                                tc::mma_bf16_acc(d1, y2 + o, k1 + o, OZT_IDESC);
                            }
                        }
                        tc::mma_commit(empty(st));
                    }
                    if (ok) tc::mma_commit(accf(a));
                }
            }
            if (!ok) {   // MMAs in flight finish before TMEM is released
                tc::mma_commit(drain);
                drain_wait(drain, 0);
            }
        }
    } else {
        const int wq = warp & 3, row = wq * 32 + lane, c0 = ((warp - 2) >> 2) * 64;
        const uint32_t tl = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)c0;
        float hi[64], lo[64];
#pragma unroll
        for (int q = 0; q < 64; ++q) hi[q] = lo[q] = 0.f;
        bool ok = true;
        int c = 0;
        for (int w = 0; w < nwin && ok; ++w) {
            for (int g = 0; g < OZT_GROUPS; ++g, ++c) {
                const int a = c & 1;
                ok = __all_sync(0xffffffffu, tc::mbar_wait(accf(a), (uint32_t)((c >> 1) & 1), abort, err));
                if (!ok) break;
                tc::fence_after();
                // 2^{-7 l} for the group's levels l = 2g + 2 and 2g + 3 (normal FP32 powers of two)
                const float sc0 = __int_as_float((127 - GP_OZ_BITS * (2 * g + 2)) << 23);
                const float sc1 = __int_as_float((127 - GP_OZ_BITS * (2 * g + 3)) << 23);
                const uint32_t ta = tl + (uint32_t)(a * 256);
#pragma unroll
                for (int q8 = 0; q8 < 8; ++q8) {
                    float v0[8], v1[8];
                    tc::tmem_ld8x2(ta + 8 * q8, ta + 128 + 8 * q8, v0, v1);
#pragma unroll
                    for (int e = 0; e < 8; ++e) {   // chunk sums are exact; the scaling by 2^-7l too
                        two_sum_acc(hi[8 * q8 + e], lo[8 * q8 + e], v0[e] * sc0);
                        two_sum_acc(hi[8 * q8 + e], lo[8 * q8 + e], v1[e] * sc1);
                    }
                }
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(acce(a));
            }
        }
        // The running sums go back to tensor memory (every MMA has completed: the last
        // chunk's commit covers all earlier ones), so the epilogue below can walk the
        // columns in a rolled loop instead of holding 128 sums in registers.
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
                tc::tmem_st16(tl + 256 + 16 * q, l16);
            }
            tc::tmem_st_wait();
        }
        // fused epilogue, one output row and 64 columns per thread
        const int64_t gm = m0 + row;
        const bool live = ok && gm < m;
        const double sc = live ? mu[gm] * (*kappa_p) : 0.0;
        double s1 = 0.0, s2 = 0.0;
        const double* r64 = R64 + gm * Np + n0 + c0;
        const float* yrow = Y + gm * Np + n0 + c0;
        float* rr = Rr32 + gm * Np + n0 + c0;
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            float h[16], l[16];
            if (ok) tc::tmem_ld16x2(tl + 16 * q, tl + 256 + 16 * q, h, l);
            double kc[16];
            float x[16];
            if (live) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const double2 v = __ldcs((const double2*)(r64 + 16 * q) + e);
                    kc[2 * e] = v.x;
                    kc[2 * e + 1] = v.y;
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float4 v = __ldcs((const float4*)(yrow + 16 * q) + e);
                    x[4 * e] = v.x;
                    x[4 * e + 1] = v.y;
                    x[4 * e + 2] = v.z;
                    x[4 * e + 3] = v.w;
                }
            }
            float outv[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int64_t gn = n0 + c0 + 16 * q + e;
                outv[e] = 0.f;
                if (!ok) {
                    outv[e] = __int_as_float(0x7fc00000);
                } else if (live && gn < n_valid) {
                    const double Cv = ((double)h[e] + (double)l[e]) * sc;
                    const double r = kc[e] - Cv;
                    outv[e] = (float)r;
                    s1 = fma(kc[e], (double)x[e], s1);
                    s2 = fma((double)x[e], r, s2);
                }
            }
#pragma unroll
            for (int e = 0; e < 4; ++e)
                __stcs((float4*)(rr + 16 * q) + e,
                       make_float4(outv[4 * e], outv[4 * e + 1], outv[4 * e + 2], outv[4 * e + 3]));
        }
        if (!ok) s1 = s2 = __longlong_as_double(0x7ff8000000000000ll);
        const int64_t nslot = Np / 64, slot = (n0 + c0) / 64;
        qpart[slot * ldm + gm] = s1;
        qpart[(nslot + slot) * ldm + gm] = s2;
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc::fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
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

// Row-major BF16 matrix (rows x cols, row stride cols) as 32-column x
// 128-row boxes (one 8 KB operand tile), 64-byte swizzle.
bool map_bf16_tiles32(CUtensorMap* map, const void* p, int64_t rows, int64_t cols)
{
    auto enc = encode_fn();
    if (!enc || ((uintptr_t)p & 15) || (cols * 2) % 16 || rows >= (1ll << 31) || cols >= (1ll << 31)) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)OZT_KS, 128}, es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(p), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int* tc_error_dev()
{
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tc_error) != cudaSuccess) return nullptr;
    return (int*)p;
}

bool ozaki_tc(gp_t h, int64_t m, int64_t ldm)
{
    static int done_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (done_dev != dev) {
        cudaFuncSetAttribute(k_ozaki_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, OZT_SMEM);
        done_dev = dev;
    }
    const int64_t Np = h->Np;
    if (Np % 128 || ldm % 128) return false;
    CUtensorMap mY, mK;
    if (!map_bf16_tiles32(&mY, h->YS, GP_OZ_YSLICES * ldm, Np) || !map_bf16_tiles32(&mK, h->KS, GP_OZ_SLICES * Np, Np))
        return false;
    int* err = tc_error_dev();
    if (!err) return false;
    const int64_t tiles = (Np / 128) * (ldm / 128);
    if (tiles >= (1ll << 31)) return false;
    GPK_LAUNCH(h, GP_PH_OZAKI, k_ozaki_tc, (unsigned)tiles, OZT_THREADS, OZT_SMEM, mY, mK, ldm, Np,
               (const double*)h->mu, (const double*)h->kappa, (const double*)h->R64, (const float*)h->R32, h->Rr32,
               h->qpart, m, h->n, err);
    return true;
}

// Reads the tensor-core wait-timeout word (stream-ordered; valid after a
// stream synchronisation) into *out and clears it on the device.
cudaError_t tc_error_fetch(gp_t h, int* out)
{
    int* err = tc_error_dev();
    if (!err) return cudaErrorInvalidSymbol;
    cudaError_t e = cudaMemcpyAsync(out, err, sizeof(int), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), h->st);
    return e;
}

}  // namespace gpk
