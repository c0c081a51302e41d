// tcgen05 kernels of the mixed-precision path (5th-generation tensor cores,
// accumulators in tensor memory, operands staged by TMA).
//
// k_ozaki_tc: C = Y K for the third-order variance correction, Y (test rows x
// Np) and K (Np x Np, symmetric) each given as BF16 slices of signed
// GP_OZ_BITS-bit digits (|d| <= 2^GP_OZ_BITS), C = sum over kept digit pairs
// (s, u) of 2^{-GP_OZ_BITS (s+u)} Y_s K_u.  Each pair's product is summed
// exactly in FP32 over chunks of 2^(24 - 2 GP_OZ_BITS) k (1024 for 7-bit
// digits: a product is at most 2^(2 GP_OZ_BITS), so a chunk sum stays within
// 2^24), and each chunk sum is added into a double-FP32
// (hi + lo) running sum, which carries about 48 bits.  The fused epilogue
// forms r0 = Kc - C and the partial row sums of Kc Y and Y r0 (the terms
// k*^T x0 and x0^T r0 of the corrected variance).
//
// Clusters of 2 x 2 CTAs (two row blocks x two column blocks): the two CTAs
// of a row block share its Y tile and the two of a column block its K tile,
// so each CTA loads half of each (64 rows) and multicasts it to the CTA that
// shares it, halving the operand traffic from L2.  A stage of a CTA's ring is
// written by three CTAs (itself, its Y partner, its K partner) and released
// to all three by a multicast MMA commit; before leaving, a CTA waits for its
// partners' last releases and the cluster synchronises, so no cross-CTA
// arrival or copy can land in a CTA that has exited.
//
// Roles (320 threads, one CTA per SM): warp 0 issues TMA loads into a
// 3-stage ring of 128-k stages {Y tile, K tile} (64 KB per stage, eight
// MMAs per stage and one release commit); warp 1 owns the 512
// TMEM columns and issues the MMAs; warps 2-9 (two per TMEM lane quarter,
// one output row and 64 columns per thread) flush chunk sums and run the
// epilogue.  TMEM columns: two 128-column accumulators used alternately per
// chunk (the MMAs of chunk c+1 run while chunk c is flushed), hi at 256, lo
// at 384.
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

constexpr int OZT_STAGES = 3;
constexpr int OZT_KS = 128;                                      // k per stage
constexpr int OZT_KCH = (1 << (24 - 2 * GP_OZ_BITS)) / OZT_KS;   // stages per exact chunk
constexpr int OZT_THREADS = 320;
constexpr int OZT_EPI_WARPS = 8;
constexpr int OZT_STAGE_BYTES = 4 * tc::TILE_BYTES;            // Y (two 64-k tiles), K (two 64-k tiles)
constexpr int OZT_BAR_OFF = OZT_STAGES * OZT_STAGE_BYTES;
constexpr int OZT_SMEM = 1024 + OZT_BAR_OFF + 256;
constexpr uint32_t OZT_IDESC = tc::idesc_bf16(128, 128);

// p-th kept digit pair (s, u), 1-based, s-major, s + u <= lmax, s, u <= GP_OZ_SLICES.
__device__ __forceinline__ void oz_pair_tc(int p, int lmax, int& s, int& u)
{
    s = 1;
    while (true) {
        const int cnt = max(0, min(GP_OZ_SLICES, lmax - s));
        if (p < cnt) break;
        p -= cnt;
        ++s;
    }
    u = p + 1;
}

__device__ __forceinline__ bool drain_wait(uint32_t mbar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!tc::mbar_try(mbar, parity))
        if (clock64() - t0 > tc::WAIT_CYCLES) return false;
    return true;
}

__global__ __launch_bounds__(OZT_THREADS, 1) void k_ozaki_tc(
    const __grid_constant__ CUtensorMap mapY, const __grid_constant__ CUtensorMap mapK, int64_t ldm, int64_t Np,
    const double* mu, const double* kappa_p, const double* R64, const float* Y, float* Rr32, double* qpart,
    int64_t m, int64_t n_valid, int lmax, int* err)
{
    extern __shared__ unsigned char dyn[];
    unsigned char* base = dyn + ((1024 - (tc::su32(dyn) & 1023)) & 1023);
    const uint32_t sbase = tc::su32(base);
    const uint32_t bar = sbase + OZT_BAR_OFF;   // full[6], empty[6], accf[2], acce[2], drain
    auto full = [&](int s) { return bar + 8 * s; };
    auto empty = [&](int s) { return bar + 8 * (OZT_STAGES + s); };
    auto accf = [&](int a) { return bar + 8 * (2 * OZT_STAGES + a); };
    auto acce = [&](int a) { return bar + 8 * (2 * OZT_STAGES + 2 + a); };
    const uint32_t drain = bar + 8 * (2 * OZT_STAGES + 4);
    uint32_t* tmem_slot = (uint32_t*)(base + OZT_BAR_OFF + 8 * (2 * OZT_STAGES + 5));
    volatile int* abort = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // cluster rank = 2 cm + cn: row block pair member cm, column block pair member cn
    const uint32_t rank = tc::cluster_rank();
    const int cm = (int)(rank >> 1), cn = (int)(rank & 1);
    const uint16_t mask_y = (uint16_t)(3u << (2 * cm)), mask_k = (uint16_t)((1u << cn) | (1u << (cn + 2)));
    const uint16_t mask_rel = (uint16_t)((1u << rank) | (1u << (rank ^ 1)) | (1u << (rank ^ 2)));
    // grouped raster over 2 x 2 block clusters: 4 cluster rows share each cluster column in flight
    const int64_t nbn = Np / 128, nbm = ldm / 128;
    const int64_t nbn2 = (nbn + 1) / 2, nbm2 = (nbm + 1) / 2;
    const int64_t g = blockIdx.x >> 2, G = 4;
    const int64_t grp = g / (G * nbn2), first = grp * G;
    const int64_t gsz = (nbm2 - first) < G ? (nbm2 - first) : G;
    const int64_t mc = first + (g % (G * nbn2)) % gsz, nc = (g % (G * nbn2)) / gsz;
    // odd block counts: the missing block of a pair repeats the last one and stores nothing
    const bool valid = 2 * mc + cm < nbm && 2 * nc + cn < nbn;
    const int64_t mb = min(2 * mc + cm, nbm - 1), nb = min(2 * nc + cn, nbn - 1);
    const int64_t m0 = mb * 128, n0 = nb * 128;

    if (threadIdx.x == 0) {
        for (int s = 0; s < OZT_STAGES; ++s) {
            tc::mbar_init(full(s), 1);
            tc::mbar_init(empty(s), 3);
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
    tc::cluster_sync();   // every barrier of the cluster initialised before any copy or commit
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    int np = 0;
    for (int s = 1; s <= GP_OZ_SLICES; ++s) np += max(0, min(GP_OZ_SLICES, lmax - s));
    const int kst = (int)(Np / OZT_KS);
    const int nkc = (kst + OZT_KCH - 1) / OZT_KCH;   // exact chunks along k; all pairs of a chunk run together

    if (warp == 0) {
        if (lane == 0) {
            int gs = 0;
            bool ok = true;
            const uint64_t pol = tc::policy_evict_last();
            for (int kc = 0; kc < nkc && ok; ++kc)
            for (int p = 0; p < np && ok; ++p) {
                int s, u;
                oz_pair_tc(p, lmax, s, u);
                const int ya = (int)((s - 1) * ldm + m0), kb = (int)((u - 1) * Np + n0);
                for (int k = kc * OZT_KCH; k < min(kst, (kc + 1) * OZT_KCH); ++k, ++gs) {
                    const int st = gs % OZT_STAGES, use = gs / OZT_STAGES;
                    if (use > 0 && !tc::mbar_wait(empty(st), (uint32_t)((use - 1) & 1), abort, err)) {
                        ok = false;
                        break;
                    }
                    const uint32_t dst = sbase + st * OZT_STAGE_BYTES;
                    tc::mbar_expect_tx(full(st), OZT_STAGE_BYTES);   // eight 8 KB halves from three CTAs
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const int kx = k * OZT_KS + 64 * j;
                        tc::tma_load_2d_mc_hint(dst + j * tc::TILE_BYTES + cn * (tc::TILE_BYTES / 2), &mapY, kx,
                                                ya + 64 * cn, full(st), mask_y, pol);
                        tc::tma_load_2d_mc_hint(dst + (2 + j) * tc::TILE_BYTES + cm * (tc::TILE_BYTES / 2), &mapK, kx,
                                                kb + 64 * cm, full(st), mask_k, pol);
                    }
                }
            }
            if (!ok) {   // let the copies in flight land before the CTA exits
                for (int q = gs - 1; q >= 0 && q >= gs - OZT_STAGES; --q)
                    drain_wait(full(q % OZT_STAGES), (uint32_t)((q / OZT_STAGES) & 1));
            }
            // the partners' releases of each stage's last use have landed here
            for (int q = gs - 1; q >= 0 && q >= gs - OZT_STAGES; --q)
                drain_wait(empty(q % OZT_STAGES), (uint32_t)((q / OZT_STAGES) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int gs = 0, c = 0;
            bool ok = true;
            for (int kc = 0; kc < nkc && ok; ++kc) {
                for (int p = 0; p < np && ok; ++p, ++c) {
                    const int k0 = kc * OZT_KCH;
                    const int a = c & 1;
                    if (c >= 2 && !tc::mbar_wait(acce(a), (uint32_t)(((c >> 1) - 1) & 1), abort, err)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const uint32_t d = tmem + (uint32_t)(a * 128);
                    const int k1 = min(kst, k0 + OZT_KCH);
                    for (int k = k0; k < k1; ++k, ++gs) {
                        const int st = gs % OZT_STAGES;
                        if (!tc::mbar_wait(full(st), (uint32_t)((gs / OZT_STAGES) & 1), abort, err)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after();
                        // descriptors of the stage's first Y and K tiles; a 16-k step adds 32 bytes (2 in the
                        // address field) inside a 64-k tile, the second 64-k tile starts TILE_BYTES on
                        const uint64_t da = tc::desc_sw128(sbase + st * OZT_STAGE_BYTES);
                        const uint64_t db = da + (uint64_t)((2 * tc::TILE_BYTES) >> 4);
                        constexpr uint64_t tstep = (uint64_t)(tc::TILE_BYTES >> 4);
                        if (k == k0) tc::mma_bf16(d, da, db, OZT_IDESC, 0u);
                        else tc::mma_bf16_acc(d, da, db, OZT_IDESC);
#pragma unroll
                        for (int kk = 1; kk < 8; ++kk) {
                            const uint64_t off = (uint64_t)((kk >> 2) * tstep + 2 * (kk & 3));
                            tc::mma_bf16_acc(d, da + off, db + off, OZT_IDESC);
                        }
                        tc::mma_commit_mc(empty(st), mask_rel);
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
        const uint32_t lrow = (uint32_t)(wq * 32) << 16;
        const uint32_t t_hi = tmem + lrow + 256, t_lo = tmem + lrow + 384;
        bool ok = true;
        int c = 0;
        for (int kc = 0; kc < nkc && ok; ++kc) {
            for (int p = 0; p < np; ++p, ++c) {
                int s, u;
                oz_pair_tc(p, lmax, s, u);
                const float scale = ldexpf(1.f, -GP_OZ_BITS * (s + u));
                const int a = c & 1;
                ok = __all_sync(0xffffffffu, tc::mbar_wait(accf(a), (uint32_t)((c >> 1) & 1), abort, err));
                if (!ok) break;
                tc::fence_after();
                const uint32_t t_acc = tmem + lrow + (uint32_t)(a * 128);
#pragma unroll 1
                for (int col = c0; col < c0 + 64; col += 16) {
                    float v[16], hi[16], lo[16];
                    tc::tmem_ld16(t_acc + col, v);
                    if (c == 0) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            hi[q] = v[q] * scale;
                            lo[q] = 0.f;
                        }
                    } else {
                        tc::tmem_ld16(t_hi + col, hi);
                        tc::tmem_ld16(t_lo + col, lo);
#pragma unroll
                        for (int q = 0; q < 16; ++q) {   // TwoSum of an exact term into hi + lo
                            const float x = v[q] * scale;
                            const float sm = hi[q] + x;
                            const float bv = sm - hi[q];
                            const float er = (hi[q] - (sm - bv)) + (x - bv);
                            hi[q] = sm;
                            lo[q] += er;
                        }
                    }
                    tc::tmem_st16(t_hi + col, hi);
                    tc::tmem_st16(t_lo + col, lo);
                }
                tc::tmem_st_wait();
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(acce(a));
            }
        }
        // fused epilogue, one output row and 64 columns per thread
        const int64_t gm = m0 + row;
        const bool live = ok && valid && gm < m;
        const double sc = live ? mu[gm] * (*kappa_p) : 0.0;
        double s1 = 0.0, s2 = 0.0;
        const double* r64 = R64 + gm * Np + n0;
        const float* yrow = Y + gm * Np + n0;
        float* rr = Rr32 + gm * Np + n0;
#pragma unroll 1
        for (int col = c0; col < c0 + 64; col += 16) {
            float hi[16], lo[16];
            if (ok) {
                tc::tmem_ld16(t_hi + col, hi);
                tc::tmem_ld16(t_lo + col, lo);
            }
            if (!valid) continue;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int64_t gn = n0 + col + q;
                float outv = 0.f;
                if (!ok) {
                    outv = __int_as_float(0x7fc00000);
                } else if (live && gn < n_valid) {
                    const double Cv = ((double)hi[q] + (double)lo[q]) * sc;
                    const double kc = r64[col + q], x = (double)yrow[col + q];
                    const double r = kc - Cv;
                    outv = (float)r;
                    s1 = fma(kc, x, s1);
                    s2 = fma(x, r, s2);
                }
                rr[col + q] = outv;
            }
        }
        if (!ok) s1 = s2 = __longlong_as_double(0x7ff8000000000000ll);
        if (valid) {
            const int64_t nslot = Np / 64, slot = (n0 + c0) / 64;
            qpart[slot * ldm + gm] = s1;
            qpart[(nslot + slot) * ldm + gm] = s2;
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::cluster_sync();   // no partner still sends copies or releases into this CTA
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

// Row-major BF16 matrix (rows x cols, row stride cols) as 64 x 64 boxes
// (half operand tiles), 128-byte swizzle.
bool map_bf16_tiles(CUtensorMap* map, const void* p, int64_t rows, int64_t cols)
{
    auto enc = encode_fn();
    if (!enc || ((uintptr_t)p & 15) || (cols * 2) % 16 || rows >= (1ll << 31)) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {64, 64}, es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(p), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
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
    CUtensorMap mY, mK;
    if (!map_bf16_tiles(&mY, h->YS, GP_OZ_SLICES * ldm, Np) || !map_bf16_tiles(&mK, h->KS, GP_OZ_SLICES * Np, Np))
        return false;
    int* err = tc_error_dev();
    if (!err) return false;
    const int64_t nbn2 = (Np / 128 + 1) / 2, nbm2 = (ldm / 128 + 1) / 2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(4 * nbn2 * nbm2));
    cfg.blockDim = dim3(OZT_THREADS);
    cfg.dynamicSmemBytes = OZT_SMEM;
    cfg.stream = h->st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 4;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool p_ = h->prof_on && prof_begin(h, GP_PH_OZAKI);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_ozaki_tc, mY, mK, ldm, Np, (const double*)h->mu,
                                             (const double*)h->kappa, (const double*)h->R64, (const float*)h->R32,
                                             h->Rr32, h->qpart, m, h->n, h->oz_lmax, err);
    h->launches++;
    if (p_) prof_end(h);
    return e == cudaSuccess;
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
