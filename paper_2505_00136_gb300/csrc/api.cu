// C ABI entry points (include/gprat_gb.h): handle lifecycle, argument
// validation, host/device pointer detection and stream-ordered orchestration
// of the kernels.  No call throws; every failure becomes a gp_status.
#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "gp_internal.cuh"

namespace {

constexpr int64_t TB = GP_TB;

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// True when this device's kernels may address p directly: managed memory or
// device memory of the current device.  Device memory of another GPU is then
// handled like host memory, through staging buffers and cudaMemcpyDefault
// copies, so no kernel dereferences it without peer access.
bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    int dev = -1;
    return a.type == cudaMemoryTypeDevice && cudaGetDevice(&dev) == cudaSuccess && a.device == dev;
}

gp_status cuda_status(gp_t h, cudaError_t e)
{
    if (e == cudaSuccess) return GP_OK;
    if (h) h->last_info = (int64_t)e;
    return e == cudaErrorMemoryAllocation ? GP_ERR_OOM : GP_ERR_CUDA;
}

gp_status check_launch(gp_t h)
{
    if (h->host_fail) {   // a launch that could not be set up on the host (tensor-map encoding)
        h->host_fail = false;
        return GP_ERR_CUDA;
    }
    return cuda_status(h, cudaGetLastError());
}

template <class T>
gp_status dev_alloc(gp_t h, T** p, int64_t count)
{
    *p = nullptr;
    if (count <= 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, (size_t)count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return cuda_status(h, e);
    }
    h->bytes += count * (int64_t)sizeof(T);
    return GP_OK;
}

template <class T>
void dev_free(gp_t h, T** p, int64_t count)
{
    if (*p) {
        cudaFree(*p);
        h->bytes -= (count <= 0 ? 1 : count) * (int64_t)sizeof(T);
    }
    *p = nullptr;
}

int64_t ntri(gp_t h) { return h->T * (h->T + 1) / 2; }

bool hyper_ok(const gp_hyper* hp)
{
    return hp && isfinite(hp->lengthscale) && isfinite(hp->vertical) && isfinite(hp->noise_var) &&
           hp->lengthscale > 0.0 && hp->vertical > 0.0 && hp->noise_var >= 0.0;
}

void hyper_to_dev(const gp_hyper* hp, GpHyperDev* d)
{
    d->l = hp->lengthscale;
    d->nu = hp->vertical;
    d->s2 = hp->noise_var;
    d->inv2l2 = 1.0 / (2.0 * hp->lengthscale * hp->lengthscale);
    d->log_theta[0] = log(hp->lengthscale);
    d->log_theta[1] = log(hp->vertical);
    d->log_theta[2] = hp->noise_var > 0.0 ? log(hp->noise_var) : -INFINITY;
}

gp_status sync(gp_t h) { return cuda_status(h, cudaStreamSynchronize(h->st)); }

// Copies `count` doubles between any two of {host, device} memory on h's stream.
gp_status copy_any(gp_t h, void* dst, const void* src, int64_t count)
{
    if (count <= 0) return GP_OK;
    return cuda_status(h, cudaMemcpyAsync(dst, src, (size_t)count * sizeof(double), cudaMemcpyDefault, h->st));
}

gp_status ensure_grad_buffers(gp_t h)
{
    gp_status s;
    const int64_t tiles = ntri(h) * h->b * h->b;
    const int64_t P = h->b / TB;
    if (h->opt.prec == GP_MIXED) {
        if (h->ZP) return GP_OK;
        if ((s = dev_alloc(h, &h->ZP, 3 * tiles)) != GP_OK) return s;
        if ((s = dev_alloc(h, &h->U32, tiles)) != GP_OK) return s;
        if ((s = dev_alloc(h, &h->Kinv32, tiles)) != GP_OK) return s;
        h->gpart_cap = ntri(h) * P * P * 3;
        return dev_alloc(h, &h->gpart, h->gpart_cap);
    }
    if (h->Xinv) return GP_OK;
    if (h->opt.prec == GP_FP64_OZAKI) {   // column digit slices of L^{-1} for the emulated inverse
        const int64_t Np = h->Np;
        if ((s = dev_alloc(h, &h->OGT, (int64_t)gpk::GP_OG_SLICES * Np * h->b)) != GP_OK) return s;
        if ((s = dev_alloc(h, &h->ogt_mu, Np)) != GP_OK) return s;
        if ((s = dev_alloc(h, &h->OGTS, (int64_t)gpk::GP_OG_SLICES * Np * gpk::GP_OG_SP * h->b)) != GP_OK) return s;
        if ((s = dev_alloc(h, &h->OGX, (int64_t)gpk::GP_OG_SLICES * Np * Np)) != GP_OK) return s;
        if ((s = dev_alloc(h, &h->ogx_mu, Np)) != GP_OK) return s;
        if ((s = dev_alloc(h, &h->ogx_bits, Np)) != GP_OK) return s;
    }
    if ((s = dev_alloc(h, &h->Xinv, tiles)) != GP_OK) return s;
    if ((s = dev_alloc(h, &h->Kinv, tiles)) != GP_OK) return s;
    h->gpart_cap = ntri(h) * P * P * 3;
    return dev_alloc(h, &h->gpart, h->gpart_cap);
}

gp_status ensure_predict_space_mixed(gp_t h, int64_t m)
{
    const int64_t ldm = round_up(m, 2 * TB);
    if (ldm <= h->m_cap) return GP_OK;
    const int64_t old = h->m_cap;
    dev_free(h, &h->Xs, old * h->d);
    dev_free(h, &h->R32, old * h->Np);
    dev_free(h, &h->RP, 3 * old * gpk::GP_SOLVE_SB * h->b);
    dev_free(h, &h->WP, 3 * old * h->Np);
    dev_free(h, &h->mpart, old * (h->Np / TB));
    dev_free(h, &h->vpart, old * (h->Np / 64));
    dev_free(h, &h->outm, old);
    dev_free(h, &h->outv, old);
    dev_free(h, &h->R64, old * h->Np);
    dev_free(h, &h->Rr32, old * h->Np);
    dev_free(h, &h->YS, (int64_t)gpk::GP_OZ_YSLICES * old * h->Np);
    dev_free(h, &h->mu, old);
    dev_free(h, &h->qpart, 2 * old * (h->Np / 64));
    dev_free(h, &h->vpart2, old * (h->Np / 64));
    dev_free(h, &h->ZSS, 6 * old * h->dp);
    dev_free(h, &h->zs_mu, old);
    dev_free(h, &h->zs_nrm, old);
    h->m_cap = 0;
    gp_status s;
    if ((s = dev_alloc(h, &h->Xs, ldm * h->d)) != GP_OK) return s;
    if ((s = dev_alloc(h, &h->R32, ldm * h->Np)) != GP_OK) return s;
    if (h->opt.var_correction) {
        if ((s = dev_alloc(h, &h->R64, ldm * h->Np)) != GP_OK) return s;
        if ((s = dev_alloc(h, &h->Rr32, ldm * h->Np)) != GP_OK) return s;
        if ((s = dev_alloc(h, &h->YS, (int64_t)gpk::GP_OZ_YSLICES * ldm * h->Np)) != GP_OK) return s;
        if ((s = dev_alloc(h, &h->mu, ldm)) != GP_OK) return s;
        if ((s = dev_alloc(h, &h->qpart, 2 * ldm * (h->Np / 64))) != GP_OK) return s;   // one slot per 64 columns
        if ((s = dev_alloc(h, &h->vpart2, ldm * (h->Np / 64))) != GP_OK) return s;   // one slot per 64 columns
    }
    if ((s = dev_alloc(h, &h->RP, 3 * ldm * gpk::GP_SOLVE_SB * h->b)) != GP_OK) return s;   // one super-block
    if ((s = dev_alloc(h, &h->WP, 3 * ldm * h->Np)) != GP_OK) return s;
    if ((s = dev_alloc(h, &h->mpart, ldm * (h->Np / TB))) != GP_OK) return s;
    if ((s = dev_alloc(h, &h->vpart, ldm * (h->Np / 64))) != GP_OK) return s;     // one slot per 64 columns
    if ((s = dev_alloc(h, &h->outm, ldm)) != GP_OK) return s;
    if ((s = dev_alloc(h, &h->outv, ldm)) != GP_OK) return s;
    if (h->tc_dist) {
        if ((s = dev_alloc(h, &h->ZSS, 6 * ldm * h->dp)) != GP_OK) return s;
        if ((s = dev_alloc(h, &h->zs_mu, ldm)) != GP_OK) return s;
        if ((s = dev_alloc(h, &h->zs_nrm, ldm)) != GP_OK) return s;
    }
    h->m_cap = ldm;
    return GP_OK;
}

gp_status ensure_kslices(gp_t h)
{
    if (h->KS) return GP_OK;
    h->ks_valid = false;
    return dev_alloc(h, &h->KS, (int64_t)gpk::GP_OZ_SLICES * h->Np * h->Np);
}

gp_status ensure_predict_space(gp_t h, int64_t m)
{
    if (h->opt.prec == GP_MIXED) return ensure_predict_space_mixed(h, m);
    const bool emu = h->opt.prec == GP_FP64_OZAKI;   // 128-column blocks of test points
    const int64_t ldm = round_up(m, emu ? 2 * TB : TB);
    if (ldm <= h->m_cap) return GP_OK;
    const int64_t old = h->m_cap;
    const int64_t old_part = old ? (2 * (h->Np / TB) > 64 ? 2 * (h->Np / TB) : 64) * old : 0;
    dev_free(h, &h->OGV, (int64_t)gpk::GP_OG_SLICES * old * h->b);
    dev_free(h, &h->OGVS, (int64_t)gpk::GP_OG_SLICES * old * gpk::GP_OG_SP * h->b);
    dev_free(h, &h->ogv_mu, old);
    dev_free(h, &h->Xs, old * h->d);
    dev_free(h, &h->B, old * h->Np);
    dev_free(h, &h->V, old * h->Np);
    dev_free(h, &h->part, old_part);
    dev_free(h, &h->outm, old);
    dev_free(h, &h->outv, old);
    h->m_cap = 0;
    gp_status s;
    const int64_t rows_part = 2 * (h->Np / TB) > 64 ? 2 * (h->Np / TB) : 64;
    if ((s = dev_alloc(h, &h->Xs, ldm * h->d)) != GP_OK) return s;
    if ((s = dev_alloc(h, &h->B, ldm * h->Np)) != GP_OK) return s;
    if ((s = dev_alloc(h, &h->V, ldm * h->Np)) != GP_OK) return s;
    if ((s = dev_alloc(h, &h->part, rows_part * ldm)) != GP_OK) return s;
    if ((s = dev_alloc(h, &h->outm, ldm)) != GP_OK) return s;
    if ((s = dev_alloc(h, &h->outv, ldm)) != GP_OK) return s;
    if (emu) {
        if ((s = dev_alloc(h, &h->OGV, (int64_t)gpk::GP_OG_SLICES * ldm * h->b)) != GP_OK) return s;
        if ((s = dev_alloc(h, &h->OGVS, (int64_t)gpk::GP_OG_SLICES * ldm * gpk::GP_OG_SP * h->b)) != GP_OK)
            return s;
        if ((s = dev_alloc(h, &h->ogv_mu, ldm)) != GP_OK) return s;
    }
    h->m_cap = ldm;
    return GP_OK;
}

// GP_FP64_OZAKI full covariance: digit slices of all of V (7 x m_cap x Np).
gp_status ensure_cov_slices(gp_t h)
{
    if (h->ogc_cap >= h->m_cap) return GP_OK;
    dev_free(h, &h->OGC, (int64_t)gpk::GP_OG_SLICES * h->ogc_cap * h->Np);
    dev_free(h, &h->ogc_mu, h->ogc_cap);
    dev_free(h, &h->ogc_bits, h->ogc_cap);
    h->ogc_cap = 0;
    gp_status s;
    if ((s = dev_alloc(h, &h->OGC, (int64_t)gpk::GP_OG_SLICES * h->m_cap * h->Np)) != GP_OK) return s;
    if ((s = dev_alloc(h, &h->ogc_mu, h->m_cap)) != GP_OK) return s;
    if ((s = dev_alloc(h, &h->ogc_bits, h->m_cap)) != GP_OK) return s;
    h->ogc_cap = h->m_cap;
    return GP_OK;
}

gp_status ensure_cov_space(gp_t h, int64_t m)
{
    if (m * m <= h->cov_cap) return GP_OK;
    dev_free(h, &h->cov, h->cov_cap);
    h->cov_cap = 0;
    gp_status s = dev_alloc(h, &h->cov, m * m);
    if (s == GP_OK) h->cov_cap = m * m;
    return s;
}

// Task queue of the persistent factorisation: POTRF(0), TRSM(., 0), then per
// step k the updates of column k+1, POTRF(k+1), TRSM(., k+1) (lookahead) and
// the rest of step k's updates.  Every task follows all tasks it depends on.
gp_status build_dag(gp_t h)
{
    const int64_t T = h->T, nt = T * (T + 1) / 2;
    int64_t cap = T + T * (T - 1) / 2;
    for (int64_t k = 0; k < T; ++k) cap += (T - k - 1) * (T - k) / 2;
    int* host = (int*)malloc((size_t)cap * 4 * sizeof(int));
    if (!host) return GP_ERR_OOM;
    int64_t n = 0;
    auto push = [&](int type, int64_t i, int64_t j, int64_t k) {
        host[4 * n + 0] = type;
        host[4 * n + 1] = (int)i;
        host[4 * n + 2] = (int)j;
        host[4 * n + 3] = (int)k;
        ++n;
    };
    push(0, 0, 0, 0);
    for (int64_t i = 1; i < T; ++i) push(1, i, 0, 0);
    for (int64_t k = 0; k + 1 < T; ++k) {
        for (int64_t i = k + 1; i < T; ++i) push(2, i, k + 1, k);
        push(0, k + 1, k + 1, k + 1);
        for (int64_t i = k + 2; i < T; ++i) push(1, i, k + 1, k + 1);
        for (int64_t j = k + 2; j < T; ++j)
            for (int64_t i = j; i < T; ++i) push(2, i, j, k);
    }
    gp_status s = dev_alloc(h, &h->dag_tasks, 4 * n);
    if (s == GP_OK) s = dev_alloc(h, &h->dag_ctl, 2);
    if (s == GP_OK) s = dev_alloc(h, &h->dag_upd, nt);
    if (s == GP_OK) s = dev_alloc(h, &h->dag_fin, nt);
    if (s == GP_OK)
        s = cuda_status(h, cudaMemcpy(h->dag_tasks, host, (size_t)n * 4 * sizeof(int), cudaMemcpyHostToDevice));
    if (s == GP_OK) s = cuda_status(h, cudaMemset(h->dag_ctl, 0, 2 * sizeof(int)));
    free(host);
    h->dag_ntasks = n;
    return s;
}

// Assemble, factor and solve for beta and alpha; NLML into scal[0].  No sync,
// no reset of the failure flag (a failure stays visible to later kernels).
void launch_factor_body(gp_t h, bool reset_err)
{
    gpk::assemble_train(h);
    if (h->opt.scheduler == GP_SCHED_PERSISTENT) gpk::factor_dag(h, reset_err);
    else if (!gpk::factor_fp64(h)) h->host_fail = true;
    gpk::solve_lower(h, h->y, h->beta);
    gpk::solve_upper(h, h->beta, h->alpha);
    gpk::nlml_reduce(h);
}

void launch_factor(gp_t h)
{
    gpk::set_info_none(h);
    launch_factor_body(h, true);
}

// Reads the device word that a tensor-core kernel sets when one of its
// bounded waits runs out (synchronises the stream).
gp_status tc_status(gp_t h)
{
    if (!h->tc_pending) return GP_OK;
    int flag = 0;
    gp_status s = cuda_status(h, gpk::tc_error_fetch(h, &flag));
    if (s == GP_OK) s = sync(h);
    if (s != GP_OK) return s;
    h->tc_pending = false;
    return flag ? GP_ERR_TIMEOUT : GP_OK;
}

gp_status read_info(gp_t h)
{
    unsigned long long info = 0;
    int ctl[2] = {0, 0};
    gp_status s = cuda_status(h, cudaMemcpyAsync(&info, h->info, sizeof(info), cudaMemcpyDeviceToHost, h->st));
    if (s != GP_OK) return s;
    if (h->dag_ctl && (s = cuda_status(h, cudaMemcpyAsync(ctl, h->dag_ctl, sizeof(ctl), cudaMemcpyDeviceToHost,
                                                          h->st))) != GP_OK)
        return s;
    if ((s = sync(h)) != GP_OK) return s;
    if ((s = tc_status(h)) != GP_OK) {
        h->factored = false;
        return s;
    }
    if (ctl[1] == 1) {
        h->last_info = 0;
        h->factored = false;
        return GP_ERR_TIMEOUT;
    }
    if (info != ~0ull) {
        h->last_info = (int64_t)info;
        h->factored = false;
        return GP_ERR_NOT_PD;
    }
    return GP_OK;
}

// GP_MIXED: mixed factor, then alpha by iterative refinement against the
// FP64 residual (host loop; one small device-to-host read per sweep).
gp_status factor_mixed_refined(gp_t h)
{
    gpk::set_info_none(h);
    if (h->tc_dist) {
        if (!gpk::dist_train_tc(h)) return GP_ERR_CUDA;
    } else {
        gpk::assemble_train(h);
    }
    if (!gpk::factor_mixed(h)) return GP_ERR_CUDA;
    gp_status s = check_launch(h);
    if (s != GP_OK) return s;
    if ((s = read_info(h)) != GP_OK) return s;
    gpk::refine_start(h, h->y, h->alpha);
    if ((s = check_launch(h)) != GP_OK) return s;
    // Each pass measures the FP64 residual of the current iterate first and
    // corrects only while that residual still falls: a pass whose residual
    // fell by less than half ends the loop without another correction, and
    // one that rose brings back the previous iterate.
    double prev = INFINITY, nrm[2];
    int it = 0;
    for (;;) {
        gpk::refine_residual(h, h->y, h->alpha, h->res, h->norms);
        if ((s = check_launch(h)) != GP_OK) return s;
        if ((s = cuda_status(h, cudaMemcpyAsync(nrm, h->norms, sizeof(nrm), cudaMemcpyDeviceToHost, h->st))) != GP_OK)
            return s;
        if ((s = sync(h)) != GP_OK) return s;
        double rel = nrm[1] > 0.0 ? sqrt(nrm[0] / nrm[1]) : 0.0;
        if (rel > prev) {
            if ((s = cuda_status(h, cudaMemcpyAsync(h->alpha, h->xprev, h->Np * sizeof(double),
                                                    cudaMemcpyDeviceToDevice, h->st))) != GP_OK)
                return s;
            rel = prev;
        }
        h->refine_residual = rel;
        if (!(rel > h->opt.refine_tol) || rel > 0.5 * prev || it >= h->opt.refine_max_iter) break;
        prev = rel;
        if ((s = cuda_status(h, cudaMemcpyAsync(h->xprev, h->alpha, h->Np * sizeof(double),
                                                cudaMemcpyDeviceToDevice, h->st))) != GP_OK)
            return s;
        gpk::refine_correct(h, h->res, h->alpha);
        ++it;
    }
    h->refine_iters = it;
    if ((s = tc_status(h)) != GP_OK) return s;   // bounded waits of the persistent solves
    gpk::nlml_mixed(h);
    return check_launch(h);
}

gp_status factor_once(gp_t h)
{
    gp_status s;
    if (h->opt.prec == GP_MIXED) {
        h->ks_valid = false;
        return factor_mixed_refined(h);
    }
    launch_factor(h);
    if ((s = check_launch(h)) != GP_OK) return s;
    return read_info(h);
}

// Sets sigma^2 on the host copy and on the device (natural and log scale).
gp_status put_noise(gp_t h, double s2)
{
    h->h_hyp.s2 = s2;
    h->h_hyp.log_theta[2] = s2 > 0.0 ? log(s2) : -INFINITY;
    gp_status s = cuda_status(h, cudaMemcpyAsync(h->hyp, &h->h_hyp, sizeof(GpHyperDev), cudaMemcpyHostToDevice, h->st));
    return s == GP_OK ? sync(h) : s;
}

gp_status ensure_factored(gp_t h)
{
    if (h->factored) return GP_OK;
    h->jitter_added = 0.0;
    gp_status s = factor_once(h);
    if (s == GP_ERR_NOT_PD && h->opt.jitter_retries > 0) {
        // Optional recovery: retry with a growing diagonal jitter on sigma^2.
        const int64_t pivot = h->last_info;
        gp_status r = cuda_status(h, cudaMemcpyAsync(&h->h_hyp, h->hyp, sizeof(GpHyperDev),
                                                     cudaMemcpyDeviceToHost, h->st));
        if (r == GP_OK) r = sync(h);
        if (r != GP_OK) return r;
        const double s2 = h->h_hyp.s2;
        double add = 1e-10 * h->h_hyp.nu;
        for (int t = 0; t < h->opt.jitter_retries && s == GP_ERR_NOT_PD; ++t, add *= 100.0) {
            if ((r = put_noise(h, s2 + add)) != GP_OK) return r;
            s = factor_once(h);
        }
        if (s == GP_OK) {
            h->jitter_added = add / 100.0;
        } else if (s == GP_ERR_NOT_PD) {
            if ((r = put_noise(h, s2)) != GP_OK) return r;
            h->last_info = pivot;
        }
    }
    if (s != GP_OK) return s;
    h->factored = true;
    return GP_OK;
}

// Shared front half of the three predict calls.
gp_status predict_common(gp_t h, const double* Xs, int64_t m, int64_t* ldm_out)
{
    if (!h || !Xs || m < 1) return GP_ERR_ARG;
    gp_status s;
    if ((s = ensure_factored(h)) != GP_OK) return s;
    if ((s = ensure_predict_space(h, m)) != GP_OK) return s;
    *ldm_out = round_up(m, h->opt.prec != GP_FP64 ? 2 * TB : TB);
    if ((s = copy_any(h, h->Xs, Xs, m * h->d)) != GP_OK) return s;
    if (h->opt.prec != GP_MIXED) gpk::assemble_cross(h, m, *ldm_out);
    return check_launch(h);
}

gp_status finish_outputs(gp_t h, bool any_host)
{
    gp_status s = check_launch(h);
    if (s != GP_OK) return s;
    if (!any_host) return GP_OK;
    if ((s = sync(h)) != GP_OK) return s;
    return tc_status(h);
}

}  // namespace

// ---------------------------------------------------------------- launch profiling
bool prof_begin(gp_t h, int phase)
{
    if (h->ev_used + 2 > h->ev_cap) {
        int64_t cap = h->ev_cap ? 2 * h->ev_cap : 4096;
        cudaEvent_t* pool = (cudaEvent_t*)realloc(h->ev_pool, (size_t)cap * sizeof(cudaEvent_t));
        int* ph = (int*)realloc(h->ev_phase, (size_t)(cap / 2) * sizeof(int));
        if (!pool || !ph) {
            if (pool) h->ev_pool = pool;
            if (ph) h->ev_phase = ph;
            return false;
        }
        for (int64_t i = h->ev_cap; i < cap; ++i) cudaEventCreate(&pool[i]);
        h->ev_pool = pool;
        h->ev_phase = ph;
        h->ev_cap = cap;
    }
    h->ev_phase[h->ev_used / 2] = phase;
    cudaEventRecord(h->ev_pool[h->ev_used], h->st);
    return true;
}

void prof_end(gp_t h)
{
    cudaEventRecord(h->ev_pool[h->ev_used + 1], h->st);
    h->ev_used += 2;
}

namespace {
gp_status prof_collect(gp_t h)
{
    if (h->ev_used == 0) return GP_OK;
    gp_status s = sync(h);
    if (s != GP_OK) return s;
    for (int64_t i = 0; i < h->ev_used; i += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev_pool[i], h->ev_pool[i + 1]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        int ph = h->ev_phase[i / 2];
        h->prof_ms[ph] += ms;
        h->prof_cnt[ph] += 1;
    }
    h->ev_used = 0;
    return GP_OK;
}
}  // namespace

extern "C" {

gp_status gp_profile(gp_t h, int enable)
{
    if (!h) return GP_ERR_ARG;
    gp_status s = prof_collect(h);
    h->prof_on = enable != 0;
    return s;
}

gp_status gp_profile_read(gp_t h, double* ms, int64_t* launches, int nphase)
{
    if (!h || nphase < 0 || nphase > GP_NPHASE) return GP_ERR_ARG;
    gp_status s = prof_collect(h);
    if (s != GP_OK) return s;
    for (int p = 0; p < nphase; ++p) {
        if (ms) ms[p] = h->prof_ms[p];
        if (launches) launches[p] = h->prof_cnt[p];
    }
    for (int p = 0; p < GP_NPHASE; ++p) {
        h->prof_ms[p] = 0.0;
        h->prof_cnt[p] = 0;
    }
    return GP_OK;
}

int64_t gp_launch_count(gp_t h) { return h ? h->launches : -1; }

}  // extern "C"

extern "C" {

int64_t gp_auto_tiles(int64_t n)
{
    constexpr int64_t kTile = 256;   // fastest tile edge measured on GB300, both precisions
    return n < 1 ? 0 : (n + kTile - 1) / kTile;
}

void gp_default_options(gp_options* opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->n_tiles = 16;
    opt->prec = GP_FP64;
    opt->noisy_test_var = 0;
    opt->refine_tol = 1e-14;
    opt->refine_max_iter = 20;
    opt->adam_beta1 = 0.9;
    opt->adam_beta2 = 0.999;
    opt->adam_eps = 1e-8;
    opt->cuda_stream = nullptr;
    opt->scheduler = GP_SCHED_STREAM;
    opt->var_correction = 1;
    opt->dag_timeout_ms = 10000;
    opt->kernel = GP_KERNEL_SE;
    opt->jitter_retries = 0;
}

const char* gp_status_str(gp_status s)
{
    switch (s) {
    case GP_OK: return "ok";
    case GP_ERR_ARG: return "invalid argument";
    case GP_ERR_NOT_PD: return "matrix not positive definite";
    case GP_ERR_CUDA: return "CUDA error";
    case GP_ERR_OOM: return "out of device memory";
    case GP_ERR_TIMEOUT: return "device wait timed out";
    case GP_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

int64_t gp_last_error_info(gp_t h) { return h ? h->last_info : -1; }

void gp_destroy(gp_t h)
{
    if (!h) return;
    cudaStreamSynchronize(h->st);
    void* ptrs[] = {h->X, h->y, h->hyp, h->adam, h->L, h->Linv, h->beta, h->alpha, h->work,
                    h->logdet_part, h->info, h->scal, h->Xinv, h->Kinv, h->gpart, h->Xs, h->B,
                    h->V, h->part, h->outm, h->outv, h->cov, h->A32, h->LP, h->Linv32, h->LinvP,
                    h->PA, h->r32, h->t32, h->w32, h->solve_flags, h->res, h->xprev, h->Xsb, h->XsbP, h->norms, h->R32, h->RP,
                    h->WP, h->mpart, h->vpart, h->ZP, h->U32, h->Kinv32, h->R64, h->Rr32,
                    h->YS, h->KS, h->mu, h->kappa, h->qpart, h->vpart2, h->dag_tasks, h->dag_ctl,
                    h->dag_upd, h->dag_fin, h->OGP, h->OGS, h->og_mu, h->OGL, h->ogl_mu, h->OGT, h->OGTS, h->ogt_mu, h->OGX, h->ogx_mu, h->ogx_bits, h->OGV, h->OGVS, h->ogv_mu,
                    h->OGC, h->ogc_mu, h->ogc_bits, h->ZXS, h->zx_mu, h->zx_nrm, h->ZSS, h->zs_mu, h->zs_nrm};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int64_t i = 0; i < h->ev_cap; ++i) cudaEventDestroy(h->ev_pool[i]);
    free(h->ev_pool);
    free(h->ev_phase);
    delete h;
}

gp_status gp_create(const double* X, const double* y, int64_t n, int64_t d, const gp_hyper* hyper,
                    const gp_options* opt_in, gp_t* out)
{
    if (!out) return GP_ERR_ARG;
    *out = nullptr;
    gp_options opt;
    if (opt_in) opt = *opt_in;
    else gp_default_options(&opt);
    if (!X || !y || n < 1 || d < 1 || d > 1024 || !hyper_ok(hyper) || opt.n_tiles < 0 ||
        (opt.prec != GP_FP64 && opt.prec != GP_MIXED && opt.prec != GP_FP64_OZAKI) ||
        (opt.scheduler != GP_SCHED_STREAM && opt.scheduler != GP_SCHED_PERSISTENT) ||
        (opt.scheduler == GP_SCHED_PERSISTENT && opt.prec != GP_FP64) || opt.dag_timeout_ms < 0 ||
        opt.kernel < GP_KERNEL_SE || opt.kernel > GP_KERNEL_MATERN52 || opt.jitter_retries < 0 ||
        opt.jitter_retries > 8)
        return GP_ERR_ARG;
    if (opt.dag_timeout_ms == 0) opt.dag_timeout_ms = 10000;
    if (opt.n_tiles == 0) {
        const int64_t t = gp_auto_tiles(n);
        if (t > INT_MAX) return GP_ERR_ARG;
        opt.n_tiles = (int)t;
    }
    gp_t h = new (std::nothrow) gp_handle();
    if (!h) return GP_ERR_OOM;
    memset((void*)h, 0, sizeof(*h));
    h->opt = opt;
    h->st = (cudaStream_t)opt.cuda_stream;
    cudaGetDevice(&h->device);
    h->n = n;
    h->d = d;
    h->dag_stall = -1;
    h->solve_stall = false;
    h->solve_wait_cycles = 4000000000ll;   // about 2 s at the maximum SM clock
    int64_t per = (n + opt.n_tiles - 1) / opt.n_tiles;
    h->b = round_up(per, opt.prec != GP_FP64 ? 2 * TB : TB);   // tensor-core paths: 128-row blocks
    h->T = (n + h->b - 1) / h->b;
    h->Np = h->T * h->b;
    for (int p = 0; p < 3; ++p) h->trainable[p] = hyper->trainable[p] ? 1 : 0;
    hyper_to_dev(hyper, &h->h_hyp);
    h->h_hyp.kernel = opt.kernel;

    gp_status s = GP_OK;
    const int64_t tiles = ntri(h) * h->b * h->b;
#define TRY(x)                    \
    if ((s = (x)) != GP_OK) {     \
        gp_destroy(h);            \
        return s;                 \
    }
    TRY(dev_alloc(h, &h->X, h->Np * d));
    TRY(dev_alloc(h, &h->y, h->Np));
    TRY(dev_alloc(h, &h->hyp, 1));
    TRY(dev_alloc(h, &h->adam, 1));
    TRY(dev_alloc(h, &h->L, tiles));
    TRY(dev_alloc(h, &h->Linv, h->T * h->b * h->b));
    TRY(dev_alloc(h, &h->beta, h->Np));
    TRY(dev_alloc(h, &h->alpha, h->Np));
    TRY(dev_alloc(h, &h->work, h->Np));
    TRY(dev_alloc(h, &h->logdet_part, h->T));
    TRY(dev_alloc(h, &h->info, 1));
    TRY(dev_alloc(h, &h->scal, 16));
    if (opt.scheduler == GP_SCHED_PERSISTENT) TRY(build_dag(h));
    if (opt.prec == GP_FP64_OZAKI) {   // digit slices of one panel and of one diagonal-tile inverse
        if (h->T > 1) {
            TRY(dev_alloc(h, &h->OGP, (int64_t)gpk::GP_OG_SLICES * (h->Np - h->b) * h->b));
            TRY(dev_alloc(h, &h->OGS, (int64_t)gpk::GP_OG_SLICES * (h->Np - h->b) * gpk::GP_OG_SP * h->b));
            TRY(dev_alloc(h, &h->og_mu, h->Np - h->b));
        }
        TRY(dev_alloc(h, &h->OGL, (int64_t)gpk::GP_OG_SLICES * h->b * h->b));
        TRY(dev_alloc(h, &h->ogl_mu, h->b));
        TRY(dev_alloc(h, &h->solve_flags, 2));   // grid barrier of the diagonal-tile factor
        TRY(cuda_status(h, cudaMemset(h->solve_flags, 0, 2 * sizeof(int))));
    }
    if (opt.prec == GP_MIXED) {
        const int64_t bb = h->b * h->b;
        TRY(dev_alloc(h, &h->A32, tiles));
        TRY(dev_alloc(h, &h->LP, 3 * tiles));
        TRY(dev_alloc(h, &h->Linv32, h->T * bb));
        TRY(dev_alloc(h, &h->LinvP, 3 * h->T * bb));
        TRY(dev_alloc(h, &h->PA, 3 * (h->T > 1 ? h->T - 1 : 1) * bb));
        TRY(dev_alloc(h, &h->r32, h->Np));
        TRY(dev_alloc(h, &h->t32, h->Np));
        TRY(dev_alloc(h, &h->w32, h->Np * gpk::GP_SOLVE_SB));   // partial sums of the solves (one copy per tile of a super-block)
        const int64_t sbx = (h->T + gpk::GP_SOLVE_SB - 1) / gpk::GP_SOLVE_SB * (gpk::GP_SOLVE_SB * h->b) *
                            (gpk::GP_SOLVE_SB * h->b);
        TRY(dev_alloc(h, &h->Xsb, sbx));
        TRY(dev_alloc(h, &h->XsbP, 3 * sbx));
        TRY(dev_alloc(h, &h->solve_flags, 2));
        TRY(cuda_status(h, cudaMemset(h->solve_flags, 0, 2 * sizeof(int))));
        TRY(dev_alloc(h, &h->res, h->Np));
        TRY(dev_alloc(h, &h->xprev, h->Np));
        TRY(dev_alloc(h, &h->norms, 2));
        TRY(dev_alloc(h, &h->kappa, 1));
        h->tc_dist = gpk::use_tc_dist(h);
        if (h->tc_dist) {   // digit slices of the training rows for the tensor-core distances
            h->dp = round_up(d, 32);
            TRY(dev_alloc(h, &h->ZXS, 6 * h->Np * h->dp));
            TRY(dev_alloc(h, &h->zx_mu, h->Np));
            TRY(dev_alloc(h, &h->zx_nrm, h->Np));
        }
    }
    TRY(cuda_status(h, cudaMemsetAsync(h->X, 0, (size_t)(h->Np * d) * sizeof(double), h->st)));
    TRY(cuda_status(h, cudaMemsetAsync(h->y, 0, (size_t)h->Np * sizeof(double), h->st)));
    TRY(cuda_status(h, cudaMemsetAsync(h->adam, 0, sizeof(GpAdamDev), h->st)));
    TRY(copy_any(h, h->X, X, n * d));
    TRY(copy_any(h, h->y, y, n));
    TRY(cuda_status(h, cudaMemcpyAsync(h->hyp, &h->h_hyp, sizeof(GpHyperDev), cudaMemcpyHostToDevice, h->st)));
    if (h->tc_dist) {
        gpk::zslices(h, h->X, h->X, h->Np, h->n, h->ZXS, h->zx_mu, h->zx_nrm, GP_PH_ASSEMBLE);
        TRY(check_launch(h));
    }
    TRY(sync(h));
#undef TRY
    *out = h;
    return GP_OK;
}

gp_status gp_factor(gp_t h)
{
    if (!h) return GP_ERR_ARG;
    return ensure_factored(h);
}

gp_status gp_predict(gp_t h, const double* Xs, int64_t m, double* mean, double* var, double* cov)
{
    if (!mean && !var && !cov) return GP_ERR_ARG;
    int64_t ldm;
    gp_status s = predict_common(h, Xs, m, &ldm);
    if (s != GP_OK) return s;
    bool any_host = false;
    if (h->opt.prec == GP_MIXED) {
        if (!gpk::predict_mixed(h, m, ldm, var != nullptr, cov != nullptr)) return GP_ERR_CUDA;
    } else if (!var && !cov) {  // Eq. 3 alone: one pass K_{Z*,Z} alpha, no solve
        gpk::predict_mean_only(h, m, ldm);
    } else {
        if (!gpk::predict_solve(h, m, ldm)) return GP_ERR_CUDA;
        gpk::predict_finish(h, m, ldm, var != nullptr);
    }
    if (cov) {
        const bool cov_dev = is_device_ptr(cov);
        double* target = cov;
        if (!cov_dev) {
            if ((s = ensure_cov_space(h, m)) != GP_OK) return s;
            target = h->cov;
        }
        if (h->opt.prec != GP_MIXED) {
            if (h->opt.prec == GP_FP64_OZAKI && (s = ensure_cov_slices(h)) != GP_OK) return s;
            if (!gpk::full_cov(h, m, ldm, target)) return GP_ERR_CUDA;
        }
        else if (!gpk::full_cov_mixed(h, m, ldm, target)) return GP_ERR_CUDA;
        if (!cov_dev) {
            if ((s = copy_any(h, cov, target, m * m)) != GP_OK) return s;
            any_host = true;
        }
    }
    if (var && h->opt.prec == GP_MIXED && h->opt.var_correction) {
        if ((s = ensure_kslices(h)) != GP_OK) return s;
        if (!gpk::var_correction_mixed(h, m, ldm)) return GP_ERR_CUDA;
        h->tc_pending = true;
    }
    if (mean) {
        if ((s = copy_any(h, mean, h->outm, m)) != GP_OK) return s;
        any_host = any_host || !is_device_ptr(mean);
    }
    if (var) {
        if ((s = copy_any(h, var, h->outv, m)) != GP_OK) return s;
        any_host = any_host || !is_device_ptr(var);
    }
    return finish_outputs(h, any_host);
}

gp_status gp_predict_mean(gp_t h, const double* Xs, int64_t m, double* mean)
{
    if (!mean) return GP_ERR_ARG;
    return gp_predict(h, Xs, m, mean, nullptr, nullptr);
}

gp_status gp_predict_var(gp_t h, const double* Xs, int64_t m, double* mean, double* var)
{
    if (!var) return GP_ERR_ARG;
    return gp_predict(h, Xs, m, mean, var, nullptr);
}

gp_status gp_predict_full_cov(gp_t h, const double* Xs, int64_t m, double* mean, double* cov)
{
    if (!cov) return GP_ERR_ARG;
    return gp_predict(h, Xs, m, mean, nullptr, cov);
}

gp_status gp_nlml(gp_t h, double* nlml)
{
    if (!h || !nlml) return GP_ERR_ARG;
    gp_status s = ensure_factored(h);
    if (s != GP_OK) return s;
    if ((s = copy_any(h, nlml, h->scal, 1)) != GP_OK) return s;
    return sync(h);
}

gp_status gp_nlml_grad(gp_t h, double* nlml, double grad[3])
{
    if (!h || !grad) return GP_ERR_ARG;
    gp_status s = ensure_factored(h);
    if (s != GP_OK) return s;
    if ((s = ensure_grad_buffers(h)) != GP_OK) return s;
    if (h->opt.prec != GP_MIXED) {
        if (!gpk::inverse_tiles(h)) return GP_ERR_CUDA;
    }
    else if (!gpk::inverse_mixed(h)) return GP_ERR_CUDA;
    gpk::adjoint_grad(h);
    if ((s = check_launch(h)) != GP_OK) return s;
    double tmp[4];
    if ((s = cuda_status(h, cudaMemcpyAsync(tmp, h->scal, sizeof(tmp), cudaMemcpyDeviceToHost, h->st))) != GP_OK)
        return s;
    if ((s = sync(h)) != GP_OK) return s;
    if ((s = tc_status(h)) != GP_OK) return s;
    if (nlml) *nlml = tmp[0];
    grad[0] = tmp[1];
    grad[1] = tmp[2];
    grad[2] = tmp[3];
    return GP_OK;
}

gp_status gp_optimize(gp_t h, int steps, double lr, double* nlml_hist)
{
    if (!h || steps < 0 || !(lr > 0.0)) return GP_ERR_ARG;
    if (steps == 0) return GP_OK;
    gp_status s;
    if ((s = ensure_grad_buffers(h)) != GP_OK) return s;
    double* hist = nullptr;
    const bool hist_dev = nlml_hist && is_device_ptr(nlml_hist);
    if (nlml_hist && !hist_dev) {
        if ((s = dev_alloc(h, &hist, steps)) != GP_OK) return s;
    } else {
        hist = nlml_hist;
    }
    // A factor that is current for the starting hyperparameters is reused by
    // the first iteration; every later iteration refactors at the updated ones.
    const bool reuse_first = h->factored;
    h->factored = false;
    if (!reuse_first) gpk::set_info_none(h);
    const bool mixed = h->opt.prec == GP_MIXED;
    for (int it = 0; it < steps; ++it) {
        if (!(it == 0 && reuse_first)) {
            if (mixed) {
                // the refinement loop synchronises per sweep; a failed factor ends the loop
                h->ks_valid = false;
                if ((s = factor_mixed_refined(h)) != GP_OK) break;
            } else {
                launch_factor_body(h, it == 0);
            }
        }
        if (!mixed) {
            if (!gpk::inverse_tiles(h)) {
                s = GP_ERR_CUDA;
                break;
            }
        } else if (!gpk::inverse_mixed(h)) {
            s = GP_ERR_CUDA;
            break;
        }
        gpk::adjoint_grad(h);
        gpk::adam_step(h, lr, hist ? hist + it : nullptr);
    }
    if (s == GP_OK) s = check_launch(h);
    if (s == GP_OK) s = read_info(h);
    if (s == GP_OK && nlml_hist && !hist_dev) {
        s = copy_any(h, nlml_hist, hist, steps);
        if (s == GP_OK) s = sync(h);
    }
    if (hist && !hist_dev) dev_free(h, &hist, steps);
    if (s == GP_OK) {
        s = cuda_status(h, cudaMemcpyAsync(&h->h_hyp, h->hyp, sizeof(GpHyperDev), cudaMemcpyDeviceToHost, h->st));
        if (s == GP_OK) s = sync(h);
    }
    return s;
}

gp_status gp_get_hyper(gp_t h, gp_hyper* out)
{
    if (!h || !out) return GP_ERR_ARG;
    gp_status s = cuda_status(h, cudaMemcpyAsync(&h->h_hyp, h->hyp, sizeof(GpHyperDev), cudaMemcpyDeviceToHost, h->st));
    if (s == GP_OK) s = sync(h);
    if (s != GP_OK) return s;
    out->lengthscale = h->h_hyp.l;
    out->vertical = h->h_hyp.nu;
    out->noise_var = h->h_hyp.s2;
    for (int p = 0; p < 3; ++p) out->trainable[p] = h->trainable[p];
    return GP_OK;
}

gp_status gp_set_hyper(gp_t h, const gp_hyper* hyper)
{
    if (!h || !hyper_ok(hyper)) return GP_ERR_ARG;
    hyper_to_dev(hyper, &h->h_hyp);
    h->h_hyp.kernel = h->opt.kernel;
    for (int p = 0; p < 3; ++p) h->trainable[p] = hyper->trainable[p] ? 1 : 0;
    gp_status s = cuda_status(h, cudaMemcpyAsync(h->hyp, &h->h_hyp, sizeof(GpHyperDev), cudaMemcpyHostToDevice, h->st));
    if (s == GP_OK) s = sync(h);
    h->factored = false;
    return s;
}

gp_status gp_get_state(gp_t h, gp_state* out)
{
    if (!h || !out) return GP_ERR_ARG;
    GpAdamDev a;
    gp_status s = cuda_status(h, cudaMemcpyAsync(&a, h->adam, sizeof(a), cudaMemcpyDeviceToHost, h->st));
    if (s == GP_OK)
        s = cuda_status(h, cudaMemcpyAsync(&h->h_hyp, h->hyp, sizeof(GpHyperDev), cudaMemcpyDeviceToHost, h->st));
    if (s == GP_OK) s = sync(h);
    if (s != GP_OK) return s;
    for (int p = 0; p < 3; ++p) {
        out->log_theta[p] = h->h_hyp.log_theta[p];
        out->adam_m[p] = a.m[p];
        out->adam_v[p] = a.v[p];
    }
    out->adam_t = (int64_t)a.t;
    return GP_OK;
}

gp_status gp_set_state(gp_t h, const gp_state* st)
{
    if (!h || !st || st->adam_t < 0) return GP_ERR_ARG;
    GpAdamDev a;
    for (int p = 0; p < 3; ++p) {
        if (!isfinite(st->log_theta[p]) || !isfinite(st->adam_m[p]) || !(st->adam_v[p] >= 0.0))
            return GP_ERR_ARG;
        a.m[p] = st->adam_m[p];
        a.v[p] = st->adam_v[p];
        h->h_hyp.log_theta[p] = st->log_theta[p];
    }
    a.t = (double)st->adam_t;
    h->h_hyp.l = exp(st->log_theta[0]);
    h->h_hyp.nu = exp(st->log_theta[1]);
    h->h_hyp.s2 = exp(st->log_theta[2]);
    h->h_hyp.inv2l2 = 1.0 / (2.0 * h->h_hyp.l * h->h_hyp.l);
    gp_status s = cuda_status(h, cudaMemcpyAsync(h->adam, &a, sizeof(a), cudaMemcpyHostToDevice, h->st));
    if (s == GP_OK)
        s = cuda_status(h, cudaMemcpyAsync(h->hyp, &h->h_hyp, sizeof(GpHyperDev), cudaMemcpyHostToDevice, h->st));
    if (s == GP_OK) s = sync(h);
    h->factored = false;
    return s;
}

gp_status gp_get_factor(gp_t h, double* L_out)
{
    if (!h || !L_out) return GP_ERR_ARG;
    gp_status s = ensure_factored(h);
    if (s != GP_OK) return s;
    auto dense = [&](double* out) {
        if (h->opt.prec == GP_MIXED) gpk::copy_factor_dense_mixed(h, out);
        else gpk::copy_factor_dense(h, out);
    };
    if (is_device_ptr(L_out)) {
        dense(L_out);
        return finish_outputs(h, false);
    }
    double* tmp = nullptr;
    if ((s = dev_alloc(h, &tmp, h->n * h->n)) != GP_OK) return s;
    dense(tmp);
    s = copy_any(h, L_out, tmp, h->n * h->n);
    if (s == GP_OK) s = finish_outputs(h, true);
    dev_free(h, &tmp, h->n * h->n);
    return s;
}

gp_status gp_get_alpha(gp_t h, double* alpha_out)
{
    if (!h || !alpha_out) return GP_ERR_ARG;
    gp_status s = ensure_factored(h);
    if (s != GP_OK) return s;
    if ((s = copy_any(h, alpha_out, h->alpha, h->n)) != GP_OK) return s;
    return finish_outputs(h, !is_device_ptr(alpha_out));
}

gp_status gp_dag_stall_tile(gp_t h, int64_t i, int64_t j)
{
    if (!h || (i >= 0 && (j < 0 || j > i || i >= h->T))) return GP_ERR_ARG;
    h->dag_stall = i < 0 ? -1 : tri_index(i, j);
    h->factored = false;
    return GP_OK;
}

gp_status gp_solve_stall(gp_t h, int enable, int64_t wait_us)
{
    if (!h || (enable && (wait_us < 1 || wait_us > 2000000))) return GP_ERR_ARG;
    h->solve_stall = enable != 0;
    // clock64 counts SM cycles: 2100 per microsecond bounds the wait from above at any clock up to 2.1 GHz
    h->solve_wait_cycles = enable ? (long long)wait_us * 2100 : 4000000000ll;
    h->factored = false;
    return GP_OK;
}

gp_status gp_info(gp_t h, gp_info_t* out)
{
    if (!h || !out) return GP_ERR_ARG;
    out->n = h->n;
    out->d = h->d;
    out->tile = h->b;
    out->n_tiles = h->T;
    out->n_padded = h->Np;
    out->device_bytes = h->bytes;
    out->refine_iters = h->refine_iters;
    out->refine_residual = h->refine_residual;
    out->jitter_added = h->jitter_added;
    return GP_OK;
}

}  // extern "C"
