// C ABI entry points (include/gprat_gb.h): handle lifecycle, argument
// validation, host/device pointer detection and stream-ordered orchestration
// of the kernels.  No call throws; every failure becomes a gp_status.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "gp_internal.cuh"

namespace {

constexpr int64_t TB = GP_TB;

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

gp_status cuda_status(gp_t h, cudaError_t e)
{
    if (e == cudaSuccess) return GP_OK;
    if (h) h->last_info = (int64_t)e;
    return e == cudaErrorMemoryAllocation ? GP_ERR_OOM : GP_ERR_CUDA;
}

gp_status check_launch(gp_t h)
{
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
    if (h->Xinv) return GP_OK;
    gp_status s;
    const int64_t tiles = ntri(h) * h->b * h->b;
    const int64_t P = h->b / TB;
    if ((s = dev_alloc(h, &h->Xinv, tiles)) != GP_OK) return s;
    if ((s = dev_alloc(h, &h->Kinv, tiles)) != GP_OK) return s;
    h->gpart_cap = ntri(h) * P * P * 3;
    return dev_alloc(h, &h->gpart, h->gpart_cap);
}

gp_status ensure_predict_space(gp_t h, int64_t m)
{
    const int64_t ldm = round_up(m, TB);
    if (ldm <= h->m_cap) return GP_OK;
    const int64_t old = h->m_cap;
    const int64_t old_part = old ? (2 * (h->Np / TB) > 64 ? 2 * (h->Np / TB) : 64) * old : 0;
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
    h->m_cap = ldm;
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

// Assemble, factor and solve for beta and alpha; NLML into scal[0].  No sync.
void launch_factor(gp_t h)
{
    gpk::set_info_none(h);
    gpk::assemble_train(h);
    gpk::factor_fp64(h);
    gpk::solve_lower(h, h->y, h->beta);
    gpk::solve_upper(h, h->beta, h->alpha);
    gpk::nlml_reduce(h);
}

gp_status read_info(gp_t h)
{
    unsigned long long info = 0;
    gp_status s = cuda_status(h, cudaMemcpyAsync(&info, h->info, sizeof(info), cudaMemcpyDeviceToHost, h->st));
    if (s != GP_OK) return s;
    if ((s = sync(h)) != GP_OK) return s;
    if (info != ~0ull) {
        h->last_info = (int64_t)info;
        h->factored = false;
        return GP_ERR_NOT_PD;
    }
    return GP_OK;
}

gp_status ensure_factored(gp_t h)
{
    if (h->factored) return GP_OK;
    launch_factor(h);
    gp_status s = check_launch(h);
    if (s != GP_OK) return s;
    if ((s = read_info(h)) != GP_OK) return s;
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
    *ldm_out = round_up(m, TB);
    if ((s = copy_any(h, h->Xs, Xs, m * h->d)) != GP_OK) return s;
    gpk::assemble_cross(h, m, *ldm_out);
    return check_launch(h);
}

gp_status finish_outputs(gp_t h, bool any_host)
{
    gp_status s = check_launch(h);
    if (s != GP_OK) return s;
    return any_host ? sync(h) : GP_OK;
}

}  // namespace

extern "C" {

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
                    h->V, h->part, h->outm, h->outv, h->cov};
    for (void* p : ptrs)
        if (p) cudaFree(p);
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
    if (!X || !y || n < 1 || d < 1 || d > 1024 || !hyper_ok(hyper) || opt.n_tiles < 1 ||
        (opt.prec != GP_FP64 && opt.prec != GP_MIXED) ||
        (opt.scheduler != GP_SCHED_STREAM && opt.scheduler != GP_SCHED_PERSISTENT))
        return GP_ERR_ARG;
    gp_t h = new (std::nothrow) gp_handle();
    if (!h) return GP_ERR_OOM;
    memset((void*)h, 0, sizeof(*h));
    h->opt = opt;
    h->st = (cudaStream_t)opt.cuda_stream;
    cudaGetDevice(&h->device);
    h->n = n;
    h->d = d;
    int64_t per = (n + opt.n_tiles - 1) / opt.n_tiles;
    h->b = round_up(per, TB);
    h->T = (n + h->b - 1) / h->b;
    h->Np = h->T * h->b;
    for (int p = 0; p < 3; ++p) h->trainable[p] = hyper->trainable[p] ? 1 : 0;
    hyper_to_dev(hyper, &h->h_hyp);

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
    TRY(cuda_status(h, cudaMemsetAsync(h->X, 0, (size_t)(h->Np * d) * sizeof(double), h->st)));
    TRY(cuda_status(h, cudaMemsetAsync(h->y, 0, (size_t)h->Np * sizeof(double), h->st)));
    TRY(cuda_status(h, cudaMemsetAsync(h->adam, 0, sizeof(GpAdamDev), h->st)));
    TRY(copy_any(h, h->X, X, n * d));
    TRY(copy_any(h, h->y, y, n));
    TRY(cuda_status(h, cudaMemcpyAsync(h->hyp, &h->h_hyp, sizeof(GpHyperDev), cudaMemcpyHostToDevice, h->st)));
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

gp_status gp_predict_mean(gp_t h, const double* Xs, int64_t m, double* mean)
{
    if (!mean) return GP_ERR_ARG;
    int64_t ldm;
    gp_status s = predict_common(h, Xs, m, &ldm);
    if (s != GP_OK) return s;
    gpk::predict_mean_only(h, m, ldm);
    if ((s = copy_any(h, mean, h->outm, m)) != GP_OK) return s;
    return finish_outputs(h, !is_device_ptr(mean));
}

gp_status gp_predict_var(gp_t h, const double* Xs, int64_t m, double* mean, double* var)
{
    if (!var) return GP_ERR_ARG;
    int64_t ldm;
    gp_status s = predict_common(h, Xs, m, &ldm);
    if (s != GP_OK) return s;
    gpk::predict_solve(h, m, ldm);
    gpk::predict_finish(h, m, ldm, true);
    if (mean && (s = copy_any(h, mean, h->outm, m)) != GP_OK) return s;
    if ((s = copy_any(h, var, h->outv, m)) != GP_OK) return s;
    return finish_outputs(h, (mean && !is_device_ptr(mean)) || !is_device_ptr(var));
}

gp_status gp_predict_full_cov(gp_t h, const double* Xs, int64_t m, double* mean, double* cov)
{
    if (!cov) return GP_ERR_ARG;
    int64_t ldm;
    gp_status s = predict_common(h, Xs, m, &ldm);
    if (s != GP_OK) return s;
    gpk::predict_solve(h, m, ldm);
    gpk::predict_finish(h, m, ldm, false);
    const bool cov_dev = is_device_ptr(cov);
    double* target = cov;
    if (!cov_dev) {
        if ((s = ensure_cov_space(h, m)) != GP_OK) return s;
        target = h->cov;
    }
    gpk::full_cov(h, m, ldm, target);
    if (mean && (s = copy_any(h, mean, h->outm, m)) != GP_OK) return s;
    if (!cov_dev && (s = copy_any(h, cov, target, m * m)) != GP_OK) return s;
    return finish_outputs(h, (mean && !is_device_ptr(mean)) || !cov_dev);
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
    gpk::inverse_tiles(h);
    gpk::adjoint_grad(h);
    if ((s = check_launch(h)) != GP_OK) return s;
    double tmp[4];
    if ((s = cuda_status(h, cudaMemcpyAsync(tmp, h->scal, sizeof(tmp), cudaMemcpyDeviceToHost, h->st))) != GP_OK)
        return s;
    if ((s = sync(h)) != GP_OK) return s;
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
    h->factored = false;
    gpk::set_info_none(h);
    for (int it = 0; it < steps; ++it) {
        gpk::assemble_train(h);
        gpk::factor_fp64(h);
        gpk::solve_lower(h, h->y, h->beta);
        gpk::solve_upper(h, h->beta, h->alpha);
        gpk::nlml_reduce(h);
        gpk::inverse_tiles(h);
        gpk::adjoint_grad(h);
        gpk::adam_step(h, lr, hist ? hist + it : nullptr);
    }
    s = check_launch(h);
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
    if (is_device_ptr(L_out)) {
        gpk::copy_factor_dense(h, L_out);
        return finish_outputs(h, false);
    }
    double* tmp = nullptr;
    if ((s = dev_alloc(h, &tmp, h->n * h->n)) != GP_OK) return s;
    gpk::copy_factor_dense(h, tmp);
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
    return GP_OK;
}

}  // extern "C"
