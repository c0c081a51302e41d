/*
 * Plain, unblocked FP64 CPU oracle for exact Gaussian-process regression
 * (GPRat, arXiv 2505.00136, Section 4.1, Eqs. 2-5).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this library: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or helper with
 * the CUDA library; both read the same seeded inputs and nothing else.
 *
 * Conventions: all matrices are row-major, dense, float64.  Hyperparameters
 * are passed on their natural scale as hyp[3] = {l, nu, sigma^2} (length
 * scale, vertical scale, noise variance; Eq. 2).  Gradients are with respect
 * to (log l, log nu, log sigma^2).  Functions that factor return -1 on
 * success or the 0-based row at which a non-positive pivot appeared.
 *
 * Parity status: every function below is pinned by the CPU tests (closed
 * forms, exact rational arithmetic, LAPACK special cases, invariants and
 * finite differences) except where its comment says "parity unpinned".
 */
#ifndef GPRAT_ORACLE_H
#define GPRAT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

int orc_version(void);

/* out[i*nb+j] = nu * exp(-|a_i - b_j|^2 / (2 l^2)); Eq. 2 without the delta term. */
void orc_se_cross(const double* A, int64_t na, const double* B, int64_t nb, int64_t d,
                  double l, double nu, double* out);
/* K = K_f + sigma^2 I over the training points (Eq. 2 with the Kronecker delta). */
void orc_cov_train(const double* X, int64_t n, int64_t d, const double* hyp, double* K);
/* Cholesky-Banachiewicz, K = L L^T, L lower (upper part zeroed). */
int64_t orc_cholesky(const double* K, int64_t n, double* L);
/* In place: x <- L^{-1} x (forward substitution). */
void orc_forward(const double* L, int64_t n, double* x);
/* In place: x <- L^{-T} x (backward substitution). */
void orc_backward(const double* L, int64_t n, double* x);
/* Linv = L^{-1} (lower), column by column. */
void orc_tri_inverse(const double* L, int64_t n, double* Linv);
/* Kinv = L^{-T} L^{-1} = K^{-1} (full symmetric). */
void orc_chol_inverse(const double* L, int64_t n, double* Kinv);

/* Prediction (Eqs. 3 and 4).  Any of mean / var / cov may be NULL.
 * var[i] = k(x*_i, x*_i) - k*_i^T K^{-1} k*_i (+ sigma^2 if noisy);
 * cov is m x m row-major (+ sigma^2 on its diagonal if noisy). */
int64_t orc_predict(const double* X, const double* y, int64_t n, int64_t d,
                    const double* Xs, int64_t m, const double* hyp, int noisy,
                    double* mean, double* var, double* cov);
/* NLML = -(Eq. 5) = 1/2 y^T K^{-1} y + sum_i log L_ii + n/2 log(2 pi). */
int64_t orc_nlml(const double* X, const double* y, int64_t n, int64_t d,
                 const double* hyp, double* nlml);
/* NLML and its gradient with respect to (log l, log nu, log sigma^2):
 * g_p = 1/2 sum_ij (K^{-1} - alpha alpha^T)_ij (dK/dtheta_p)_ij. */
int64_t orc_nlml_grad(const double* X, const double* y, int64_t n, int64_t d,
                      const double* hyp, double* nlml, double* grad);
/* One Adam step (Kingma & Ba 2015) on log-hyperparameters, t >= 1. */
void orc_adam(double* theta, double* mom, double* vel, const double* g, int64_t t,
              double lr, double beta1, double beta2, double eps, const int* trainable);
/* steps x (NLML+grad, Adam) from hyp (natural scale, updated in place). */
int64_t orc_optimize(const double* X, const double* y, int64_t n, int64_t d, double* hyp,
                     const int* trainable, int64_t steps, double lr, double beta1,
                     double beta2, double eps, double* nlml_hist);

/* The same with a choice of kernel: kind 0 = squared exponential (Eq. 2),
 * 1 / 2 / 3 = Matern of order 1/2, 3/2, 5/2 (nu * m(r), Rasmussen & Williams
 * Eq. 4.17; the paper's future work, Section 6). */
void orc_kernel_cross(int kind, const double* A, int64_t na, const double* B, int64_t nb, int64_t d,
                      double l, double nu, double* out);
void orc_cov_train_k(int kind, const double* X, int64_t n, int64_t d, const double* hyp, double* K);
int64_t orc_predict_k(int kind, const double* X, const double* y, int64_t n, int64_t d,
                      const double* Xs, int64_t m, const double* hyp, int noisy,
                      double* mean, double* var, double* cov);
int64_t orc_nlml_k(int kind, const double* X, const double* y, int64_t n, int64_t d,
                   const double* hyp, double* nlml);
int64_t orc_nlml_grad_k(int kind, const double* X, const double* y, int64_t n, int64_t d,
                        const double* hyp, double* nlml, double* grad);
int64_t orc_optimize_k(int kind, const double* X, const double* y, int64_t n, int64_t d, double* hyp,
                       const int* trainable, int64_t steps, double lr, double beta1,
                       double beta2, double eps, double* nlml_hist);

/* 64-d data summary for the learned initialiser (not in the paper). */
void orc_summary(const double* X, const double* y, int64_t n, int64_t d,
                 const double* omega, double* s);
/* MLP 64 -> 256 -> 256 -> 3 with ReLU; flat weights W1,b1,W2,b2,W3,b3. */
void orc_mlp_forward(const double* W, int64_t batch, const double* S, double* out);
/* Mean-squared error over batch x 3 outputs and its gradient in the weights. */
double orc_mlp_loss_grad(const double* W, int64_t batch, const double* S,
                         const double* target, double* gW);

#ifdef __cplusplus
}
#endif
#endif
