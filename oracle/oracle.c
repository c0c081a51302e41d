/*
 * Plain, unblocked FP64 CPU oracle for exact Gaussian-process regression
 * (GPRat, arXiv 2505.00136, Section 4.1).  TEST INFRASTRUCTURE ONLY: see
 * oracle.h.  Every routine is the textbook definition written out with no
 * blocking, tiling, fusion or reordering, so it can be checked against the
 * paper's equations by eye.  It shares nothing with the CUDA library.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

int orc_version(void) { return 1; }

/* Squared Euclidean distance by direct differences (never |a|^2+|b|^2-2ab). */
static double sqdist(const double* a, const double* b, int64_t d)
{
    double s = 0.0;
    for (int64_t k = 0; k < d; ++k) {
        double t = a[k] - b[k];
        s += t * t;
    }
    return s;
}

/* Eq. 2, noise-free part: nu * exp(-r^2 / (2 l^2)). */
void orc_se_cross(const double* A, int64_t na, const double* B, int64_t nb, int64_t d,
                  double l, double nu, double* out)
{
    for (int64_t i = 0; i < na; ++i)
        for (int64_t j = 0; j < nb; ++j)
            out[i * nb + j] = nu * exp(-sqdist(A + i * d, B + j * d, d) / (2.0 * l * l));
}

/*
 * Matern kernels of half-integer order (Rasmussen & Williams 2006, Eq. 4.17;
 * the paper lists them as future work, Section 6), nu * m(r) with
 * s = sqrt(2 p) r / l for order p = 1/2, 3/2, 5/2:
 *   p = 1/2: m = exp(-s),  p = 3/2: m = (1 + s) exp(-s),
 *   p = 5/2: m = (1 + s + s^2 / 3) exp(-s).
 * kind: 1, 2, 3 for p = 1/2, 3/2, 5/2 (0 is the squared exponential of Eq. 2).
 */
static double matern_s(int kind, double r, double l)
{
    double c = kind == 1 ? 1.0 : (kind == 2 ? sqrt(3.0) : sqrt(5.0));
    return c * r / l;
}

static double matern(int kind, double r, double l, double nu)
{
    double s = matern_s(kind, r, l);
    if (kind == 1) return nu * exp(-s);
    if (kind == 2) return nu * (1.0 + s) * exp(-s);
    return nu * (1.0 + s + s * s / 3.0) * exp(-s);
}

/* d/d(log l) of the Matern kernel: ds/dlog l = -s, so with dm/ds
 * p = 1/2: s exp(-s),  p = 3/2: s^2 exp(-s),  p = 5/2: s^2 (1 + s) exp(-s) / 3. */
static double matern_dlogl(int kind, double r, double l, double nu)
{
    double s = matern_s(kind, r, l);
    if (kind == 1) return nu * s * exp(-s);
    if (kind == 2) return nu * s * s * exp(-s);
    return nu * s * s * (1.0 + s) * exp(-s) / 3.0;
}

/* out[i*nb+j] = kernel `kind` between a_i and b_j, no delta term. */
void orc_kernel_cross(int kind, const double* A, int64_t na, const double* B, int64_t nb, int64_t d,
                      double l, double nu, double* out)
{
    if (kind == 0) {
        orc_se_cross(A, na, B, nb, d, l, nu, out);
        return;
    }
    for (int64_t i = 0; i < na; ++i)
        for (int64_t j = 0; j < nb; ++j)
            out[i * nb + j] = matern(kind, sqrt(sqdist(A + i * d, B + j * d, d)), l, nu);
}

/* Eq. 2 over all training pairs; the Kronecker delta adds sigma^2 when i == j. */
void orc_cov_train_k(int kind, const double* X, int64_t n, int64_t d, const double* hyp, double* K)
{
    orc_kernel_cross(kind, X, n, X, n, d, hyp[0], hyp[1], K);
    for (int64_t i = 0; i < n; ++i) K[i * n + i] += hyp[2];
}

void orc_cov_train(const double* X, int64_t n, int64_t d, const double* hyp, double* K)
{
    orc_cov_train_k(0, X, n, d, hyp, K);
}

/* Cholesky-Banachiewicz: row i, column j <= i, L_ij = (K_ij - sum_{k<j} L_ik L_jk) / L_jj. */
int64_t orc_cholesky(const double* K, int64_t n, double* L)
{
    memset(L, 0, (size_t)(n * n) * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j <= i; ++j) {
            double s = K[i * n + j];
            for (int64_t k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            if (i == j) {
                if (!(s > 0.0)) return i;
                L[i * n + i] = sqrt(s);
            } else {
                L[i * n + j] = s / L[j * n + j];
            }
        }
    }
    return -1;
}

/* Forward substitution, L x' = x. */
void orc_forward(const double* L, int64_t n, double* x)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = x[i];
        for (int64_t k = 0; k < i; ++k) s -= L[i * n + k] * x[k];
        x[i] = s / L[i * n + i];
    }
}

/* Backward substitution, L^T x' = x. */
void orc_backward(const double* L, int64_t n, double* x)
{
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int64_t k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
        x[i] = s / L[i * n + i];
    }
}

/* Column c of L^{-1} is the forward-substitution solution of L x = e_c. */
void orc_tri_inverse(const double* L, int64_t n, double* Linv)
{
    double* col = (double*)malloc((size_t)n * sizeof(double));
    memset(Linv, 0, (size_t)(n * n) * sizeof(double));
    for (int64_t c = 0; c < n; ++c) {
        for (int64_t i = 0; i < n; ++i) col[i] = (i == c) ? 1.0 : 0.0;
        orc_forward(L, n, col);
        for (int64_t i = 0; i < n; ++i) Linv[i * n + c] = col[i];
    }
    free(col);
}

/* K^{-1} = (L L^T)^{-1} = L^{-T} L^{-1}: (K^{-1})_ij = sum_k Linv_ki Linv_kj. */
void orc_chol_inverse(const double* L, int64_t n, double* Kinv)
{
    double* Linv = (double*)malloc((size_t)(n * n) * sizeof(double));
    orc_tri_inverse(L, n, Linv);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double s = 0.0;
            for (int64_t k = 0; k < n; ++k) s += Linv[k * n + i] * Linv[k * n + j];
            Kinv[i * n + j] = s;
        }
    free(Linv);
}

/* Shared first stage of prediction and likelihood: K, L, beta = L^{-1} y, alpha = K^{-1} y. */
static int64_t factor_and_solve(int kind, const double* X, const double* y, int64_t n, int64_t d,
                                const double* hyp, double** L_out, double** beta_out,
                                double** alpha_out)
{
    double* K = (double*)malloc((size_t)(n * n) * sizeof(double));
    double* L = (double*)malloc((size_t)(n * n) * sizeof(double));
    orc_cov_train_k(kind, X, n, d, hyp, K);
    int64_t info = orc_cholesky(K, n, L);
    free(K);
    if (info >= 0) {
        free(L);
        return info;
    }
    double* beta = (double*)malloc((size_t)n * sizeof(double));
    double* alpha = (double*)malloc((size_t)n * sizeof(double));
    memcpy(beta, y, (size_t)n * sizeof(double));
    orc_forward(L, n, beta);
    memcpy(alpha, beta, (size_t)n * sizeof(double));
    orc_backward(L, n, alpha);
    *L_out = L;
    *beta_out = beta;
    *alpha_out = alpha;
    return -1;
}

int64_t orc_predict_k(int kind, const double* X, const double* y, int64_t n, int64_t d,
                      const double* Xs, int64_t m, const double* hyp, int noisy,
                      double* mean, double* var, double* cov)
{
    double *L, *beta, *alpha;
    int64_t info = factor_and_solve(kind, X, y, n, d, hyp, &L, &beta, &alpha);
    if (info >= 0) return info;
    double* Kc = (double*)malloc((size_t)(m * n) * sizeof(double)); /* K_{Z*,Z}, m x n */
    orc_kernel_cross(kind, Xs, m, X, n, d, hyp[0], hyp[1], Kc);

    /* Eq. 3: mean = K_{Z*,Z} K^{-1} y = K_{Z*,Z} alpha. */
    if (mean)
        for (int64_t i = 0; i < m; ++i) {
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) s += Kc[i * n + j] * alpha[j];
            mean[i] = s;
        }

    if (var || cov) {
        /* Eq. 4: K_{Z*,Z} K^{-1} K_{Z*,Z}^T = V^T V with V = L^{-1} K_{Z*,Z}^T.
         * Row i of Vt holds column i of V (the forward solve of test point i). */
        double* Vt = Kc;
        for (int64_t i = 0; i < m; ++i) orc_forward(L, n, Vt + i * n);
        double prior = hyp[1] + (noisy ? hyp[2] : 0.0); /* k(x*, x*) = nu exp(0) */
        if (var)
            for (int64_t i = 0; i < m; ++i) {
                double s = 0.0;
                for (int64_t j = 0; j < n; ++j) s += Vt[i * n + j] * Vt[i * n + j];
                var[i] = prior - s;
            }
        if (cov) {
            orc_kernel_cross(kind, Xs, m, Xs, m, d, hyp[0], hyp[1], cov); /* K_{Z*,Z*} */
            for (int64_t i = 0; i < m; ++i) {
                if (noisy) cov[i * m + i] += hyp[2];
                for (int64_t k = 0; k < m; ++k) {
                    double s = 0.0;
                    for (int64_t j = 0; j < n; ++j) s += Vt[i * n + j] * Vt[k * n + j];
                    cov[i * m + k] -= s;
                }
            }
        }
    }
    free(Kc);
    free(L);
    free(beta);
    free(alpha);
    return -1;
}

int64_t orc_predict(const double* X, const double* y, int64_t n, int64_t d,
                    const double* Xs, int64_t m, const double* hyp, int noisy,
                    double* mean, double* var, double* cov)
{
    return orc_predict_k(0, X, y, n, d, Xs, m, hyp, noisy, mean, var, cov);
}

/* log|K| = 2 sum log L_ii and y^T K^{-1} y = beta^T beta give -(Eq. 5). */
static double nlml_from(const double* L, const double* beta, int64_t n)
{
    double fit = 0.0, logdet_half = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        fit += beta[i] * beta[i];
        logdet_half += log(L[i * n + i]);
    }
    return 0.5 * fit + logdet_half + 0.5 * (double)n * log(2.0 * M_PI);
}

int64_t orc_nlml_k(int kind, const double* X, const double* y, int64_t n, int64_t d,
                   const double* hyp, double* nlml)
{
    double *L, *beta, *alpha;
    int64_t info = factor_and_solve(kind, X, y, n, d, hyp, &L, &beta, &alpha);
    if (info >= 0) return info;
    *nlml = nlml_from(L, beta, n);
    free(L);
    free(beta);
    free(alpha);
    return -1;
}

int64_t orc_nlml(const double* X, const double* y, int64_t n, int64_t d,
                 const double* hyp, double* nlml)
{
    return orc_nlml_k(0, X, y, n, d, hyp, nlml);
}

/*
 * dNLML/dtheta_p = 1/2 tr((K^{-1} - alpha alpha^T) dK/dtheta_p)
 * (Rasmussen & Williams 2006, Eq. 5.9, sign flipped for the negative), with
 *   dK/dlog l      = K_f .* r^2 / l^2,
 *   dK/dlog nu     = K_f,
 *   dK/dlog sigma2 = sigma^2 I
 * for the squared exponential, and dK/dlog l = matern_dlogl for a Matern kernel.
 */
int64_t orc_nlml_grad_k(int kind, const double* X, const double* y, int64_t n, int64_t d,
                        const double* hyp, double* nlml, double* grad)
{
    double *L, *beta, *alpha;
    int64_t info = factor_and_solve(kind, X, y, n, d, hyp, &L, &beta, &alpha);
    if (info >= 0) return info;
    *nlml = nlml_from(L, beta, n);
    double* Kinv = (double*)malloc((size_t)(n * n) * sizeof(double));
    orc_chol_inverse(L, n, Kinv);
    const double l = hyp[0], nu = hyp[1], s2 = hyp[2];
    double g_l = 0.0, g_nu = 0.0, g_s2 = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double w = Kinv[i * n + j] - alpha[i] * alpha[j];
            double r2 = sqdist(X + i * d, X + j * d, d);
            double kf;
            if (kind == 0) {
                kf = nu * exp(-r2 / (2.0 * l * l));
                g_l += w * kf * r2 / (l * l);
            } else {
                kf = matern(kind, sqrt(r2), l, nu);
                g_l += w * matern_dlogl(kind, sqrt(r2), l, nu);
            }
            g_nu += w * kf;
            if (i == j) g_s2 += w * s2;
        }
    grad[0] = 0.5 * g_l;
    grad[1] = 0.5 * g_nu;
    grad[2] = 0.5 * g_s2;
    free(Kinv);
    free(L);
    free(beta);
    free(alpha);
    return -1;
}

int64_t orc_nlml_grad(const double* X, const double* y, int64_t n, int64_t d,
                      const double* hyp, double* nlml, double* grad)
{
    return orc_nlml_grad_k(0, X, y, n, d, hyp, nlml, grad);
}

/* Adam (Kingma & Ba 2015, Algorithm 1), only on trainable components. */
void orc_adam(double* theta, double* mom, double* vel, const double* g, int64_t t,
              double lr, double beta1, double beta2, double eps, const int* trainable)
{
    for (int p = 0; p < 3; ++p) {
        if (trainable && !trainable[p]) continue;
        mom[p] = beta1 * mom[p] + (1.0 - beta1) * g[p];
        vel[p] = beta2 * vel[p] + (1.0 - beta2) * g[p] * g[p];
        double mhat = mom[p] / (1.0 - pow(beta1, (double)t));
        double vhat = vel[p] / (1.0 - pow(beta2, (double)t));
        theta[p] -= lr * mhat / (sqrt(vhat) + eps);
    }
}

int64_t orc_optimize_k(int kind, const double* X, const double* y, int64_t n, int64_t d, double* hyp,
                       const int* trainable, int64_t steps, double lr, double beta1,
                       double beta2, double eps, double* nlml_hist)
{
    double theta[3] = {log(hyp[0]), log(hyp[1]), log(hyp[2])};
    double mom[3] = {0, 0, 0}, vel[3] = {0, 0, 0};
    for (int64_t s = 0; s < steps; ++s) {
        double h[3] = {exp(theta[0]), exp(theta[1]), exp(theta[2])};
        double f, g[3];
        int64_t info = orc_nlml_grad_k(kind, X, y, n, d, h, &f, g);
        if (info >= 0) return info;
        if (nlml_hist) nlml_hist[s] = f;
        orc_adam(theta, mom, vel, g, s + 1, lr, beta1, beta2, eps, trainable);
    }
    hyp[0] = exp(theta[0]);
    hyp[1] = exp(theta[1]);
    hyp[2] = exp(theta[2]);
    return -1;
}

int64_t orc_optimize(const double* X, const double* y, int64_t n, int64_t d, double* hyp,
                     const int* trainable, int64_t steps, double lr, double beta1,
                     double beta2, double eps, double* nlml_hist)
{
    return orc_optimize_k(0, X, y, n, d, hyp, trainable, steps, lr, beta1, beta2, eps, nlml_hist);
}

/* ------------------------------------------------------------------------ */
/* Learned initialiser (not in the paper).                                    */
/* ------------------------------------------------------------------------ */

static int cmp_desc(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x < y) - (x > y);
}

/*
 * s[0..31]  per-regressor population standard deviations, sorted descending,
 *           truncated or zero-padded to 32;
 * s[32..47] autocorrelation of y at lags 1..16 (sum over the n-k overlapping
 *           pairs of centred values / sum of squared centred values);
 * s[48..63] random-Fourier-feature mean embedding of y: for q = 0..7,
 *           s[48+2q] = mean cos(omega_q y_i), s[49+2q] = mean sin(omega_q y_i).
 */
void orc_summary(const double* X, const double* y, int64_t n, int64_t d,
                 const double* omega, double* s)
{
    memset(s, 0, 64 * sizeof(double));
    double* sd = (double*)calloc((size_t)(d > 32 ? d : 32), sizeof(double));
    for (int64_t k = 0; k < d; ++k) {
        double mu = 0.0;
        for (int64_t i = 0; i < n; ++i) mu += X[i * d + k];
        mu /= (double)n;
        double v = 0.0;
        for (int64_t i = 0; i < n; ++i) v += (X[i * d + k] - mu) * (X[i * d + k] - mu);
        sd[k] = sqrt(v / (double)n);
    }
    qsort(sd, (size_t)d, sizeof(double), cmp_desc);
    for (int k = 0; k < 32; ++k) s[k] = sd[k];
    free(sd);

    double ybar = 0.0;
    for (int64_t i = 0; i < n; ++i) ybar += y[i];
    ybar /= (double)n;
    double c0 = 0.0;
    for (int64_t i = 0; i < n; ++i) c0 += (y[i] - ybar) * (y[i] - ybar);
    for (int lag = 1; lag <= 16; ++lag) {
        double c = 0.0;
        for (int64_t i = 0; i + lag < n; ++i) c += (y[i] - ybar) * (y[i + lag] - ybar);
        s[31 + lag] = (c0 > 0.0) ? c / c0 : 0.0;
    }
    for (int q = 0; q < 8; ++q) {
        double cs = 0.0, sn = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            cs += cos(omega[q] * y[i]);
            sn += sin(omega[q] * y[i]);
        }
        s[48 + 2 * q] = cs / (double)n;
        s[49 + 2 * q] = sn / (double)n;
    }
}

enum { MLP_IN = 64, MLP_H = 256, MLP_OUT = 3 };
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + MLP_H * MLP_IN)
#define OFF_W2 (OFF_B1 + MLP_H)
#define OFF_B2 (OFF_W2 + MLP_H * MLP_H)
#define OFF_W3 (OFF_B2 + MLP_H)
#define OFF_B3 (OFF_W3 + MLP_OUT * MLP_H)
#define MLP_NPARAM (OFF_B3 + MLP_OUT)

/* One sample: h1 = relu(W1 s + b1), h2 = relu(W2 h1 + b2), o = W3 h2 + b3. */
static void mlp_one(const double* W, const double* s, double* h1, double* h2, double* o)
{
    for (int j = 0; j < MLP_H; ++j) {
        double a = W[OFF_B1 + j];
        for (int k = 0; k < MLP_IN; ++k) a += W[OFF_W1 + j * MLP_IN + k] * s[k];
        h1[j] = a > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < MLP_H; ++j) {
        double a = W[OFF_B2 + j];
        for (int k = 0; k < MLP_H; ++k) a += W[OFF_W2 + j * MLP_H + k] * h1[k];
        h2[j] = a > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < MLP_OUT; ++j) {
        double a = W[OFF_B3 + j];
        for (int k = 0; k < MLP_H; ++k) a += W[OFF_W3 + j * MLP_H + k] * h2[k];
        o[j] = a;
    }
}

void orc_mlp_forward(const double* W, int64_t batch, const double* S, double* out)
{
    double h1[MLP_H], h2[MLP_H];
    for (int64_t b = 0; b < batch; ++b) mlp_one(W, S + b * MLP_IN, h1, h2, out + b * MLP_OUT);
}

/* Loss = 1/(3 batch) sum (o - t)^2; reverse-mode chain rule through the three layers. */
double orc_mlp_loss_grad(const double* W, int64_t batch, const double* S,
                         const double* target, double* gW)
{
    memset(gW, 0, MLP_NPARAM * sizeof(double));
    double h1[MLP_H], h2[MLP_H], o[MLP_OUT], d2[MLP_H], d1[MLP_H], dO[MLP_OUT];
    double loss = 0.0, scale = 1.0 / (3.0 * (double)batch);
    for (int64_t b = 0; b < batch; ++b) {
        const double* s = S + b * MLP_IN;
        mlp_one(W, s, h1, h2, o);
        for (int j = 0; j < MLP_OUT; ++j) {
            double e = o[j] - target[b * MLP_OUT + j];
            loss += e * e * scale;
            dO[j] = 2.0 * e * scale;
            gW[OFF_B3 + j] += dO[j];
            for (int k = 0; k < MLP_H; ++k) gW[OFF_W3 + j * MLP_H + k] += dO[j] * h2[k];
        }
        for (int k = 0; k < MLP_H; ++k) {
            double a = 0.0;
            for (int j = 0; j < MLP_OUT; ++j) a += W[OFF_W3 + j * MLP_H + k] * dO[j];
            d2[k] = h2[k] > 0.0 ? a : 0.0;
        }
        for (int j = 0; j < MLP_H; ++j) {
            gW[OFF_B2 + j] += d2[j];
            for (int k = 0; k < MLP_H; ++k) gW[OFF_W2 + j * MLP_H + k] += d2[j] * h1[k];
        }
        for (int k = 0; k < MLP_H; ++k) {
            double a = 0.0;
            for (int j = 0; j < MLP_H; ++j) a += W[OFF_W2 + j * MLP_H + k] * d2[j];
            d1[k] = h1[k] > 0.0 ? a : 0.0;
        }
        for (int j = 0; j < MLP_H; ++j) {
            gW[OFF_B1 + j] += d1[j];
            for (int k = 0; k < MLP_IN; ++k) gW[OFF_W1 + j * MLP_IN + k] += d1[j] * s[k];
        }
    }
    return loss;
}
