/*
 * gprat_gb.h - C ABI of the GB300-native exact Gaussian-process regression
 * library (GPRat, arXiv 2505.00136).
 *
 * The calls follow the paper's statement of the problem (Section 4.3): a GP
 * object is created from training data, a tile configuration and the
 * hyperparameters of the squared-exponential kernel (Eq. 2); it can then be
 * factored (tiled Cholesky, Section 4.2 / Fig. 1), asked for predictions with
 * or without uncertainty (Eqs. 3-4), for its loss (Eq. 5) and its gradient,
 * and optimised with Adam (Section 4.1).
 *
 * Conventions shared by every call:
 *  - Matrices are row-major float64: X is n x d, Xs is m x d, cov is m x m.
 *  - Pointers may be host or device memory; each call detects which with
 *    cudaPointerGetAttributes.  Host outputs are written before the call
 *    returns; device outputs are written in order on the handle's stream.
 *    Device memory of a GPU other than the current one is treated like host
 *    memory (moved by copies, never addressed by a kernel).
 *  - gp_create copies X and y into device memory owned by the handle; the
 *    caller owns every output buffer; gp_destroy frees all handle memory.
 *  - Work is issued on gp_options.cuda_stream (NULL: the legacy default
 *    stream).  Calls that return host scalars or status from the device
 *    synchronise that stream.
 *  - No call throws, aborts or exits.  Each returns a gp_status;
 *    gp_last_error_info gives detail (failing pivot row for GP_ERR_NOT_PD,
 *    the cudaError_t for GP_ERR_CUDA).
 *  - Hyperparameters are given on their natural scale (length scale l,
 *    vertical scale nu, noise variance sigma^2); internally, and for
 *    gradients and Adam, the library works with (log l, log nu, log sigma^2).
 *  - Ragged sizes are allowed: n need not be a multiple of the tile size (the
 *    factor is padded with an identity block that changes no result), m is
 *    any value >= 1, n >= 1, 1 <= d <= 1024.
 */
#ifndef GPRAT_GB_H
#define GPRAT_GB_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gp_handle* gp_t;

typedef enum {
    GP_OK = 0,
    GP_ERR_ARG = 1,     /* bad argument (NULL, size, option); nothing was changed */
    GP_ERR_NOT_PD = 2,  /* K + sigma^2 I not positive definite in working precision */
    GP_ERR_CUDA = 3,    /* a CUDA runtime call failed */
    GP_ERR_OOM = 4,     /* device allocation failed */
    GP_ERR_TIMEOUT = 5, /* a bounded device-side wait expired (persistent scheduler) */
    GP_ERR_STATE = 6    /* call not valid in the handle's current state */
} gp_status;

/* GP_FP64: every step in FP64 arithmetic.  GP_MIXED: FP32-accurate factor on
 * the BF16 tensor cores, alpha, mean and variances refined or corrected to
 * FP64 level (the NLML, gradient and full covariance stay FP32-accurate).
 * GP_FP64_OZAKI: the FP64 path with the factorisation's trailing updates taken
 * as exact digit products on the BF16 tensor cores (the Ozaki scheme: operands
 * rounded to 49 bits, every level of digit products summed exactly), FP64
 * level throughout; no counterpart in the paper. */
typedef enum { GP_FP64 = 0, GP_MIXED = 1, GP_FP64_OZAKI = 2 } gp_precision;

/* Covariance function.  GP_KERNEL_SE is Eq. 2, nu exp(-r^2 / (2 l^2)); the
 * Matern kernels (the paper's future work, Section 6; Rasmussen & Williams
 * Eq. 4.17) are nu m(r) with s = sqrt(2p) r / l for order p:
 * p = 1/2: exp(-s), p = 3/2: (1 + s) exp(-s), p = 5/2: (1 + s + s^2/3) exp(-s).
 * All share the hyperparameters (l, nu, sigma^2) and their gradients. */
typedef enum {
    GP_KERNEL_SE = 0,
    GP_KERNEL_MATERN12 = 1,
    GP_KERNEL_MATERN32 = 2,
    GP_KERNEL_MATERN52 = 3
} gp_kernel;

typedef enum {
    GP_SCHED_STREAM = 0,     /* one launch per tile step, stream ordered */
    GP_SCHED_PERSISTENT = 1  /* one persistent launch walking the tile DAG (GP_FP64 only) */
} gp_scheduler;

/* Eq. 2 hyperparameters.  trainable[p] = 0 freezes parameter p in gp_optimize
 * (the paper's trainable-parameter flags, Section 4.3). */
typedef struct {
    double lengthscale; /* l > 0 */
    double vertical;    /* nu > 0 (linear factor, not squared) */
    double noise_var;   /* sigma^2 >= 0 */
    int trainable[3];   /* order: l, nu, sigma^2 */
} gp_hyper;

typedef struct {
    int n_tiles;            /* tiles per dimension T (paper: 1, 4, 16); tile size is
                               ceil(n / T) rounded up to a multiple of 64 (128 for
                               GP_MIXED and GP_FP64_OZAKI); 0 chooses T = gp_auto_tiles(n) */
    gp_precision prec;      /* GP_FP64, GP_MIXED or GP_FP64_OZAKI */
    int noisy_test_var;     /* 1: add sigma^2 to predictive (co)variances */
    double refine_tol;      /* GP_MIXED: stop refinement at ||r|| / ||y|| < tol */
    int refine_max_iter;    /* GP_MIXED: at most this many refinement sweeps */
    double adam_beta1, adam_beta2, adam_eps;
    void* cuda_stream;      /* cudaStream_t used for all work */
    gp_scheduler scheduler; /* how the Cholesky tile DAG is executed */
    int var_correction;     /* GP_MIXED: 1 corrects the predictive variances to FP64 level
                               (see gp_predict_var), 0 returns the mixed-factor variances */
    int dag_timeout_ms;     /* GP_SCHED_PERSISTENT: bound on any single dependency wait of
                               the persistent kernel; expiry ends the call with GP_ERR_TIMEOUT */
    gp_kernel kernel;       /* covariance function (default GP_KERNEL_SE) */
    int jitter_retries;     /* recovery from GP_ERR_NOT_PD, 0..8 (default 0: off).  With k > 0,
                               a factorisation that meets a non-positive pivot is retried up
                               to k times, try t with sigma^2 = sigma0^2 + 1e-10 nu 100^(t-1);
                               the first that succeeds is kept (gp_get_hyper returns it,
                               gp_info reports the added jitter); if none does, sigma0^2 is
                               restored and GP_ERR_NOT_PD returned.  Applies to gp_factor and
                               the calls that factor on demand, not to gp_optimize's steps. */
} gp_options;

/* Fills defaults: n_tiles 16, FP64, latent variance, refine_tol 1e-14,
 * refine_max_iter 20, Adam (0.9, 0.999, 1e-8), default stream, stream
 * scheduler, variance correction on, DAG wait bound 10000 ms, squared
 * exponential kernel, no jitter retries. */
void gp_default_options(gp_options* opt);

/* Automatic tile count (the tile-size selection the paper leaves to future
 * work, Section 6): T = ceil(n / 256), i.e. tiles of 256.  Measured on GB300
 * for both precisions at n = 8192, 16384 and 32768 against tiles of 128, 512
 * and 1024: larger tiles lengthen the single-SM diagonal factor on the
 * critical path of the tile DAG (Fig. 1), smaller ones give narrower tensor
 * units and more launches.  Returns 0 for n < 1.  Pure host function: no
 * device work, callable without a GPU. */
int64_t gp_auto_tiles(int64_t n);

/* Creates a GP over n training points X (n x d) with targets y (n).  Copies
 * X and y to the device.  Fails with GP_ERR_ARG on NULL pointers, n < 1,
 * d < 1 or d > 1024, n_tiles < 0, non-positive l or nu or negative sigma^2.
 * n_tiles = 0 takes gp_auto_tiles(n). */
gp_status gp_create(const double* X, const double* y, int64_t n, int64_t d,
                    const gp_hyper* hyper, const gp_options* opt, gp_t* out);

/* Assembles K = K_f + sigma^2 I in lower tiles (Eq. 2) and factors it in
 * place, K = L L^T, by the tiled right-looking Cholesky of Fig. 1 (POTRF,
 * TRSM, SYRK, GEMM tiles), then solves beta = L^{-1} y and
 * alpha = L^{-T} beta.  Idempotent until the hyperparameters change.
 * Synchronises.  GP_ERR_NOT_PD: gp_last_error_info gives the first row whose
 * pivot was not positive. */
gp_status gp_factor(gp_t h);

/* Predictive mean at m test points (Eq. 3): mean = K_{Z*,Z} K^{-1} y. */
gp_status gp_predict_mean(gp_t h, const double* Xs, int64_t m, double* mean);

/* Mean and predictive variance (diagonal of Eq. 4):
 * var_i = k(x*_i, x*_i) - || L^{-1} k_*i ||^2 (+ sigma^2 if noisy_test_var). */
gp_status gp_predict_var(gp_t h, const double* Xs, int64_t m, double* mean, double* var);

/* Mean and full posterior covariance (Eq. 4), cov m x m row-major:
 * cov = K_{Z*,Z*} - V^T V with V = L^{-1} K_{Z*,Z}^T. */
gp_status gp_predict_full_cov(gp_t h, const double* Xs, int64_t m, double* mean, double* cov);

/* Negative log marginal likelihood, the negative of Eq. 5:
 * 1/2 y^T K^{-1} y + 1/2 log|K| + n/2 log(2 pi).  Synchronises. */
gp_status gp_nlml(gp_t h, double* nlml);

/* NLML and its gradient with respect to (log l, log nu, log sigma^2):
 * g_p = 1/2 tr((K^{-1} - alpha alpha^T) dK/dtheta_p), with K^{-1} formed as
 * L^{-T} L^{-1} from tiles and dK/dtheta regenerated inside the reduction (no
 * dK is stored).  Synchronises. */
gp_status gp_nlml_grad(gp_t h, double* nlml, double grad_log_theta[3]);

/* steps Adam iterations (lr, the handle's beta1/beta2/eps) on the trainable
 * log-hyperparameters, each on the NLML gradient at the current point.
 * nlml_hist (host or device, steps entries, may be NULL) receives the NLML
 * before each update.  Adam state persists across calls (see gp_get_state). */
gp_status gp_optimize(gp_t h, int steps, double lr, double* nlml_hist);

gp_status gp_get_hyper(gp_t h, gp_hyper* out);
/* Sets new hyperparameters; invalidates the factor.  Does not reset Adam. */
gp_status gp_set_hyper(gp_t h, const gp_hyper* hyper);

/* Optimiser checkpoint: theta[3] (log scale), m[3], v[3] and step count t. */
typedef struct {
    double log_theta[3];
    double adam_m[3];
    double adam_v[3];
    int64_t adam_t;
} gp_state;
gp_status gp_get_state(gp_t h, gp_state* out);
gp_status gp_set_state(gp_t h, const gp_state* st);

/* Copies the Cholesky factor L (n x n row-major, upper triangle zero) to L_out
 * (host or device).  Factors first if needed. */
gp_status gp_get_factor(gp_t h, double* L_out);

/* General prediction: any of mean (m), var (m) and cov (m x m) may be NULL;
 * all requested outputs come from one forward solve V = L^{-1} K_{Z*,Z}^T
 * (Eqs. 3-4).  At least one output must be non-NULL. */
gp_status gp_predict(gp_t h, const double* Xs, int64_t m, double* mean, double* var, double* cov);

/* Per-launch timing of the library's kernels with CUDA events on the handle's
 * stream, accumulated by phase.  Off by default. */
typedef enum {
    GP_PH_ASSEMBLE = 0, /* K tiles (Eq. 2) */
    GP_PH_POTRF,        /* diagonal-tile Cholesky + inverse */
    GP_PH_TRSM,         /* panel solves */
    GP_PH_UPDATE,       /* trailing SYRK / GEMM */
    GP_PH_SOLVE,        /* beta, alpha (single right-hand side) */
    GP_PH_CROSS,        /* K_{Z*,Z}, K_{Z*,Z*} */
    GP_PH_VSOLVE,       /* V = L^{-1} K_{Z*,Z}^T with fused row sums */
    GP_PH_REDUCE,       /* mean / variance / NLML / gradient reductions */
    GP_PH_COV,          /* K_{Z*,Z*} - V^T V */
    GP_PH_TRTRI,        /* L^{-1} tiles */
    GP_PH_LAUUM,        /* K^{-1} = L^{-T} L^{-1} tiles */
    GP_PH_ADJOINT,      /* fused dK/dtheta reduction */
    GP_PH_ADAM,
    GP_PH_REFINE,       /* mixed path: FP64 residuals and corrections of alpha */
    GP_PH_BSOLVE,       /* mixed variance correction: x0^T = W L~^{-1} (backward multi-RHS solve) */
    GP_PH_OZAKI,        /* mixed variance correction: the exact digit-pair product K x~0 */
    GP_PH_RSOLVE,       /* mixed variance correction: L~^{-1} r0 (forward multi-RHS solve) */
    GP_PH_SLICES,       /* mixed variance correction: x0 rounded to x~0, digit slices of x~0 and K */
    GP_PH_OTHER,
    GP_NPHASE
} gp_phase;
/* enable != 0 turns per-launch event timing on. */
gp_status gp_profile(gp_t h, int enable);
/* Synchronises, then writes per-phase milliseconds and launch counts
 * accumulated since the last read (arrays of nphase <= GP_NPHASE entries,
 * either may be NULL) and resets them. */
gp_status gp_profile_read(gp_t h, double* ms, int64_t* launches, int nphase);
/* Kernels launched by this handle since it was created. */
int64_t gp_launch_count(gp_t h);

/* Copies alpha = K^{-1} y (n entries, host or device), the weights of the
 * predictive mean (Eq. 3: mean = K_{Z*,Z} alpha).  Factors first if needed. */
gp_status gp_get_alpha(gp_t h, double* alpha_out);

/* ------------------------------------------------------------------------
 * Learned hyperparameter initialiser (no counterpart in the paper).  A
 * 64-dimensional summary of a data set feeds a 64 -> 256 -> 256 -> 3 ReLU
 * MLP whose outputs are initial (log l, log nu, log sigma^2).  The buffers of
 * the training calls below are DEVICE memory of the current GPU (GP_ERR_ARG
 * otherwise; gp_learned_init also takes host memory); calls are
 * stream-ordered on `stream`.
 *
 * Model blob (GP_MLP_MODEL_FLOATS floats): W1[256][64] b1[256] W2[256][256]
 * b2[256] W3[3][256] b3[3] (the GP_MLP_NPARAM trained values), then the
 * feature mean[64] and standard deviation[64] that standardise summaries. */
#define GP_MLP_NPARAM 83203
#define GP_MLP_MODEL_FLOATS (GP_MLP_NPARAM + 128)
#define GP_LEARNED_INIT_SCRATCH 72

/* s (64 doubles) = summary of (X n x d, y n): the 32 largest per-regressor
 * standard deviations (descending, zero-padded), the autocorrelation of y at
 * lags 1..16, and the means of cos(omega_q y) and sin(omega_q y) for the 8
 * frequencies omega (doubles).  Requires n >= 2, 1 <= d <= 1024. */
gp_status gp_summary(const double* X, const double* y, int64_t n, int64_t d, const double* omega,
                     double* s, void* stream);
/* Feature mean and standard deviation over B summaries (B x 64 doubles) into
 * the model blob's standardisation slots. */
gp_status gp_mlp_feature_stats(const double* S, int64_t B, float* model, void* stream);
/* Floats of workspace gp_mlp_loss_grad needs for a batch of B. */
int64_t gp_mlp_workspace_floats(int64_t B);
/* out (B x 3 floats) = network outputs for B summaries S (B x 64 doubles). */
gp_status gp_mlp_forward(const float* model, const double* S, int64_t B, float* out, void* stream);
/* Mean-squared error 1/(3B) sum (out - target)^2 into *loss (device float,
 * may be NULL) and its gradient in the GP_MLP_NPARAM weights into gW. */
gp_status gp_mlp_loss_grad(const float* model, const double* S, const float* target, int64_t B,
                           float* gW, float* loss, float* workspace, void* stream);
/* One Adam step (t >= 1) on the model's GP_MLP_NPARAM weights; m and v are
 * GP_MLP_NPARAM-float moment buffers owned by the caller. */
gp_status gp_mlp_adam(float* model, const float* gW, float* m, float* v, int64_t t, double lr,
                      double beta1, double beta2, double eps, void* stream);
/* Initial hyperparameters for a data set: summary -> network -> exp, written
 * to *out (host) on their natural scale; scratch holds GP_LEARNED_INIT_SCRATCH
 * doubles.  Unlike the calls above, X, y, model and omega may each be host or
 * device memory (detected per pointer; host ones, and those on another GPU,
 * are copied into stream-ordered device memory for the call), and scratch may
 * be NULL, host memory or another GPU's (a device scratch is then allocated
 * for the call); with buffers of the current device throughout nothing is
 * allocated.  Synchronises.  GP_ERR_STATE if the
 * network output is not finite. */
gp_status gp_learned_init(const double* X, const double* y, int64_t n, int64_t d, const float* model,
                          const double* omega, double* scratch, gp_hyper* out, void* stream);

/* Testing aid for the persistent scheduler's bounded waits: until called
 * again with i < 0, every persistent factorisation treats the update counter
 * of tile (i, j) as never complete, so the waits on it expire after
 * dag_timeout_ms and the call returns GP_ERR_TIMEOUT with the device still
 * usable.  GP_ERR_ARG unless 0 <= j <= i < n_tiles (or i < 0). */
gp_status gp_dag_stall_tile(gp_t h, int64_t i, int64_t j);

/* Testing aid for the bounded grid-barrier waits of GP_MIXED's persistent
 * FP32 triangular solves (one cooperative launch per solve): with enable != 0,
 * every such solve runs with its last CTA never arriving at the first
 * barrier and with each barrier wait bounded by wait_us microseconds (at
 * the GPU's maximum SM clock; longer at lower clocks), so the other CTAs'
 * waits expire, the kernel leaves and the call that factors returns
 * GP_ERR_TIMEOUT with the device still usable.  enable = 0 restores the
 * default bound (about 2 s) and normal solves.  The next call refactors.
 * GP_ERR_ARG if enable != 0 and wait_us is outside [1, 2e6]. */
gp_status gp_solve_stall(gp_t h, int enable, int64_t wait_us);

/* Tile geometry and last-call diagnostics. */
typedef struct {
    int64_t n, d, tile, n_tiles, n_padded;
    int64_t device_bytes;      /* bytes currently held on the device */
    int refine_iters;          /* GP_MIXED: sweeps used by the last alpha solve */
    double refine_residual;    /* GP_MIXED: ||y - K alpha|| / ||y|| after refinement */
    double jitter_added;       /* sigma^2 added by the last factorisation's retries (0: none) */
} gp_info_t;
gp_status gp_info(gp_t h, gp_info_t* out);

/* Allocation-free predictive mean (no counterpart in the paper).  For callers
 * that cannot allocate device memory - servers whose device memory belongs to
 * a pool fixed at start-up, latency-bound loops that must not enter the
 * allocator, plug-ins of hosts that forbid allocation - this computes
 * mean = K_{Z*,Z} alpha (Eq. 3)
 * from trained weights (alpha from gp_get_alpha) without a handle and without
 * any cudaMalloc, cudaFree or allocating library call.  The kernel is the
 * squared exponential of Eq. 2.
 *   X (n x d), alpha (n), Xs (m x d) and mean (m): caller-owned DEVICE memory,
 *   row-major float64; lengthscale l and vertical nu as in Eq. 2; cuda_stream
 *   as in gp_options (NULL: legacy default stream).  Stream-ordered, no sync.
 * Limits: 1 <= m <= GP_NOALLOC_MAX_TEST, 1 <= d <= 1024; larger or invalid
 * arguments, host pointers (pinned ones included) and device memory of a GPU
 * other than the current one return GP_ERR_ARG before any work.
 * Scratch: a fixed GP_NOALLOC_CHUNKS x GP_NOALLOC_MAX_TEST array of doubles
 * (16 MiB) in the library's device data, held by every GPU that loads the
 * library until the process exits and shared by all calls on that GPU.  The
 * first call on a device looks its address up (cudaGetSymbolAddress) with that
 * device current.  Calls whose work overlaps on the GPU (different streams,
 * no ordering) race on the scratch and must not be issued. */
#define GP_NOALLOC_MAX_TEST 32768
#define GP_NOALLOC_CHUNKS 64
gp_status gp_predict_mean_noalloc(const double* X, const double* alpha, int64_t n, int64_t d,
                                  const double* Xs, int64_t m, double lengthscale, double vertical,
                                  double* mean, void* cuda_stream);

/* Measurement aid (no counterpart in the paper): the FP64 arithmetic peaks of
 * the current GPU in TFLOP/s, from register-only throughput loops of
 * mma.sync.m8n8k4.f64 (the FP64 tensor path the FP64 tile products use) and
 * of DFMA, timed with CUDA events on cuda_stream (the third of three
 * repetitions).  They are the denominators of the FP64 path's roofline
 * fractions.  Allocates and frees two small device buffers; synchronises. */
gp_status gp_measure_fp64_peaks(double* dmma_tflops, double* dfma_tflops, void* cuda_stream);

int64_t gp_last_error_info(gp_t h);
const char* gp_status_str(gp_status s);
void gp_destroy(gp_t h);

#ifdef __cplusplus
}
#endif
#endif
