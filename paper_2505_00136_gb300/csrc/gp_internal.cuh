// Internal declarations of the GB300 exact-GP library: handle, tile geometry,
// launch helpers.  Not part of the C ABI (see include/gprat_gb.h).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gprat_gb.h"

// Square tiles of TB x TB doubles; the tile size b is a multiple of TB.
#define GP_TB 64
#define GP_THREADS 256

// Device-side hyperparameter record, updated in place by the Adam kernel so
// that an optimisation loop never round-trips through the host.
struct GpHyperDev {
    double l, nu, s2;         // natural scale (Eq. 2)
    double inv2l2;            // 1 / (2 l^2)
    double log_theta[3];      // (log l, log nu, log sigma^2)
    int kernel;               // gp_kernel (fixed per handle)
};

struct GpAdamDev {
    double m[3], v[3];
    double t;                 // step count as a double (Adam's bias correction)
};

// Lower-triangular tile storage: tile (i, j), i >= j, holds rows i*b.. and
// columns j*b.. of the matrix, row-major with leading dimension b, at
// offset tri_index(i, j) * b * b.  Only T (T + 1) / 2 tiles exist.
__host__ __device__ inline int64_t tri_index(int64_t i, int64_t j) { return i * (i + 1) / 2 + j; }

struct gp_handle {
    int64_t n, d, b, T, Np;   // Np = T * b >= n; rows n..Np-1 are identity padding
    gp_options opt;
    cudaStream_t st;
    int device;

    // Resident training data (padded rows are zero).
    double* X;                // Np x d
    double* y;                // Np
    GpHyperDev* hyp;          // device copy
    GpHyperDev h_hyp;         // host mirror
    int trainable[3];
    GpAdamDev* adam;

    // Factor and solves.
    double* L;                // T(T+1)/2 tiles: K, then L in place
    double* Linv;             // T tiles: inverses of the diagonal tiles of L
    double* beta;             // L^{-1} y
    double* alpha;            // K^{-1} y
    double* work;             // Np scratch vector
    double* logdet_part;      // T partial sums of log L_ii
    unsigned long long* info; // first failing pivot row (ULLONG_MAX: none)
    double* scal;             // device scalars: [0] nlml, [1..3] grad, [4..] reductions
    bool factored;

    // Gradient buffers (allocated on first use).
    double* Xinv;             // T(T+1)/2 tiles of L^{-1}
    double* Kinv;             // T(T+1)/2 tiles of K^{-1} (lower)
    double* gpart;            // per-block partial gradient sums
    int64_t gpart_cap;

    // Prediction workspace (grown on demand).
    int64_t m_cap;            // capacity in test points (multiple of 64)
    double* Xs;               // m_cap x d
    double* B;                // Np x m_cap: K_{Z*,Z}^T, overwritten by the solve
    double* V;                // Np x m_cap: L^{-1} K_{Z*,Z}^T
    double* part;             // (Np/64) x m_cap x 2 partial column sums
    double* outm;             // m_cap mean
    double* outv;             // m_cap var
    double* cov;              // m_cap x m_cap (full covariance), allocated on demand
    int64_t cov_cap;

    // Mixed precision (GP_MIXED).  h->L then holds the FP64 K (never factored).
    float* A32;               // T(T+1)/2 tiles: FP32 K, then the mixed factor in place
    __nv_bfloat16* LP;        // T(T+1)/2 tiles x 3 BF16 planes of the off-diagonal factor tiles
    float* Linv32;            // T tiles: inverses of the diagonal factor tiles
    __nv_bfloat16* LinvP;     // T tiles x 3 planes of Linv32
    __nv_bfloat16* PA;        // (T-1) tiles x 3 planes: panel operand scratch
    float *r32, *t32, *w32;   // FP32 vectors of the refinement solves (w32: b / 64 copies of Np)
    double* res;              // Np FP64 residual
    double* xprev;            // Np: the refinement's previous iterate
    float* Xsb;               // inverses of the super-blocks of GP_SOLVE_SB diagonal tiles, (GP_SOLVE_SB b)^2 each
    __nv_bfloat16* XsbP;      // their three BF16 planes (upper tiles zero), plane-major
    double* norms;            // 2 FP64 norms
    float* R32;               // m_cap x Np: K_{Z*,Z}, overwritten by the W solve
    __nv_bfloat16 *RP, *WP;   // planes: RP 3 x m_cap x b (scratch), WP 3 x m_cap x Np (all of W)
    double* mpart;            // (Np/64) x m_cap mean partial sums
    double* vpart;            // (Np/64) x m_cap variance partial sums (one per 64 columns)
    // variance correction (GP_MIXED)
    double* R64;              // m_cap x Np: FP64 K_{Z*,Z}
    float* Rr32;              // m_cap x Np: r0 = K_{Z*,Z} - x0^T K
    __nv_bfloat16* YS;        // digit slices of x~0^T, GP_OZ_YSLICES x m_cap x Np
    __nv_bfloat16* KS;        // digit slices of K, OZ_S x Np x Np (allocated on first use)
    double* mu;               // m_cap row scales of x0^T
    double* kappa;            // scale of K
    double* qpart;            // 2 x (Np/64) x m_cap partial sums (one per 64 columns)
    double* vpart2;           // (Np/64) x m_cap partial sums of ||L~^{-1} r0||^2
    bool ks_valid;            // KS matches the current K
    // tensor-core squared distances (GP_MIXED, d >= GP_TC_DIST_MIN_D; kernels_dist.cu)
    bool tc_dist;
    bool host_fail;           // a launch could not be set up on the host; reported by the next check
    // GP_FP64_OZAKI: digit slices of the current panel, 7 x (Np - b) x b, and their row scales
    __nv_bfloat16 *OGP, *OGS;   // OGS: slices of one super-panel, 7 x (Np - b) x (GP_OG_SP b)
    double* og_mu;
    // GP_FP64_OZAKI gradient: column slices of one row block of L^{-1} (7 x Np x b), of all
    // of L^{-1} (7 x Np x Np), their column scales and the column maxima
    __nv_bfloat16 *OGT, *OGX, *OGL;   // OGL: row slices of one diagonal-tile inverse (7 x b x b)
    __nv_bfloat16* OGTS;              // columns of GP_OG_SP row blocks of L^{-1} (7 x Np x SP b)
    double* ogl_mu;
    double *ogt_mu, *ogx_mu;
    unsigned long long* ogx_bits;
    // GP_FP64_OZAKI prediction: test columns of one row block of V (7 x m_cap x b), all of V
    // (7 x m_cap x Np, allocated with the full covariance), their scales and column maxima
    __nv_bfloat16 *OGV, *OGC, *OGVS;   // OGVS: columns of GP_OG_SP row blocks of V (7 x m_cap x SP b)
    double *ogv_mu, *ogc_mu;
    unsigned long long* ogc_bits;
    int64_t ogc_cap;
    int64_t dp;               // regressors padded to a multiple of 32
    __nv_bfloat16* ZXS;       // digit slices of the training rows, 6 x Np x dp
    double *zx_mu, *zx_nrm;   // their row scales and |zhat|^2 (Np)
    __nv_bfloat16* ZSS;       // digit slices of the test rows, 6 x m_cap x dp
    double *zs_mu, *zs_nrm;   // their row scales and |zhat|^2 (m_cap)
    bool tc_pending;          // a tensor-core kernel ran since its timeout word was last read
    int* solve_flags;         // grid barrier of the persistent FP32 solve and of the grid POTRF: count, generation
    __nv_bfloat16* ZP;        // T(T+1)/2 tiles x 3 planes of (L^{-1})^T tiles (gradient)
    float* U32;               // T(T+1)/2 tiles: TRTRI accumulators (gradient)
    float* Kinv32;            // T(T+1)/2 tiles: K^{-1} lower (gradient)

    // Persistent tile-DAG scheduler (GP_SCHED_PERSISTENT).
    int* dag_tasks;           // int4 (type, i, j, k) per task, topological order
    int64_t dag_ntasks;
    int* dag_ctl;             // [0] ticket, [1] abort code (1 timeout, 2 pivot)
    int* dag_upd;             // T(T+1)/2 update counters
    int* dag_fin;             // T(T+1)/2 final flags
    int64_t dag_stall;        // test aid: tile whose counter is poisoned (-1: none)
    bool solve_stall;         // test aid: the last CTA of each persistent FP32 solve never arrives
    long long solve_wait_cycles;   // bound on one grid-barrier wait of the persistent FP32 solve

    int64_t bytes;            // device bytes held
    int64_t last_info;
    int refine_iters;
    double refine_residual;
    double jitter_added;      // sigma^2 added by the last factorisation's NOT_PD retries

    // Launch accounting and optional per-launch event timing (gp_profile).
    int64_t launches;
    bool prof_on;
    cudaEvent_t* ev_pool;     // grown on demand
    int64_t ev_cap, ev_used;
    int* ev_phase;            // phase of each recorded (start, stop) pair
    double prof_ms[GP_NPHASE];
    int64_t prof_cnt[GP_NPHASE];
};

// Launch wrapper: counts the launch and, when profiling is on, brackets it
// with a pair of events tagged with its phase.
bool prof_begin(gp_t h, int phase);
void prof_end(gp_t h);
#define GPK_LAUNCH(h, phase, kern, grid, block, smem, ...)                   \
    do {                                                                     \
        bool p_ = (h)->prof_on && prof_begin((h), (phase));                  \
        kern<<<(grid), (block), (smem), (h)->st>>>(__VA_ARGS__);             \
        (h)->launches++;                                                     \
        if (p_) prof_end(h);                                                 \
    } while (0)

// ---------------------------------------------------------------- kernels.cu
namespace gpk {
void assemble_train(gp_t h);                                   // K tiles into h->L
void assemble_cross(gp_t h, int64_t m, int64_t ldm);           // B = K_{Z*,Z}^T (Np x ldm)
void assemble_test_prior(gp_t h, int64_t m, double* out);      // out = K_{Z*,Z*} (+ noise), m x m
bool factor_fp64(gp_t h);                                      // tiled Cholesky in place (false: host set-up failed)
bool og_chol_update_cols(gp_t h, int64_t k, int64_t e);         // GP_FP64_OZAKI: columns k+1..e-1 by column k
bool og_chol_update_sp(gp_t h, int64_t K0, int64_t e);          // GP_FP64_OZAKI: trailing update by a super-panel
constexpr int GP_OG_SP = 4;                                     // GP_FP64_OZAKI super-panel width (tile columns)
bool og_trtri_accum(gp_t h, int64_t t, int64_t e);             // GP_FP64_OZAKI inverse: S_ij += L_it X_tj, i < e
bool og_trtri_accum_sp(gp_t h, int64_t T0, int64_t e);          // ... by row blocks T0..e-1 for i >= e
bool og_lauum(gp_t h);                                         // GP_FP64_OZAKI K^{-1} = X^T X
bool og_vsolve_update(gp_t h, int64_t j, int64_t e, int64_t ldm);   // GP_FP64_OZAKI V solve: B_i -= L_ij V_j, i < e
bool og_vsolve_update_sp(gp_t h, int64_t J0, int64_t e, int64_t ldm);   // ... by columns J0..e-1 for i >= e
bool og_vsolve_diag(gp_t h, int64_t j, int64_t ldm);            // GP_FP64_OZAKI V solve: V_j = Linv_jj B_j
bool og_panel(gp_t h, int64_t k);                              // GP_FP64_OZAKI panel: L_ik = A_ik Linv_kk^T
bool og_trtri_scale(gp_t h, int64_t t);                        // GP_FP64_OZAKI inverse: X_tj = -Linv_tt S_tj
bool og_full_cov(gp_t h, int64_t m, int64_t ldm, double* cov);  // GP_FP64_OZAKI cov -= V^T V
void solve_lower(gp_t h, const double* rhs, double* out);      // out = L^{-1} rhs
void solve_upper(gp_t h, const double* rhs, double* out);      // out = L^{-T} rhs
void nlml_reduce(gp_t h);                                      // scal[0] = NLML
bool predict_solve(gp_t h, int64_t m, int64_t ldm);            // V, partial sums (false: host set-up failed)
void predict_finish(gp_t h, int64_t m, int64_t ldm, bool want_var);  // outm, outv
void predict_mean_only(gp_t h, int64_t m, int64_t ldm);      // outm = K_{Z*,Z} alpha
bool full_cov(gp_t h, int64_t m, int64_t ldm, double* cov);    // cov -= V^T V (mirrored; false: host set-up failed)
bool inverse_tiles(gp_t h);                                    // Xinv = L^{-1}, Kinv = K^{-1} (false: host set-up failed)
void adjoint_grad(gp_t h);                                     // scal[1..3] = grad
void adam_step(gp_t h, double lr, double* hist_slot);          // Adam on log theta
void copy_factor_dense(gp_t h, double* out);                   // L as dense n x n
void set_info_none(gp_t h);
// FP64 POTRF + inverse of one b x b diagonal tile A (in place) into X; adds
// sum log L_ii to *logdet_slot; a failing pivot records row0 + its row.
void potrf_diag_launch(gp_t h, double* A, double* X, int64_t b, int64_t row0, double* logdet_slot);
// The same on the whole GPU (one cooperative launch, bounded grid barriers on
// h->solve_flags); b a multiple of 32.  False if it cannot be launched.
bool potrf_diag_grid(gp_t h, double* A, double* X, int64_t b, int64_t row0, double* logdet_slot);
// FP32 factor and inverse of an FP32 tile on one cluster of eight CTAs
// (kernels_potrf_cl.cu): A32 (lower, in place) = L, X32 = L^{-1}, XP = its
// three BF16 planes, sum log L_jj (FP64) into *logdet_slot; b a multiple of 32.
bool potrf_diag_cl32(gp_t h, float* A32, float* X32, __nv_bfloat16* XP, int64_t b, int64_t row0,
                     double* logdet_slot);
void factor_dag(gp_t h, bool reset_err);                       // persistent tile-DAG factor (FP64)

// kernels_mixed.cu
bool factor_mixed(gp_t h);                                     // mixed factor of h->A32
void refine_start(gp_t h, const double* rhs, double* x);       // x = L~^{-T} L~^{-1} rhs
void refine_residual(gp_t h, const double* rhs, const double* x, double* r,
                     double* norms);                             // r = rhs - K x (FP64), ||r||^2, ||rhs||^2
void refine_correct(gp_t h, const double* r, double* x);        // x += L~^{-T} L~^{-1} r (FP32 solves)
void residual64(gp_t h, const double* x, const double* y, double* r);              // r = y - K x (FP64)
void nlml_mixed(gp_t h);                                       // scal[0] from y^T alpha and log|K|
bool predict_mixed(gp_t h, int64_t m, int64_t ldm, bool want_var, bool want_cov);
void copy_factor_dense_mixed(gp_t h, double* out);
bool full_cov_mixed(gp_t h, int64_t m, int64_t ldm, double* cov);  // cov (prefilled prior) -= W W^T
bool inverse_mixed(gp_t h);                                    // Kinv32 = (L~ L~^T)^{-1}
bool var_correction_mixed(gp_t h, int64_t m, int64_t ldm);     // FP64-level variances into outv
// kernels_tc.cu
bool ozaki_tc(gp_t h, int64_t m, int64_t ldm);                  // C = Y K digit-pair product + fused epilogue
cudaError_t tc_error_fetch(gp_t h, int* out);                   // read and clear the tensor-core timeout word
int* tc_error_dev();                                            // device address of that word
// kernels_tgemm.cu: split-BF16 block products on tcgen05 (false: tensor map not encodable)
bool tg_panel(gp_t h, int64_t k);
bool tg_update(gp_t h, int k0, int nsrc, int j0, int w);   // A_ij -= sum_k L_ik L_jk^T on a column band
// The four multi-RHS sweep products take planes = 3 (six plane products, FP32
// accuracy) or 2 (the three of order <= 2^-8, about 2^-16 relative).
bool tg_diag_w(gp_t h, int phase, float* R, int64_t ldm, double* vpart, int64_t j, int planes);
// W_I = R_I X_I^T for super-block I (R_I planes in RP), W planes, FP32 W, row sums of W^2
bool tg_diag_w_sb(gp_t h, int phase, float* R, int64_t ldm, double* vpart, int64_t I, int planes);
bool tg_upd_w(gp_t h, int phase, float* R, int64_t ldm, int j0, int nsrc, int i0, int ni,
              int planes);   // R_i -= sum W_j L_ij^T
bool tg_syrk_cov(gp_t h, int64_t m, int64_t ldm, double* cov);
bool tg_trtri_fin(gp_t h, int64_t t);
bool tg_trtri_acc(gp_t h, int t0, int t1, int i0, int ni, int nj);   // U_ij (+)= sum_t Z_tj L_it^T
bool tg_lauum(gp_t h);
// squared distances on the tensor cores (kernels_dist.cu, kernels_mixed.cu)
bool use_tc_dist(gp_t h);
void zslices(gp_t h, const double* Z, const double* center, int64_t rows, int64_t valid, __nv_bfloat16* ZS,
             double* mu, double* nrm, int phase);                 // digits of Z - center (one row of d)
bool dist_train_tc(gp_t h);                                     // K tiles into L (FP64) and A32
bool dist_cross_tc(gp_t h, int64_t m, int64_t ldm);             // R32, R64, mean partials
bool dist_prior_tc(gp_t h, int64_t m, int64_t ldm, double* out);   // K_{Z*,Z*} (m x m)
bool tg_bdiag_sb(gp_t h, int64_t ldm, int64_t I, int planes);   // Y_I = S_I X_I (NN form), super-block I
bool tg_bupd(gp_t h, int64_t ldm, int i0, int nsrc, int j0, int nj, int planes);   // S_j -= sum Y_i L_ij (NN form)
constexpr int GP_SOLVE_SB = 4;                                 // tiles per super-block of the FP32 solves
constexpr int GP_OZ_SLICES = 6;                                // digit slices of K (kernels_mixed.cu)
constexpr int GP_OZ_YSLICES = 2;                               // digit slices of x~0: x0 rounded to 14 bits per row
constexpr int GP_OZ_BITS = 7;                                   // bits per signed digit: |d| <= 2^7, exact in BF16
constexpr int GP_OG_SLICES = 7;                                // GP_FP64_OZAKI: 7-bit digits per operand (49 bits)
constexpr int GP_TC_DIST_MIN_D = 32;                           // mixed path: tensor-core distances from this d up
constexpr int GP_OZ_LMAX = 7;                                   // digit pairs (s, u) with s + u <= 7 enter K x~0
}  // namespace gpk

#define GP_CUDA_OK(call)                                                   \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return e_;                                  \
    } while (0)
