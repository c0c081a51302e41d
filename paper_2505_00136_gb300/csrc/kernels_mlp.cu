// Learned hyperparameter initialiser (not in the paper): a 64-d summary of a
// data set, a 64 -> 256 -> 256 -> 3 ReLU MLP whose outputs are initial
// (log l, log nu, log sigma^2), its MSE gradient and an Adam step on its
// weights.  Summaries in FP64; the network in FP32.
//
// Model blob (floats): W1[256][64] b1[256] W2[256][256] b2[256] W3[3][256] b3[3]
// (GP_MLP_NPARAM trained values), then feature mean[64] and std[64] used to
// standardise the summary.
#include <math.h>
#include <stdint.h>

#include "../../include/gprat_gb.h"

namespace gpk {

constexpr int IN = 64, H = 256, OUT = 3;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * IN, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + OUT * H, NPARAM = OFF_B3 + OUT;
constexpr int OFF_MEAN = NPARAM, OFF_STD = OFF_MEAN + IN, NMODEL = OFF_STD + IN;
static_assert(NPARAM == GP_MLP_NPARAM, "parameter count");
static_assert(NMODEL == GP_MLP_MODEL_FLOATS, "model size");
constexpr int SB = 16;        // samples per CTA
constexpr int NT = 256;

__device__ double block_sum(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

// s[0..31]: per-regressor standard deviations, descending, zero-padded;
// s[32..47]: autocorrelation of y at lags 1..16; s[48..63]: means of
// cos(omega_q y) and sin(omega_q y).  One CTA per data set.
__global__ __launch_bounds__(NT) void k_summary(const double* X, const double* y, int64_t n, int64_t d,
                                                const double* omega, double* s)
{
    __shared__ double red[NT];
    __shared__ double sd[1024];
    for (int64_t k = threadIdx.x; k < d; k += NT) {
        double mu = 0.0;
        for (int64_t i = 0; i < n; ++i) mu += X[i * d + k];
        mu /= (double)n;
        double v = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double t = X[i * d + k] - mu;
            v = fma(t, t, v);
        }
        sd[k] = sqrt(v / (double)n);
    }
    __syncthreads();
    if (threadIdx.x == 0) {   // insertion sort, descending
        for (int64_t a = 1; a < d; ++a) {
            double v = sd[a];
            int64_t b = a - 1;
            while (b >= 0 && sd[b] < v) { sd[b + 1] = sd[b]; --b; }
            sd[b + 1] = v;
        }
        for (int q = 0; q < 32; ++q) s[q] = (q < d) ? sd[q] : 0.0;
    }
    __syncthreads();
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += NT) acc += y[i];
    const double ybar = block_sum(acc, red) / (double)n;
    acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += NT) acc = fma(y[i] - ybar, y[i] - ybar, acc);
    const double c0 = block_sum(acc, red);
    for (int lag = 1; lag <= 16; ++lag) {
        acc = 0.0;
        for (int64_t i = threadIdx.x; i + lag < n; i += NT) acc = fma(y[i] - ybar, y[i + lag] - ybar, acc);
        const double c = block_sum(acc, red);
        if (threadIdx.x == 0) s[31 + lag] = (c0 > 0.0) ? c / c0 : 0.0;
    }
    for (int q = 0; q < 8; ++q) {
        double cs = 0.0, sn = 0.0;
        for (int64_t i = threadIdx.x; i < n; i += NT) {
            double sv, cv;
            sincos(omega[q] * y[i], &sv, &cv);
            cs += cv;
            sn += sv;
        }
        cs = block_sum(cs, red);
        sn = block_sum(sn, red);
        if (threadIdx.x == 0) {
            s[48 + 2 * q] = cs / (double)n;
            s[49 + 2 * q] = sn / (double)n;
        }
    }
}

// Feature mean and standard deviation over B summaries into the model blob
// (a zero spread becomes 1).  One thread per feature.
__global__ void k_feat_stats(const double* S, int64_t B, float* model)
{
    const int f = threadIdx.x;
    if (f >= IN) return;
    double mu = 0.0;
    for (int64_t b = 0; b < B; ++b) mu += S[b * IN + f];
    mu /= (double)B;
    double v = 0.0;
    for (int64_t b = 0; b < B; ++b) v += (S[b * IN + f] - mu) * (S[b * IN + f] - mu);
    const double sd = sqrt(v / (double)B);
    model[OFF_MEAN + f] = (float)mu;
    model[OFF_STD + f] = sd > 0.0 ? (float)sd : 1.f;
}

// out[b][j] = act(bias[j] + sum_k W[j][k] in[b][k]) for SB samples; warp per
// output unit, lanes over k (coalesced weight rows), in[] in shared memory.
template <int K, int OW, bool RELU>
__device__ void dense_rows(const float* W, const float* bias, const float (*in)[K], float (*out)[OW], int nout)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = warp; j < nout; j += NT / 32) {
        float acc[SB];
#pragma unroll
        for (int b = 0; b < SB; ++b) acc[b] = 0.f;
        for (int k = lane; k < K; k += 32) {
            const float w = W[j * K + k];
#pragma unroll
            for (int b = 0; b < SB; ++b) acc[b] = fmaf(w, in[b][k], acc[b]);
        }
#pragma unroll
        for (int b = 0; b < SB; ++b) {
            float v = acc[b];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) {
                v += bias[j];
                out[b][j] = RELU ? fmaxf(v, 0.f) : v;
            }
        }
    }
}

// Standardised inputs and the two hidden layers for samples b0 .. b0+SB-1.
__device__ void mlp_forward_block(const float* model, const double* S, int64_t B, int64_t b0, float (*x)[IN],
                                  float (*h1)[H], float (*h2)[H], float (*o)[4])
{
    for (int e = threadIdx.x; e < SB * IN; e += NT) {
        const int b = e / IN, f = e % IN;
        const int64_t gb = b0 + b;
        x[b][f] = (gb < B) ? (float)((S[gb * IN + f] - (double)model[OFF_MEAN + f]) / (double)model[OFF_STD + f])
                           : 0.f;
    }
    __syncthreads();
    dense_rows<IN, H, true>(model + OFF_W1, model + OFF_B1, x, h1, H);
    __syncthreads();
    dense_rows<H, H, true>(model + OFF_W2, model + OFF_B2, h1, h2, H);
    __syncthreads();
    dense_rows<H, 4, false>(model + OFF_W3, model + OFF_B3, h2, o, OUT);
    __syncthreads();
}

__global__ __launch_bounds__(NT) void k_mlp_forward(const float* model, const double* S, int64_t B, float* out)
{
    __shared__ float x[SB][IN], h1[SB][H], h2[SB][H], o[SB][4];
    const int64_t b0 = (int64_t)blockIdx.x * SB;
    mlp_forward_block(model, S, B, b0, x, h1, h2, o);
    for (int e = threadIdx.x; e < SB * OUT; e += NT) {
        const int b = e / OUT, q = e % OUT;
        if (b0 + b < B) out[(b0 + b) * OUT + q] = o[b][q];
    }
}

// Loss 1/(3B) sum (o - t)^2 and its gradient for SB samples: per-CTA partial
// weight gradients into part[blockIdx.x][NPARAM], partial loss into lpart.
__global__ __launch_bounds__(NT) void k_mlp_backward(const float* model, const double* S, const float* target,
                                                     int64_t B, float* part, float* lpart)
{
    __shared__ float x[SB][IN], h1[SB][H], h2[SB][H], o[SB][4];
    __shared__ float dO[SB][OUT];
    __shared__ float red[NT];
    const int64_t b0 = (int64_t)blockIdx.x * SB;
    mlp_forward_block(model, S, B, b0, x, h1, h2, o);
    const float scale = 1.f / (3.f * (float)B);
    float l = 0.f;
    if (threadIdx.x < SB * OUT) {
        const int b = threadIdx.x / OUT, q = threadIdx.x % OUT;
        float e = 0.f;
        if (b0 + b < B) e = o[b][q] - target[(b0 + b) * OUT + q];
        l = e * e * scale;
        dO[b][q] = 2.f * e * scale;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) lpart[blockIdx.x] = red[0];
    float* g = part + (int64_t)blockIdx.x * NPARAM;
    const float* W2 = model + OFF_W2;
    const float* W3 = model + OFF_W3;
    const int q = threadIdx.x;   // hidden unit owned by this thread
    // layer 3: gW3[j][q] = sum_b dO[b][j] h2[b][q], gb3; dh2 = (W3^T dO) * [h2 > 0],
    // written over h2 (thread q owns column q)
    {
        float g3[OUT] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int b = 0; b < SB; ++b) {
            float d2 = 0.f;
#pragma unroll
            for (int j = 0; j < OUT; ++j) {
                g3[j] = fmaf(dO[b][j], h2[b][q], g3[j]);
                d2 = fmaf(W3[j * H + q], dO[b][j], d2);
            }
            h2[b][q] = h2[b][q] > 0.f ? d2 : 0.f;
        }
#pragma unroll
        for (int j = 0; j < OUT; ++j) g[OFF_W3 + j * H + q] = g3[j];
        if (q < OUT) {
            float s = 0.f;
#pragma unroll
            for (int b = 0; b < SB; ++b) s += dO[b][q];
            g[OFF_B3 + q] = s;
        }
    }
    __syncthreads();
    // layer 2: gW2[q][k] = sum_b dh2[b][q] h1[b][k] (thread q writes its row), gb2;
    // dh1[b][k] = (sum_j W2[j][k] dh2[b][j]) * [h1 > 0] (thread k), written over h1
    // once every thread has finished reading h1
    {
        float gb = 0.f;
#pragma unroll
        for (int b = 0; b < SB; ++b) gb += h2[b][q];
        g[OFF_B2 + q] = gb;
        for (int k = 0; k < H; ++k) {
            float s = 0.f;
#pragma unroll
            for (int b = 0; b < SB; ++b) s = fmaf(h2[b][q], h1[b][k], s);
            g[OFF_W2 + q * H + k] = s;
        }
        const int k = threadIdx.x;
        float d1[SB];
#pragma unroll
        for (int b = 0; b < SB; ++b) d1[b] = 0.f;
        for (int j = 0; j < H; ++j) {
            const float w = W2[j * H + k];
#pragma unroll
            for (int b = 0; b < SB; ++b) d1[b] = fmaf(w, h2[b][j], d1[b]);
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < SB; ++b) h1[b][k] = h1[b][k] > 0.f ? d1[b] : 0.f;
    }
    __syncthreads();
    // layer 1: gW1[q][f] = sum_b dh1[b][q] x[b][f], gb1
    {
        float gb = 0.f;
#pragma unroll
        for (int b = 0; b < SB; ++b) gb += h1[b][q];
        g[OFF_B1 + q] = gb;
        for (int f = 0; f < IN; ++f) {
            float s = 0.f;
#pragma unroll
            for (int b = 0; b < SB; ++b) s = fmaf(h1[b][q], x[b][f], s);
            g[OFF_W1 + q * IN + f] = s;
        }
    }
}

// gW = sum over CTAs of the partial gradients; loss = sum of the partial losses.
__global__ void k_mlp_reduce(const float* part, const float* lpart, int64_t nblk, float* gW, float* loss)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NPARAM) {
        float s = 0.f;
        for (int64_t c = 0; c < nblk; ++c) s += part[c * NPARAM + p];
        gW[p] = s;
    }
    if (p == 0 && loss) {
        float s = 0.f;
        for (int64_t c = 0; c < nblk; ++c) s += lpart[c];
        *loss = s;
    }
}

// Adam (Kingma & Ba 2015) on the trained weights; t >= 1 is the step number.
__global__ void k_mlp_adam(float* W, const float* g, float* m, float* v, int64_t count, float c1, float c2,
                           float lr, float b1, float b2, float eps)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= count) return;
    const float gp = g[p];
    const float mp = b1 * m[p] + (1.f - b1) * gp;
    const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
    m[p] = mp;
    v[p] = vp;
    W[p] -= lr * (mp / c1) / (sqrtf(vp / c2) + eps);
}

// (log l, log nu, log sigma^2) -> natural scale for gp_learned_init.
__global__ void k_theta_out(const float* o, double* out)
{
    if (threadIdx.x < 3) out[threadIdx.x] = exp((double)o[threadIdx.x]);
}

}  // namespace gpk

using namespace gpk;

namespace {
// Managed memory or device memory of the current device (memory of another
// GPU is refused by the device-only calls and copied by gp_learned_init).
bool dev_ptr(const void* p)
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
gp_status launched() { return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA; }
int64_t nblocks(int64_t B) { return (B + SB - 1) / SB; }
}  // namespace

extern "C" {

gp_status gp_summary(const double* X, const double* y, int64_t n, int64_t d, const double* omega, double* s,
                     void* stream)
{
    if (!X || !y || !omega || !s || n < 2 || d < 1 || d > 1024) return GP_ERR_ARG;
    if (!dev_ptr(X) || !dev_ptr(y) || !dev_ptr(omega) || !dev_ptr(s)) return GP_ERR_ARG;
    k_summary<<<1, NT, 0, (cudaStream_t)stream>>>(X, y, n, d, omega, s);
    return launched();
}

gp_status gp_mlp_feature_stats(const double* S, int64_t B, float* model, void* stream)
{
    if (!S || !model || B < 1 || !dev_ptr(S) || !dev_ptr(model)) return GP_ERR_ARG;
    k_feat_stats<<<1, IN, 0, (cudaStream_t)stream>>>(S, B, model);
    return launched();
}

int64_t gp_mlp_workspace_floats(int64_t B) { return B < 1 ? 0 : nblocks(B) * (NPARAM + 1); }

gp_status gp_mlp_forward(const float* model, const double* S, int64_t B, float* out, void* stream)
{
    if (!model || !S || !out || B < 1 || !dev_ptr(model) || !dev_ptr(S) || !dev_ptr(out)) return GP_ERR_ARG;
    k_mlp_forward<<<(unsigned)nblocks(B), NT, 0, (cudaStream_t)stream>>>(model, S, B, out);
    return launched();
}

gp_status gp_mlp_loss_grad(const float* model, const double* S, const float* target, int64_t B, float* gW,
                           float* loss, float* workspace, void* stream)
{
    if (!model || !S || !target || !gW || !workspace || B < 1) return GP_ERR_ARG;
    if (!dev_ptr(model) || !dev_ptr(S) || !dev_ptr(target) || !dev_ptr(gW) || !dev_ptr(workspace) ||
        (loss && !dev_ptr(loss)))
        return GP_ERR_ARG;
    const int64_t nb = nblocks(B);
    float* part = workspace;
    float* lpart = workspace + nb * NPARAM;
    cudaStream_t st = (cudaStream_t)stream;
    k_mlp_backward<<<(unsigned)nb, NT, 0, st>>>(model, S, target, B, part, lpart);
    k_mlp_reduce<<<(unsigned)((NPARAM + 255) / 256), 256, 0, st>>>(part, lpart, nb, gW, loss);
    return launched();
}

gp_status gp_mlp_adam(float* model, const float* gW, float* m, float* v, int64_t t, double lr, double beta1,
                      double beta2, double eps, void* stream)
{
    if (!model || !gW || !m || !v || t < 1 || !(lr > 0.0)) return GP_ERR_ARG;
    if (!dev_ptr(model) || !dev_ptr(gW) || !dev_ptr(m) || !dev_ptr(v)) return GP_ERR_ARG;
    const float c1 = (float)(1.0 - pow(beta1, (double)t)), c2 = (float)(1.0 - pow(beta2, (double)t));
    k_mlp_adam<<<(unsigned)((NPARAM + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        model, gW, m, v, NPARAM, c1, c2, (float)lr, (float)beta1, (float)beta2, (float)eps);
    return launched();
}

gp_status gp_learned_init(const double* X, const double* y, int64_t n, int64_t d, const float* model,
                          const double* omega, double* scratch, gp_hyper* out, void* stream)
{
    if (!X || !y || !model || !omega || !out || n < 2 || d < 1 || d > 1024) return GP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // Host arguments, those in another GPU's memory, and a NULL or host scratch
    // are staged in stream-ordered device memory for this call and released
    // before it returns.
    void* staged[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int ns = 0;
    bool ok = true;
    auto on_device = [&](const void* p, size_t bytes, bool copy) -> const void* {
        if (!ok) return nullptr;
        if (p && dev_ptr(p)) return p;
        void* q = nullptr;
        if (cudaMallocAsync(&q, bytes, st) != cudaSuccess) {
            ok = false;
            return nullptr;
        }
        staged[ns++] = q;
        if (copy && cudaMemcpyAsync(q, p, bytes, cudaMemcpyDefault, st) != cudaSuccess) ok = false;
        return q;
    };
    const double* Xd = (const double*)on_device(X, (size_t)(n * d) * sizeof(double), true);
    const double* yd = (const double*)on_device(y, (size_t)n * sizeof(double), true);
    const float* md = (const float*)on_device(model, (size_t)GP_MLP_MODEL_FLOATS * sizeof(float), true);
    const double* od = (const double*)on_device(omega, 8 * sizeof(double), true);
    double* sd = (double*)on_device(scratch, GP_LEARNED_INIT_SCRATCH * sizeof(double), false);
    double th[3];
    if (ok) {
        // scratch (doubles): [0..63] summary, [64..66] theta, [68..69] the 3 floats of network output
        float* o = (float*)(sd + 68);
        k_summary<<<1, NT, 0, st>>>(Xd, yd, n, d, od, sd);
        k_mlp_forward<<<1, NT, 0, st>>>(md, sd, 1, o);
        k_theta_out<<<1, 32, 0, st>>>(o, sd + 64);
        if (cudaMemcpyAsync(th, sd + 64, sizeof(th), cudaMemcpyDeviceToHost, st) != cudaSuccess) ok = false;
    }
    for (int i = 0; i < ns; ++i) cudaFreeAsync(staged[i], st);
    if (cudaStreamSynchronize(st) != cudaSuccess || !ok) return GP_ERR_CUDA;
    if (!(th[0] > 0.0) || !(th[1] > 0.0) || !(th[2] >= 0.0) || !isfinite(th[0]) || !isfinite(th[1]) ||
        !isfinite(th[2]))
        return GP_ERR_STATE;
    out->lengthscale = th[0];
    out->vertical = th[1];
    out->noise_var = th[2];
    out->trainable[0] = out->trainable[1] = out->trainable[2] = 1;
    return launched();
}

}  // extern "C"
