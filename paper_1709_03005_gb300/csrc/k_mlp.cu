// Learned Davidson preconditioner: a small MLP that scales the diagonal
// correction row by row (not in the paper; plain diagonal Davidson remains the
// fallback and the reference).
//
//   t_i = w(f_i) r_i / (H_ii - theta),   w = 256^tanh(o),   o = MLP(f)
//   MLP: h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), o = w3 . h2 + b3
// with n_in = 8 features, width 64, weights rounded to FP16 in the forward
// pass (inference stores them as FP16) and FP32 accumulation.
//
// Features of row i for a Ritz value theta (all divided by 10 Eh except f1):
//   f0 = (H_ii - theta), f1 = log(|H_ii - theta| + 1e-3), f2 = 1 for an L2 row,
//   f3 = E_n - theta for a continuum row of target state n (0 for L2),
//   f4 = h_jj of its continuum orbital (0 for L2), f5 = theta - theta_0,
//   f6 = H_ii, f7 = group index / number of groups (1 for L2).
// The range [1/256, 256] lets the factor damp rows whose H_ii - theta is small
// by two orders of magnitude (a shifted denominator |d| / (|d| + delta) does
// that, and a floor of 1/4 loses its gain).  Training minimises
// sum_i (w(f_i) a_i - b_i)^2 for given targets a, b (a = 1 and b a wanted
// factor fits the factor itself); the gradient is taken by a hand-written backward
// pass whose weight gradients are fixed-order chunked sums.
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "hb_davidson.cuh"

namespace hb {

constexpr int MLP_IN = 8, MLP_W = 64;
constexpr int MLP_NPARAM = MLP_W * MLP_IN + MLP_W + MLP_W * MLP_W + MLP_W + MLP_W + 1;   // 4801

struct MlpState {
    __half *wh = nullptr;        // FP16 weights (packed like the parameters)
    float *bias = nullptr;       // FP32 copy of every parameter (biases read from here)
    float *row_info = nullptr;   // [4][n]: type, E_n, h_jj, group/n_groups
    float *w = nullptr;          // [mmax][n] factors for the current iteration
    float *feats = nullptr;      // scratch features
    int64_t n = 0;
    int mmax = 0;
    bool rows_ready = false;
};

}  // namespace hb

using namespace hb;

namespace {

constexpr float kLogR = 5.545177444479562f;   // log 256: w in [1/256, 256]

// offsets inside the packed parameter vector
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_W * MLP_IN, OFF_W2 = OFF_B1 + MLP_W, OFF_B2 = OFF_W2 + MLP_W * MLP_W,
              OFF_W3 = OFF_B2 + MLP_W, OFF_B3 = OFF_W3 + MLP_W;

__device__ __forceinline__ float q16(float x) { return __half2float(__float2half_rn(x)); }

// row features for one (row, theta)
__device__ __forceinline__ void features(float d, float theta, float theta0, const float *ri, int64_t i, int64_t n,
                                         float (&f)[MLP_IN]) {
    const float type = ri[i], En = ri[n + i], hj = ri[2 * n + i], gid = ri[3 * n + i];
    const float gap = d - theta;
    f[0] = gap * 0.1f;
    f[1] = logf(fabsf(gap) + 1e-3f);
    f[2] = type;
    f[3] = type > 0.5f ? 0.0f : (En - theta) * 0.1f;
    f[4] = hj * 0.1f;
    f[5] = (theta - theta0) * 0.1f;
    f[6] = d * 0.1f;
    f[7] = gid;
}

// forward pass with weights from shared memory; returns o, fills h1, h2
__device__ __forceinline__ float mlp_forward(const float *P, const float (&f)[MLP_IN], float (&h1)[MLP_W],
                                             float (&h2)[MLP_W]) {
#pragma unroll 4
    for (int a = 0; a < MLP_W; ++a) {
        float s = P[OFF_B1 + a];
#pragma unroll
        for (int c = 0; c < MLP_IN; ++c) s = fmaf(P[OFF_W1 + a * MLP_IN + c], f[c], s);
        h1[a] = fmaxf(s, 0.0f);
    }
#pragma unroll 2
    for (int a = 0; a < MLP_W; ++a) {
        float s = P[OFF_B2 + a];
#pragma unroll
        for (int c = 0; c < MLP_W; ++c) s = fmaf(P[OFF_W2 + a * MLP_W + c], h1[c], s);
        h2[a] = fmaxf(s, 0.0f);
    }
    float o = P[OFF_B3];
#pragma unroll
    for (int c = 0; c < MLP_W; ++c) o = fmaf(P[OFF_W3 + c], h2[c], o);
    return o;
}

// stage the parameters (weights rounded to FP16) in shared memory
__device__ __forceinline__ void stage_params(const float *params, float *P) {
    for (int t = threadIdx.x; t < MLP_NPARAM; t += blockDim.x) {
        const bool is_bias = (t >= OFF_B1 && t < OFF_W2) || (t >= OFF_B2 && t < OFF_W3) || t == OFF_B3;
        P[t] = is_bias ? params[t] : q16(params[t]);
    }
    __syncthreads();
}

// ---------------------------------------------------------------- training
// Per sample: loss (w a - b)^2, and the deltas needed by the weight gradients.
__global__ void mlp_fwd_bwd_kernel(const float *__restrict__ params, const float *__restrict__ feats,
                                   const float *__restrict__ ta, const float *__restrict__ tb, int64_t n,
                                   float *__restrict__ H1, float *__restrict__ D1, float *__restrict__ H2,
                                   float *__restrict__ D2, float *__restrict__ DO, float *__restrict__ loss) {
    __shared__ float P[MLP_NPARAM];
    stage_params(params, P);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float f[MLP_IN], h1[MLP_W], h2[MLP_W];
#pragma unroll
    for (int c = 0; c < MLP_IN; ++c) f[c] = feats[i * MLP_IN + c];
    const float o = mlp_forward(P, f, h1, h2);
    const float th = tanhf(o);
    const float w = expf(kLogR * th);
    const float a = ta[i], b = tb[i];
    const float err = w * a - b;
    loss[i] = err * err;
    const float dout = 2.0f * err * a * w * kLogR * (1.0f - th * th);   // dL/do
    DO[i] = dout;
    float d2[MLP_W];
#pragma unroll
    for (int c = 0; c < MLP_W; ++c) d2[c] = h2[c] > 0.0f ? dout * P[OFF_W3 + c] : 0.0f;
#pragma unroll 2
    for (int c = 0; c < MLP_W; ++c) {
        float s = 0.0f;
#pragma unroll
        for (int a2 = 0; a2 < MLP_W; ++a2) s = fmaf(P[OFF_W2 + a2 * MLP_W + c], d2[a2], s);
        D1[i * MLP_W + c] = h1[c] > 0.0f ? s : 0.0f;
    }
#pragma unroll
    for (int c = 0; c < MLP_W; ++c) {
        H1[i * MLP_W + c] = h1[c];
        H2[i * MLP_W + c] = h2[c];
        D2[i * MLP_W + c] = d2[c];
    }
}

// partial[c][t] for parameter t over samples of chunk c (fixed order)
constexpr int kMlpChunk = 1024;
__global__ void mlp_grad_partial_kernel(const float *__restrict__ feats, const float *__restrict__ H1,
                                        const float *__restrict__ D1, const float *__restrict__ H2,
                                        const float *__restrict__ D2, const float *__restrict__ DO,
                                        const float *__restrict__ loss, int64_t n, float *__restrict__ partial) {
    const int c = blockIdx.x;
    const int64_t i0 = (int64_t)c * kMlpChunk, i1 = (n < i0 + kMlpChunk) ? n : i0 + kMlpChunk;
    for (int t = threadIdx.x; t <= MLP_NPARAM; t += blockDim.x) {
        float s = 0.0f;
        if (t == MLP_NPARAM) {                         // the loss itself
            for (int64_t i = i0; i < i1; ++i) s += loss[i];
        } else if (t < OFF_B1) {                       // W1[a][c] = sum D1[a] f[c]
            const int a = t / MLP_IN, cc = t % MLP_IN;
            for (int64_t i = i0; i < i1; ++i) s = fmaf(D1[i * MLP_W + a], feats[i * MLP_IN + cc], s);
        } else if (t < OFF_W2) {                       // b1
            const int a = t - OFF_B1;
            for (int64_t i = i0; i < i1; ++i) s += D1[i * MLP_W + a];
        } else if (t < OFF_B2) {                       // W2[a][c] = sum D2[a] H1[c]
            const int a = (t - OFF_W2) / MLP_W, cc = (t - OFF_W2) % MLP_W;
            for (int64_t i = i0; i < i1; ++i) s = fmaf(D2[i * MLP_W + a], H1[i * MLP_W + cc], s);
        } else if (t < OFF_W3) {                       // b2
            const int a = t - OFF_B2;
            for (int64_t i = i0; i < i1; ++i) s += D2[i * MLP_W + a];
        } else if (t < OFF_B3) {                       // w3[c] = sum DO H2[c]
            const int cc = t - OFF_W3;
            for (int64_t i = i0; i < i1; ++i) s = fmaf(DO[i], H2[i * MLP_W + cc], s);
        } else {                                       // b3
            for (int64_t i = i0; i < i1; ++i) s += DO[i];
        }
        partial[(int64_t)c * (MLP_NPARAM + 1) + t] = s;
    }
}

__global__ void mlp_grad_reduce_kernel(const float *__restrict__ partial, int chunks, float scale,
                                       float *__restrict__ grads, float *__restrict__ loss_out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > MLP_NPARAM) return;
    float s = 0.0f;
    for (int c = 0; c < chunks; ++c) s += partial[(int64_t)c * (MLP_NPARAM + 1) + t];
    if (t == MLP_NPARAM) *loss_out = s * scale;
    else grads[t] = s * scale;
}

__global__ void adam_kernel(int64_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void mlp_predict_kernel(const float *__restrict__ params, const float *__restrict__ feats, int64_t n,
                                   float *__restrict__ out) {
    __shared__ float P[MLP_NPARAM];
    stage_params(params, P);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float f[MLP_IN], h1[MLP_W], h2[MLP_W];
#pragma unroll
    for (int c = 0; c < MLP_IN; ++c) f[c] = feats[i * MLP_IN + c];
    out[i] = expf(kLogR * tanhf(mlp_forward(P, f, h1, h2)));
}

// ------------------------------------------------------------ inside hb_diag
// features of every row for the Ritz values theta[which[j]] -> feats[j][n][8]
__global__ void diag_features_kernel(const double *__restrict__ d, const float *__restrict__ ri, int64_t n,
                                     const double *__restrict__ theta, int q, float *__restrict__ feats) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= n || j >= q) return;
    float f[MLP_IN];
    features((float)d[i], (float)theta[j], (float)theta[0], ri, i, n, f);
#pragma unroll
    for (int c = 0; c < MLP_IN; ++c) feats[((int64_t)j * n + i) * MLP_IN + c] = f[c];
}

// w[j][i] = MLP factor for row i and Ritz value theta[j] (FP16 weights)
__global__ void diag_mlp_kernel(const __half *__restrict__ wh, const float *__restrict__ params,
                                const double *__restrict__ d, const float *__restrict__ ri, int64_t n,
                                const double *__restrict__ theta, int q, float *__restrict__ w) {
    __shared__ float P[MLP_NPARAM];
    for (int t = threadIdx.x; t < MLP_NPARAM; t += blockDim.x) {
        const bool is_bias = (t >= OFF_B1 && t < OFF_W2) || (t >= OFF_B2 && t < OFF_W3) || t == OFF_B3;
        P[t] = is_bias ? params[t] : __half2float(wh[t]);
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= n || j >= q) return;
    float f[MLP_IN], h1[MLP_W], h2[MLP_W];
    features((float)d[i], (float)theta[j], (float)theta[0], ri, i, n, f);
    const float o = mlp_forward(P, f, h1, h2);
    float v = expf(kLogR * tanhf(o));
    if (!isfinite(v)) v = 1.0f;
    w[(int64_t)j * n + i] = v;
}

// row_info from the build: type, E_n, h_jj, group id
__global__ void row_info_kernel(int64_t row0, int ns, int cn, int cf, int n_to, int n_orb, const double *__restrict__ h,
                                const double *__restrict__ E, float gid, int64_t n, float *__restrict__ ri) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)ns * cn) return;
    const int st = (int)(t / cn), j = (int)(t % cn);
    const int64_t i = row0 + t;
    const int orb = n_to + cf + j;
    ri[i] = 0.0f;
    ri[n + i] = (float)E[st * ns + st];
    ri[2 * n + i] = (float)h[(int64_t)orb * n_orb + orb];
    ri[3 * n + i] = gid;
}

}  // namespace

// ------------------------------------------------------------------- host
static int mlp_fail(hb_ctx *ctx, int code, const std::string &m) {
    if (ctx) ctx->err = m;
    return code;
}

static int ensure_rows(hb_ctx *ctx, MlpState &M, DiagWork *w, cudaStream_t s) {
    const int64_t n = ctx->dim;
    if (M.n != n || !M.row_info) {
        dfree(ctx, M.row_info);
        M.row_info = nullptr;
        if (dmalloc_n(ctx, &M.row_info, (size_t)4 * n) != cudaSuccess) return HB_ERR_OOM;
        M.n = n;
        M.rows_ready = false;
    }
    if (M.rows_ready) return HB_OK;
    // L2 rows: type 1, group id 1; continuum rows per group from the last build
    std::vector<float> init(4 * n, 0.0f);
    for (int64_t i = ctx->Dc; i < n; ++i) { init[i] = 1.0f; init[3 * n + i] = 1.0f; }
    cudaMemcpyAsync(M.row_info, init.data(), sizeof(float) * 4 * n, cudaMemcpyHostToDevice, s);
    for (auto &P : ctx->gps) {
        if (!P.same) continue;
        const GroupInfo &G = ctx->groups[P.g];
        const int64_t cnt = (int64_t)G.ns * G.cn;
        row_info_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(
            G.row_off, G.ns, G.cn, G.cf, ctx->n_to, ctx->n_orb, ctx->h, P.E,
            ctx->n_groups > 1 ? (float)P.g / (float)ctx->n_groups : 0.0f, n, M.row_info);
    }
    cudaStreamSynchronize(s);
    M.rows_ready = true;
    (void)w;
    return HB_OK;
}

int hb::mlp_weights_for(hb_ctx *ctx, DiagWork *w, const double *theta, int nr, float **out, cudaStream_t s) {
    *out = nullptr;
    MlpState *M = (MlpState *)ctx->mlp;
    if (!M || !M->wh) return mlp_fail(ctx, HB_ERR_UNSUPPORTED, "no preconditioner network");
    if (ensure_rows(ctx, *M, w, s) != HB_OK) return HB_ERR_OOM;
    if (M->mmax < nr || !M->w) {
        dfree(ctx, M->w);
        M->w = nullptr;
        if (dmalloc_n(ctx, &M->w, (size_t)nr * ctx->dim) != cudaSuccess) return HB_ERR_OOM;
        M->mmax = nr;
    }
    // theta is already on the device in w->theta (hb_diag copies it before the call)
    dim3 g((unsigned)((ctx->dim + 127) / 128), nr);
    diag_mlp_kernel<<<g, 128, 0, s>>>(M->wh, M->bias, w->d, M->row_info, ctx->dim, w->theta, nr, M->w);
    if (cudaGetLastError() != cudaSuccess) return HB_ERR_CUDA;
    (void)theta;
    *out = M->w;
    return HB_OK;
}

void hb::release_mlp(hb_ctx *ctx) {
    MlpState *M = (MlpState *)ctx->mlp;
    if (!M) return;
    for (void *p : {(void *)M->wh, (void *)M->bias, (void *)M->row_info, (void *)M->w, (void *)M->feats})
        dfree(ctx, p);
    delete M;
    ctx->mlp = nullptr;
}

extern "C" int hb_mlp_param_count(int32_t n_in, int32_t width) {
    return (n_in == MLP_IN && width == MLP_W) ? MLP_NPARAM : -1;
}

extern "C" int hb_mlp_set(hb_ctx *ctx, const hb_mlp_weights *wt) {
    if (!ctx || !wt) return mlp_fail(ctx, HB_ERR_INVALID_ARG, "NULL argument");
    if (wt->n_in != MLP_IN || wt->width != MLP_W)
        return mlp_fail(ctx, HB_ERR_UNSUPPORTED, "the preconditioner network has 8 inputs and width 64");
    if (!wt->w1 || !wt->b1 || !wt->w2 || !wt->b2 || !wt->w3 || !wt->b3)
        return mlp_fail(ctx, HB_ERR_INVALID_ARG, "NULL weight array");
    std::vector<float> p(MLP_NPARAM);
    std::memcpy(&p[OFF_W1], wt->w1, sizeof(float) * MLP_W * MLP_IN);
    std::memcpy(&p[OFF_B1], wt->b1, sizeof(float) * MLP_W);
    std::memcpy(&p[OFF_W2], wt->w2, sizeof(float) * MLP_W * MLP_W);
    std::memcpy(&p[OFF_B2], wt->b2, sizeof(float) * MLP_W);
    std::memcpy(&p[OFF_W3], wt->w3, sizeof(float) * MLP_W);
    std::memcpy(&p[OFF_B3], wt->b3, sizeof(float));
    for (float x : p)
        if (!std::isfinite(x)) return mlp_fail(ctx, HB_ERR_INVALID_ARG, "non-finite weights");
    std::vector<__half> ph(MLP_NPARAM);
    for (int i = 0; i < MLP_NPARAM; ++i) ph[i] = __float2half_rn(p[i]);
    MlpState *M = (MlpState *)ctx->mlp;
    if (!M) { M = new MlpState(); ctx->mlp = M; }
    if (!M->wh && dmalloc_n(ctx, &M->wh, (size_t)MLP_NPARAM) != cudaSuccess) return HB_ERR_OOM;
    if (!M->bias && dmalloc_n(ctx, &M->bias, (size_t)MLP_NPARAM) != cudaSuccess) return HB_ERR_OOM;
    if (cudaMemcpy(M->wh, ph.data(), sizeof(__half) * MLP_NPARAM, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(M->bias, p.data(), sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice) != cudaSuccess)
        return mlp_fail(ctx, HB_ERR_CUDA, "uploading weights");
    M->rows_ready = false;
    return HB_OK;
}

extern "C" int64_t hb_mlp_workspace_bytes(int64_t n) {
    const int64_t chunks = (n + kMlpChunk - 1) / kMlpChunk;
    return (int64_t)sizeof(float) * (n * (4 * MLP_W + 2) + chunks * (MLP_NPARAM + 1) + 64);
}

extern "C" int hb_mlp_loss_grad(const float *params, const float *feats, const float *a, const float *b, int64_t n,
                                float *grads, float *loss, void *work, void *stream) {
    if (!params || !feats || !a || !b || !grads || !loss || !work || n <= 0) return HB_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float *H1 = (float *)work, *D1 = H1 + n * MLP_W, *H2 = D1 + n * MLP_W, *D2 = H2 + n * MLP_W;
    float *DO = D2 + n * MLP_W, *L = DO + n, *partial = L + n;
    mlp_fwd_bwd_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(params, feats, a, b, n, H1, D1, H2, D2, DO, L);
    const int chunks = (int)((n + kMlpChunk - 1) / kMlpChunk);
    mlp_grad_partial_kernel<<<chunks, 256, 0, s>>>(feats, H1, D1, H2, D2, DO, L, n, partial);
    mlp_grad_reduce_kernel<<<(MLP_NPARAM + 1 + 255) / 256, 256, 0, s>>>(partial, chunks, 1.0f / (float)n, grads, loss);
    return cudaGetLastError() == cudaSuccess ? HB_OK : HB_ERR_CUDA;
}

extern "C" int hb_mlp_adam(int64_t n_param, float *params, const float *grads, float *m, float *v, int32_t step,
                           float lr, void *stream) {
    if (!params || !grads || !m || !v || step < 1) return HB_ERR_INVALID_ARG;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    adam_kernel<<<(unsigned)((n_param + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n_param, params, grads, m, v, lr,
                                                                                      b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError() == cudaSuccess ? HB_OK : HB_ERR_CUDA;
}

// Adam training over a device data set: the samples are taken in consecutive
// windows of `batch` (wrapping around), one loss-and-gradient pass and one
// update per step, the loss of the last step in *last_loss (host).  Scratch
// (gradients, moments, workspace) is allocated and freed by the call.
// The Adam loop of both training entry points; the scratch comes from `mem`
// (a context's memory) or from cudaMalloc when mem is null.
static int mlp_train_loop(hb_ctx *mem, float *params, const float *feats, const float *a, const float *b, int64_t n,
                          int64_t batch, int32_t steps, float lr, float *last_loss, void *stream) {
    if (!params || !feats || !a || !b || n <= 0 || batch <= 0 || steps < 1 || !(lr > 0.0f))
        return HB_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t bs = batch < n ? batch : n;
    float *g = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
    void *work = nullptr;
    auto alloc = [&](void **p, size_t bytes) {
        return mem ? dmalloc(mem, p, bytes) : cudaMalloc(p, bytes);
    };
    cudaError_t e = alloc((void **)&g, sizeof(float) * MLP_NPARAM);
    if (e == cudaSuccess) e = alloc((void **)&m, sizeof(float) * MLP_NPARAM);
    if (e == cudaSuccess) e = alloc((void **)&v, sizeof(float) * MLP_NPARAM);
    if (e == cudaSuccess) e = alloc((void **)&loss, sizeof(float));
    if (e == cudaSuccess) e = alloc(&work, (size_t)hb_mlp_workspace_bytes(bs));
    if (e == cudaSuccess) e = cudaMemsetAsync(m, 0, sizeof(float) * MLP_NPARAM, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, sizeof(float) * MLP_NPARAM, s);
    int rc = e == cudaSuccess ? HB_OK : HB_ERR_OOM;
    int64_t off = 0;
    for (int32_t step = 1; step <= steps && rc == HB_OK; ++step) {
        const int64_t cnt = off + bs <= n ? bs : n - off;
        rc = hb_mlp_loss_grad(params, feats + off * MLP_IN, a + off, b + off, cnt, g, loss, work, stream);
        if (rc == HB_OK) rc = hb_mlp_adam(MLP_NPARAM, params, g, m, v, step, lr, stream);
        off += cnt;
        if (off >= n) off = 0;
    }
    if (rc == HB_OK && last_loss) {
        e = cudaMemcpyAsync(last_loss, loss, sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = HB_ERR_CUDA;
    }
    cudaStreamSynchronize(s);
    for (void *p : {(void *)g, (void *)m, (void *)v, (void *)loss, work}) {
        if (mem) dfree(mem, p);
        else if (p) cudaFree(p);
    }
    return rc;
}

extern "C" int hb_mlp_train_params(float *params, const float *feats, const float *a, const float *b, int64_t n,
                                   int64_t batch, int32_t steps, float lr, float *last_loss, void *stream) {
    return mlp_train_loop(nullptr, params, feats, a, b, n, batch, steps, lr, last_loss, stream);
}

extern "C" int hb_mlp_train(hb_ctx *ctx, const hb_mlp_dataset *d, float *params, hb_stats *st, void *stream) {
    if (!ctx || !d || !params) return mlp_fail(ctx, HB_ERR_INVALID_ARG, "NULL argument");
    float last = 0.0f;
    int rc = mlp_train_loop(ctx, params, d->feats, d->a, d->b, d->n, d->batch, d->steps, d->lr, &last, stream);
    if (rc != HB_OK) return mlp_fail(ctx, rc, "training failed (arguments, memory or launch)");
    // the trained network becomes the context's preconditioner network
    std::vector<float> p(MLP_NPARAM);
    if (cudaMemcpy(p.data(), params, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess)
        return mlp_fail(ctx, HB_ERR_CUDA, "reading the trained parameters");
    hb_mlp_weights w{MLP_IN, MLP_W, &p[OFF_W1], &p[OFF_B1], &p[OFF_W2], &p[OFF_B2], &p[OFF_W3], &p[OFF_B3]};
    rc = hb_mlp_set(ctx, &w);
    if (rc != HB_OK) return rc;
    if (st) {
        memset(st, 0, sizeof(*st));
        st->iterations = d->steps;
        st->mlp_loss = last;
    }
    return HB_OK;
}

extern "C" int hb_mlp_predict(const float *params, const float *feats, int64_t n, float *out, void *stream) {
    if (!params || !feats || !out || n <= 0) return HB_ERR_INVALID_ARG;
    mlp_predict_kernel<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(params, feats, n, out);
    return cudaGetLastError() == cudaSuccess ? HB_OK : HB_ERR_CUDA;
}

extern "C" int hb_diag_features(hb_ctx *ctx, const hb_blocks *H, const double *theta, int32_t q, float *feats,
                                void *stream) {
    if (!ctx || !H || !theta || q < 1 || !feats) return mlp_fail(ctx, HB_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_diag_work(ctx, H, std::max(q, 1), s);
    if (rc != HB_OK) return rc;
    DiagWork *w = (DiagWork *)ctx->diag;
    fill_diag(ctx, H, w, s);   // the diagonal of H from the blocks
    MlpState *M = (MlpState *)ctx->mlp;
    if (!M) { M = new MlpState(); ctx->mlp = M; }
    rc = ensure_rows(ctx, *M, w, s);
    if (rc != HB_OK) return rc;
    double *th = nullptr;
    if (dmalloc_n(ctx, &th, (size_t)q) != cudaSuccess) return HB_ERR_OOM;
    cudaMemcpyAsync(th, theta, sizeof(double) * q, cudaMemcpyHostToDevice, s);
    dim3 g((unsigned)((ctx->dim + 255) / 256), q);
    diag_features_kernel<<<g, 256, 0, s>>>(w->d, M->row_info, ctx->dim, th, q, feats);
    cudaStreamSynchronize(s);
    dfree(ctx, th);
    return cudaGetLastError() == cudaSuccess ? HB_OK : HB_ERR_CUDA;
}
