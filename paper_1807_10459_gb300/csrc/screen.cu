// screen.cu -- kernels of the learned screen (a small perceptron predicting a
// candidate's largest surrogate estimate; no counterpart in the paper).
//
// Network F -> H -> H -> 1 with ReLU; flat parameters W1[H][F], b1[H],
// W2[H][H], b2[H], w3[H], b3 (fp32 master values).  Every pass reads the
// weights through a bfloat16 copy (round to nearest even) and accumulates in
// fp32; biases stay fp32.  All reductions run in a fixed order, so training is
// deterministic.  The layers are small (H = 64), so plain CUDA-core FMA
// kernels are used: a batch of 256 rows is 4 MFLOP per layer.
#include <cuda_bf16.h>

#include "idtx.h"
#include "ksg_common.cuh"

namespace idtx {

namespace {

constexpr int F = IDTX_SCREEN_F;
constexpr int H = IDTX_SCREEN_H;
constexpr int P = IDTX_SCREEN_NPARAMS;
constexpr int OFF_W1 = 0, OFF_B1 = H * F, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H;

int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

__global__ void k_round_bf16(const float *p, __nv_bfloat16 *w, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = __float2bfloat16_rn(p[i]);
}

// xn[b][i] = (feats[row(b)][i] - mean[i]) * scale[i], row(b) = order[start+b] or start+b.
__global__ void k_gather_norm(const float *feats, const int32_t *order, int64_t start, int B,
                              const float *mean, const float *scale, float *xn)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * F) return;
    const int b = idx / F, i = idx - b * F;
    const int64_t r = order ? (int64_t)order[start + b] : start + b;
    xn[idx] = (feats[r * F + i] - mean[i]) * scale[i];
}

// z[b][n] = bias[n] + sum_k W[n][k] in[b][k]; a = relu(z) (or z).
__global__ void k_dense_fwd(const float *in, const __nv_bfloat16 *W, const float *bias, float *z,
                            float *a, int B, int K, int N, int relu)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * N) return;
    const int b = idx / N, n = idx - b * N;
    float acc = bias[n];
    for (int k = 0; k < K; ++k) acc = fmaf(__bfloat162float(W[n * K + k]), in[b * K + k], acc);
    if (z) z[idx] = acc;
    a[idx] = relu ? fmaxf(acc, 0.0f) : acc;
}

// Squared error (quantile == 0): dy[b] = scale * (y - t), loss_acc += sum (y - t)^2.
// Pinball loss of quantile q: dy[b] = scale * ([t < y] - q), loss_acc += sum
// (t - y)(q - [t < y]).  One block, fixed order.
__global__ void k_loss(const float *y, const float *targets, const int32_t *order, int64_t start,
                       int B, float scale, float quantile, float *dy, double *loss_acc)
{
    __shared__ double s_part[256];
    double part = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const int64_t r = order ? (int64_t)order[start + b] : start + b;
        const float d = y[b] - targets[r];
        if (quantile > 0.0f) {
            const float below = d > 0.0f ? 1.0f : 0.0f;  // [t < y]
            if (dy) dy[b] = scale * (below - quantile);
            part += (double)(-d) * ((double)quantile - (double)below);
        } else {
            if (dy) dy[b] = scale * d;
            part += (double)d * (double)d;
        }
    }
    s_part[threadIdx.x] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int t = 0; t < (int)blockDim.x; ++t) sum += s_part[t];
        *loss_acc += sum;
    }
}

// dx[b][k] = (sum_n W[n][k] dz[b][n]) * [zin[b][k] > 0].
__global__ void k_dense_bwd_x(const float *dz, const __nv_bfloat16 *W, const float *zin,
                              float *dx, int B, int K, int N)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * K) return;
    const int b = idx / K, k = idx - b * K;
    float acc = 0.0f;
    for (int n = 0; n < N; ++n) acc = fmaf(__bfloat162float(W[n * K + k]), dz[b * N + n], acc);
    dx[idx] = zin[idx] > 0.0f ? acc : 0.0f;
}

// gW[n][k] (+)= sum_b dz[b][n] in[b][k];  gb[n] (+)= sum_b dz[b][n]  (k == K).
__global__ void k_dense_bwd_w(const float *dz, const float *in, float *gW, float *gb, int B,
                              int K, int N, int accumulate)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * (K + 1)) return;
    const int n = idx / (K + 1), k = idx - n * (K + 1);
    float acc = 0.0f;
    if (k < K) {
        for (int b = 0; b < B; ++b) acc = fmaf(dz[b * N + n], in[b * K + k], acc);
        gW[n * K + k] = accumulate ? gW[n * K + k] + acc : acc;
    } else {
        for (int b = 0; b < B; ++b) acc += dz[b * N + n];
        gb[n] = accumulate ? gb[n] + acc : acc;
    }
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, int n, float lr, float c1,
                       float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

}  // namespace

size_t mlp_work_floats(int B) { return (size_t)B * (F + 4 * H + 2 * H + 2) + 2 * (size_t)P; }

void mlp_work_carve(float *base, int B, MlpWork *w)
{
    float *q = base;
    w->xn = q, q += (size_t)B * F;
    w->z1 = q, q += (size_t)B * H;
    w->a1 = q, q += (size_t)B * H;
    w->z2 = q, q += (size_t)B * H;
    w->a2 = q, q += (size_t)B * H;
    w->d2 = q, q += (size_t)B * H;
    w->d1 = q, q += (size_t)B * H;
    w->y = q, q += B;
    w->dy = q, q += B;
    w->grad = q, q += P;
    w->wbf = reinterpret_cast<__nv_bfloat16 *>(q);
}

cudaError_t mlp_round(const float *params, MlpWork &w, cudaStream_t st)
{
    k_round_bf16<<<blocks_for(P, 256), 256, 0, st>>>(params, w.wbf, P);
    return cudaGetLastError();
}

cudaError_t mlp_forward(const float *params, MlpWork &w, const float *feats,
                        const int32_t *order, int64_t start, int B, const float *mean,
                        const float *scale, cudaStream_t st)
{
    k_gather_norm<<<blocks_for((int64_t)B * F, 256), 256, 0, st>>>(feats, order, start, B, mean,
                                                                   scale, w.xn);
    k_dense_fwd<<<blocks_for((int64_t)B * H, 256), 256, 0, st>>>(
        w.xn, w.wbf + OFF_W1, params + OFF_B1, w.z1, w.a1, B, F, H, 1);
    k_dense_fwd<<<blocks_for((int64_t)B * H, 256), 256, 0, st>>>(
        w.a1, w.wbf + OFF_W2, params + OFF_B2, w.z2, w.a2, B, H, H, 1);
    k_dense_fwd<<<blocks_for(B, 256), 256, 0, st>>>(w.a2, w.wbf + OFF_W3, params + OFF_B3,
                                                    nullptr, w.y, B, H, 1, 0);
    return cudaGetLastError();
}

cudaError_t mlp_loss(MlpWork &w, const float *targets, const int32_t *order, int64_t start, int B,
                     float dy_scale, float quantile, bool want_dy, double *loss_acc,
                     cudaStream_t st)
{
    k_loss<<<1, 256, 0, st>>>(w.y, targets, order, start, B, dy_scale, quantile,
                              want_dy ? w.dy : nullptr, loss_acc);
    return cudaGetLastError();
}

cudaError_t mlp_backward(MlpWork &w, int B, bool accumulate, cudaStream_t st)
{
    const int acc = accumulate ? 1 : 0;
    // output layer: dz = dy [B][1], input a2
    k_dense_bwd_w<<<blocks_for(1 * (H + 1), 128), 128, 0, st>>>(
        w.dy, w.a2, w.grad + OFF_W3, w.grad + OFF_B3, B, H, 1, acc);
    k_dense_bwd_x<<<blocks_for((int64_t)B * H, 256), 256, 0, st>>>(w.dy, w.wbf + OFF_W3, w.z2,
                                                                   w.d2, B, H, 1);
    // hidden layer 2: dz = d2, input a1
    k_dense_bwd_w<<<blocks_for((int64_t)H * (H + 1), 128), 128, 0, st>>>(
        w.d2, w.a1, w.grad + OFF_W2, w.grad + OFF_B2, B, H, H, acc);
    k_dense_bwd_x<<<blocks_for((int64_t)B * H, 256), 256, 0, st>>>(w.d2, w.wbf + OFF_W2, w.z1,
                                                                   w.d1, B, H, H);
    // hidden layer 1: dz = d1, input xn
    k_dense_bwd_w<<<blocks_for((int64_t)H * (F + 1), 128), 128, 0, st>>>(
        w.d1, w.xn, w.grad + OFF_W1, w.grad + OFF_B1, B, F, H, acc);
    return cudaGetLastError();
}

cudaError_t mlp_adam(float *params, const float *grad, float *m, float *v, int step, float lr,
                     cudaStream_t st)
{
    const float c1 = 1.0f - powf(0.9f, (float)step), c2 = 1.0f - powf(0.999f, (float)step);
    k_adam<<<blocks_for(P, 256), 256, 0, st>>>(params, grad, m, v, P, lr, c1, c2);
    return cudaGetLastError();
}

}  // namespace idtx
