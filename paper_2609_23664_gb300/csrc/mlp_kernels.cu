// Learned cost model kernels: MLP 12 -> 64 -> 64 -> 1 (ReLU), BF16 weights
// and activations, FP32 accumulation (sm_103a).
//
// The model stands in for the analytic materialize-versus-recompute costs of
// Eq. 2 (Sec. IV-C); the planner's analytic gate-count proxy (Sec. VI-D,
// Fig. 3) remains the fallback.  Forward pass, with bf(.) = round to BF16
// (nearest even):
//   xb = bf(x); a1 = bf(W1) xb + bf(b1); h1 = bf(relu(a1))
//   a2 = bf(W2) h1 + bf(b2); h2 = bf(relu(a2)); y = bf(w3) . h2 + bf(b3)
// Sums run in FP32 in ascending index order.  The backward pass treats the
// roundings as identities (straight-through) and returns gradients of
// mean (y - t)^2 with respect to the FP32 master parameters.  Per-CTA
// gradient partials are reduced in CTA order, so results are deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "qw_internal.h"

namespace qw {

constexpr int MI = QW_MLP_IN, MH = QW_MLP_HID;
constexpr int OFF_W1 = 0, OFF_B1 = MI * MH, OFF_W2 = OFF_B1 + MH, OFF_B2 = OFF_W2 + MH * MH,
              OFF_W3 = OFF_B2 + MH, OFF_B3 = OFF_W3 + MH, N_PARAMS = OFF_B3 + 1;
static_assert(N_PARAMS == QW_MLP_PARAMS, "parameter layout");
constexpr int MLP_SPB = 32;  // samples per CTA

__device__ __forceinline__ float bf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// 64 threads: thread i owns hidden unit i of both layers
template <bool BACKWARD>
__global__ void __launch_bounds__(MH)
mlp_kernel(const float *__restrict__ P, const float *__restrict__ X, const float *__restrict__ Tg,
           float *__restrict__ Y, uint32_t batch, float *__restrict__ partial) {
  __shared__ float sW2[MH][MH + 1];  // bf(W2), padded
  __shared__ float sx[MI], sh1[MH], sh2[MH], sda2[MH];
  __shared__ float sred[2];
  const int i = threadIdx.x;
  float w1[MI], w2[MH];
#pragma unroll
  for (int j = 0; j < MI; j++) w1[j] = bf(P[OFF_W1 + i * MI + j]);
#pragma unroll
  for (int j = 0; j < MH; j++) {
    w2[j] = bf(P[OFF_W2 + i * MH + j]);
    sW2[i][j] = w2[j];
  }
  const float b1 = bf(P[OFF_B1 + i]), b2 = bf(P[OFF_B2 + i]), w3 = bf(P[OFF_W3 + i]);
  const float b3 = bf(P[OFF_B3]);
  float gW1[MI], gW2[MH], gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f, loss = 0.f;
  if (BACKWARD) {
#pragma unroll
    for (int j = 0; j < MI; j++) gW1[j] = 0.f;
#pragma unroll
    for (int j = 0; j < MH; j++) gW2[j] = 0.f;
  }
  __syncthreads();
  const uint32_t s0 = blockIdx.x * MLP_SPB;
  for (uint32_t s = s0; s < s0 + MLP_SPB && s < batch; s++) {
    if (i < MI) sx[i] = bf(X[(size_t)s * MI + i]);
    __syncthreads();
    float a1 = 0.f;
#pragma unroll
    for (int j = 0; j < MI; j++) a1 = fmaf(w1[j], sx[j], a1);
    a1 += b1;
    sh1[i] = bf(fmaxf(a1, 0.f));
    __syncthreads();
    float a2 = 0.f;
#pragma unroll
    for (int j = 0; j < MH; j++) a2 = fmaf(w2[j], sh1[j], a2);
    a2 += b2;
    sh2[i] = bf(fmaxf(a2, 0.f));
    __syncthreads();
    if (i == 0) {
      float y = 0.f;
      for (int j = 0; j < MH; j++) y = fmaf(bf(P[OFF_W3 + j]), sh2[j], y);
      y += b3;
      sred[0] = y;
      if (Y) Y[s] = y;
    }
    __syncthreads();
    if (BACKWARD) {
      const float y = sred[0], d = y - Tg[s];
      if (i == 0) loss += d * d;
      const float dy = 2.f * d / (float)batch;
      gw3 = fmaf(dy, sh2[i], gw3);
      if (i == 0) gb3 += dy;
      const float da2 = (a2 > 0.f) ? dy * w3 : 0.f;
      sda2[i] = da2;
      gb2 += da2;
#pragma unroll
      for (int j = 0; j < MH; j++) gW2[j] = fmaf(da2, sh1[j], gW2[j]);
      __syncthreads();
      float dh1 = 0.f;
      for (int r = 0; r < MH; r++) dh1 = fmaf(sW2[r][i], sda2[r], dh1);
      const float da1 = (a1 > 0.f) ? dh1 : 0.f;
      gb1 += da1;
#pragma unroll
      for (int j = 0; j < MI; j++) gW1[j] = fmaf(da1, sx[j], gW1[j]);
    }
    __syncthreads();
  }
  if (BACKWARD) {
    float *o = partial + (size_t)blockIdx.x * (N_PARAMS + 1);
#pragma unroll
    for (int j = 0; j < MI; j++) o[OFF_W1 + i * MI + j] = gW1[j];
    o[OFF_B1 + i] = gb1;
#pragma unroll
    for (int j = 0; j < MH; j++) o[OFF_W2 + i * MH + j] = gW2[j];
    o[OFF_B2 + i] = gb2;
    o[OFF_W3 + i] = gw3;
    if (i == 0) {
      o[OFF_B3] = gb3;
      o[N_PARAMS] = loss;
    }
  }
}

// grad[p] = sum over CTAs (in order) of partial[c][p]; loss likewise / batch
__global__ void mlp_reduce_kernel(const float *__restrict__ partial, uint32_t n_cta, uint32_t batch,
                                  float *grad, float *loss) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > (uint32_t)N_PARAMS) return;
  float s = 0.f;
  for (uint32_t c = 0; c < n_cta; c++) s += partial[(size_t)c * (N_PARAMS + 1) + p];
  if (p < (uint32_t)N_PARAMS) grad[p] = s;
  else if (loss) *loss = s / (float)batch;
}

__global__ void mlp_adam_kernel(float *p, const float *g, float *m, float *v, uint32_t n, float lr,
                                float b1, float b2, float eps, float c1, float c2) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

size_t mlp_scratch_floats(uint32_t batch) {
  const uint32_t n_cta = (batch + MLP_SPB - 1) / MLP_SPB;
  return (size_t)n_cta * (N_PARAMS + 1);
}

void launch_mlp_forward(const float *params, const float *x, float *y, uint32_t batch, void *stream) {
  if (batch == 0) return;
  const uint32_t n_cta = (batch + MLP_SPB - 1) / MLP_SPB;
  mlp_kernel<false><<<n_cta, MH, 0, (cudaStream_t)stream>>>(params, x, nullptr, y, batch, nullptr);
}

void launch_mlp_loss_grad(const float *params, const float *x, const float *target, uint32_t batch,
                          float *loss, float *grad, float *scratch, void *stream) {
  if (batch == 0) return;
  const uint32_t n_cta = (batch + MLP_SPB - 1) / MLP_SPB;
  cudaStream_t s = (cudaStream_t)stream;
  mlp_kernel<true><<<n_cta, MH, 0, s>>>(params, x, target, nullptr, batch, scratch);
  mlp_reduce_kernel<<<(N_PARAMS + 1 + 255) / 256, 256, 0, s>>>(scratch, n_cta, batch, grad, loss);
}

void launch_mlp_adam(float *params, const float *grad, float *m, float *v, uint32_t n, uint32_t t,
                     float lr, float b1, float b2, float eps, void *stream) {
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  mlp_adam_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, n, lr, b1,
                                                                     b2, eps, c1, c2);
}

}  // namespace qw
