// Training and inference kernels of the learned cost model: a 3-layer FP32
// MLP, F features -> 64 -> 64 -> 1 with ReLU, trained with Adam on the mean
// squared error of the predicted log runtime.
//
// Parameter layout (floats): W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3.
//
// Training runs in ONE thread block: the model (5.3 k parameters) and its
// Adam moments stay in shared memory across the steps of a launch, each
// step's mini-batch activations and deltas too; gradients are reduced over
// the batch in a fixed order (no atomics), so training is deterministic.
#include <cuda_runtime.h>

#include "wt_mlp.hpp"

namespace wt {

namespace {

constexpr int F = kMlpFeatures;
constexpr int H = kMlpHidden;
constexpr int NP = kMlpParams;
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + H * F;
constexpr int OFF_W2 = OFF_B1 + H;
constexpr int OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H;
constexpr int OFF_B3 = OFF_W3 + H;
static_assert(OFF_B3 + 1 == NP, "parameter layout");
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads, 1)
mlp_train_kernel(float *__restrict__ params, float *__restrict__ mom1, float *__restrict__ mom2, int t0,
                 const float *__restrict__ X, const float *__restrict__ Y, const int *__restrict__ idx, int steps,
                 int B, float lr, float beta1, float beta2, float eps, float wd, float *__restrict__ loss) {
  extern __shared__ float sm[];
  float *P = sm;             // NP
  float *M = P + NP;         // NP
  float *V = M + NP;         // NP
  float *xb = V + NP;        // B * F
  float *yb = xb + B * F;    // B
  float *a1 = yb + B;        // B * H
  float *a2 = a1 + B * H;    // B * H
  float *d1 = a2 + B * H;    // B * H
  float *d2 = d1 + B * H;    // B * H
  float *gb = d2 + B * H;    // B (dLoss/dout)
  float *rb = gb + B;        // B (squared residuals)
  const int tid = threadIdx.x;
  for (int q = tid; q < NP; q += kThreads) {
    P[q] = params[q];
    M[q] = mom1[q];
    V[q] = mom2[q];
  }
  __syncthreads();
  for (int st = 0; st < steps; st++) {
    const int *bi = idx + (size_t)st * B;
    for (int i = tid; i < B * F; i += kThreads) xb[i] = X[(size_t)bi[i / F] * F + i % F];
    for (int b = tid; b < B; b += kThreads) yb[b] = Y[bi[b]];
    __syncthreads();
    // layer 1: a1 = relu(W1 x + b1)
    for (int i = tid; i < B * H; i += kThreads) {
      const int b = i / H, j = i % H;
      float z = P[OFF_B1 + j];
      for (int f = 0; f < F; f++) z = fmaf(P[OFF_W1 + j * F + f], xb[b * F + f], z);
      a1[i] = fmaxf(z, 0.f);
    }
    __syncthreads();
    // layer 2: a2 = relu(W2 a1 + b2)
    for (int i = tid; i < B * H; i += kThreads) {
      const int b = i / H, j = i % H;
      float z = P[OFF_B2 + j];
      for (int k = 0; k < H; k++) z = fmaf(P[OFF_W2 + j * H + k], a1[b * H + k], z);
      a2[i] = fmaxf(z, 0.f);
    }
    __syncthreads();
    // output and d(mean squared error)/d(output)
    for (int b = tid; b < B; b += kThreads) {
      float o = P[OFF_B3];
      for (int j = 0; j < H; j++) o = fmaf(P[OFF_W3 + j], a2[b * H + j], o);
      const float r = o - yb[b];
      gb[b] = 2.f * r / B;
      rb[b] = r * r;
    }
    __syncthreads();
    for (int i = tid; i < B * H; i += kThreads) {
      const int b = i / H, j = i % H;
      d2[i] = a2[i] > 0.f ? gb[b] * P[OFF_W3 + j] : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < B * H; i += kThreads) {
      const int b = i / H, k = i % H;
      float s = 0.f;
      for (int j = 0; j < H; j++) s = fmaf(P[OFF_W2 + j * H + k], d2[b * H + j], s);
      d1[i] = a1[i] > 0.f ? s : 0.f;
    }
    if (tid == 0) {
      float l = 0.f;
      for (int b = 0; b < B; b++) l += rb[b];
      loss[st] = l / B;
    }
    __syncthreads();
    // gradients (batch sums in sample order) and the Adam update
    const int t = t0 + st + 1;
    const float c1 = 1.f / (1.f - powf(beta1, (float)t));
    const float c2 = 1.f / (1.f - powf(beta2, (float)t));
    for (int q = tid; q < NP; q += kThreads) {
      float g = 0.f;
      bool weight = true;
      if (q < OFF_B1) {
        const int j = q / F, f = q % F;
        for (int b = 0; b < B; b++) g = fmaf(d1[b * H + j], xb[b * F + f], g);
      } else if (q < OFF_W2) {
        const int j = q - OFF_B1;
        for (int b = 0; b < B; b++) g += d1[b * H + j];
        weight = false;
      } else if (q < OFF_B2) {
        const int j = (q - OFF_W2) / H, k = (q - OFF_W2) % H;
        for (int b = 0; b < B; b++) g = fmaf(d2[b * H + j], a1[b * H + k], g);
      } else if (q < OFF_W3) {
        const int j = q - OFF_B2;
        for (int b = 0; b < B; b++) g += d2[b * H + j];
        weight = false;
      } else if (q < OFF_B3) {
        const int j = q - OFF_W3;
        for (int b = 0; b < B; b++) g = fmaf(gb[b], a2[b * H + j], g);
      } else {
        for (int b = 0; b < B; b++) g += gb[b];
        weight = false;
      }
      if (weight) g = fmaf(wd, P[q], g);
      const float m = beta1 * M[q] + (1.f - beta1) * g;
      const float v = beta2 * V[q] + (1.f - beta2) * g * g;
      M[q] = m;
      V[q] = v;
      P[q] -= lr * (m * c1) / (sqrtf(v * c2) + eps);
    }
    __syncthreads();
  }
  for (int q = tid; q < NP; q += kThreads) {
    params[q] = P[q];
    mom1[q] = M[q];
    mom2[q] = V[q];
  }
}

// One sample per thread; the parameters in shared memory.
__global__ void __launch_bounds__(128)
mlp_forward_kernel(const float *__restrict__ params, const float *__restrict__ X, int n, float *__restrict__ Y) {
  __shared__ float P[NP];
  for (int q = threadIdx.x; q < NP; q += blockDim.x) P[q] = params[q];
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float x[F], h1[H];
  for (int f = 0; f < F; f++) x[f] = X[(size_t)s * F + f];
  for (int j = 0; j < H; j++) {
    float z = P[OFF_B1 + j];
    for (int f = 0; f < F; f++) z = fmaf(P[OFF_W1 + j * F + f], x[f], z);
    h1[j] = fmaxf(z, 0.f);
  }
  float o = P[OFF_B3];
  for (int j = 0; j < H; j++) {
    float z = P[OFF_B2 + j];
    for (int k = 0; k < H; k++) z = fmaf(P[OFF_W2 + j * H + k], h1[k], z);
    o = fmaf(P[OFF_W3 + j], fmaxf(z, 0.f), o);
  }
  Y[s] = o;
}

}  // namespace

size_t mlp_train_smem(int batch) {
  return sizeof(float) * ((size_t)3 * NP + (size_t)batch * F + 3 * (size_t)batch + 4 * (size_t)batch * H);
}

cudaError_t mlp_train_launch(float *params, float *m, float *v, int t0, const float *X, const float *Y,
                             const int *idx, int steps, int batch, float lr, float beta1, float beta2, float eps,
                             float wd, float *loss, cudaStream_t stream) {
  const size_t smem = mlp_train_smem(batch);
  cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  mlp_train_kernel<<<1, kThreads, smem, stream>>>(params, m, v, t0, X, Y, idx, steps, batch, lr, beta1, beta2, eps,
                                                  wd, loss);
  return cudaGetLastError();
}

cudaError_t mlp_forward_launch(const float *params, const float *X, int n, float *Y, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  mlp_forward_kernel<<<(n + 127) / 128, 128, 0, stream>>>(params, X, n, Y);
  return cudaGetLastError();
}

}  // namespace wt
