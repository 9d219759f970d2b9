// Moduli-selection network: forward, backward (gradients of the mean binary
// cross-entropy) and Adam update, as plain CUDA kernels.  The paper picks the
// moduli count from measured accuracy bands (Section IV-A); this network is an
// addition that estimates, from features of the inputs and the requested
// accuracy, the probability that each N = 4..24 meets that accuracy.
//
// Network: x(39) -> relu(W1 x + b1)(64) -> relu(W2 h1 + b2)(64) -> W3 h2 + b3 (21 logits)
// Parameters are one float vector: W1 (64x39, row major), b1, W2 (64x64), b2, W3 (21x64), b3.
// One block of 64 threads handles one sample: thread j owns hidden unit j.
#include <cmath>

#include "emu_internal.h"

namespace emu {
namespace {

constexpr int NI = kMlpIn, NH = kMlpHidden, NO = kMlpOut;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH, NPARAM = OFF_B3 + NO;
static_assert(NPARAM == kMlpParams, "parameter count");

struct Act {
  float x[NI];
  float a1[NH], h1[NH], a2[NH], h2[NH], z[NO];
};

__device__ __forceinline__ void forward_sample(const float* __restrict__ th, const float* __restrict__ xin, Act& s) {
  const int j = threadIdx.x;
  for (int i = j; i < NI; i += NH) s.x[i] = xin[i];
  __syncthreads();
  float a = th[OFF_B1 + j];
  for (int i = 0; i < NI; ++i) a = fmaf(th[OFF_W1 + j * NI + i], s.x[i], a);
  s.a1[j] = a;
  s.h1[j] = fmaxf(a, 0.0f);
  __syncthreads();
  a = th[OFF_B2 + j];
  for (int i = 0; i < NH; ++i) a = fmaf(th[OFF_W2 + j * NH + i], s.h1[i], a);
  s.a2[j] = a;
  s.h2[j] = fmaxf(a, 0.0f);
  __syncthreads();
  if (j < NO) {
    a = th[OFF_B3 + j];
    for (int i = 0; i < NH; ++i) a = fmaf(th[OFF_W3 + j * NH + i], s.h2[i], a);
    s.z[j] = a;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NH) mlp_forward_kernel(const float* __restrict__ th, const float* __restrict__ X,
                                                         int batch, float* __restrict__ Z) {
  __shared__ Act s;
  const int b = blockIdx.x;
  if (b >= batch) return;
  forward_sample(th, X + static_cast<int64_t>(b) * NI, s);
  if (threadIdx.x < NO) Z[static_cast<int64_t>(b) * NO + threadIdx.x] = s.z[threadIdx.x];
}

// Gradient of (1/batch) sum_b sum_t BCE(sigmoid(z_bt), y_bt), accumulated with atomics.
__global__ void __launch_bounds__(NH) mlp_backward_kernel(const float* __restrict__ th, const float* __restrict__ X,
                                                          const float* __restrict__ Y, int batch,
                                                          float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ Act s;
  __shared__ float dz[NO], da2[NH], da1[NH];
  const int b = blockIdx.x;
  if (b >= batch) return;
  const int j = threadIdx.x;
  forward_sample(th, X + static_cast<int64_t>(b) * NI, s);
  const float inv_b = 1.0f / static_cast<float>(batch);
  if (j < NO) {
    const float z = s.z[j], y = Y[static_cast<int64_t>(b) * NO + j];
    dz[j] = (1.0f / (1.0f + expf(-z)) - y) * inv_b;
    const float l = fmaxf(z, 0.0f) - z * y + log1pf(expf(-fabsf(z)));
    atomicAdd(loss, l * inv_b);
  }
  __syncthreads();
  // layer 3
  if (j < NO) {
    for (int i = 0; i < NH; ++i) atomicAdd(&grad[OFF_W3 + j * NH + i], dz[j] * s.h2[i]);
    atomicAdd(&grad[OFF_B3 + j], dz[j]);
  }
  {
    float d = 0.0f;
    for (int t = 0; t < NO; ++t) d = fmaf(th[OFF_W3 + t * NH + j], dz[t], d);
    da2[j] = s.a2[j] > 0.0f ? d : 0.0f;
  }
  __syncthreads();
  // layer 2
  for (int i = 0; i < NH; ++i) atomicAdd(&grad[OFF_W2 + j * NH + i], da2[j] * s.h1[i]);
  atomicAdd(&grad[OFF_B2 + j], da2[j]);
  {
    float d = 0.0f;
    for (int t = 0; t < NH; ++t) d = fmaf(th[OFF_W2 + t * NH + j], da2[t], d);
    da1[j] = s.a1[j] > 0.0f ? d : 0.0f;
  }
  __syncthreads();
  // layer 1
  for (int i = 0; i < NI; ++i) atomicAdd(&grad[OFF_W1 + j * NI + i], da1[j] * s.x[i]);
  atomicAdd(&grad[OFF_B1 + j], da1[j]);
}

__global__ void mlp_adam_kernel(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, int n, float lr, float b1, float b2, float c1, float c2,
                                float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Inference for one feature vector: the smallest N such that every N' >= N
// has probability >= threshold (-1 when none), written to *out.
__global__ void __launch_bounds__(NH) mlp_choose_kernel(const float* __restrict__ th, const float* __restrict__ x,
                                                        float threshold, int* __restrict__ out) {
  __shared__ Act s;
  forward_sample(th, x, s);
  if (threadIdx.x == 0) {
    int best = -1;
    for (int t = NO - 1; t >= 0; --t) {
      const float p = 1.0f / (1.0f + expf(-s.z[t]));
      if (!(p >= threshold)) break;
      best = kMlpNmin + t;
    }
    *out = best;
  }
}

}  // namespace

cudaError_t launch_mlp_forward(const float* th, const float* X, int batch, float* Z, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  mlp_forward_kernel<<<batch, NH, 0, st>>>(th, X, batch, Z);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const float* th, const float* X, const float* Y, int batch, float* grad, float* loss,
                                cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * NPARAM, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
  if (e != cudaSuccess || batch <= 0) return e;
  mlp_backward_kernel<<<batch, NH, 0, st>>>(th, X, Y, batch, grad, loss);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* th, const float* g, float* m, float* v, int step, float lr, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = static_cast<float>(1.0 - std::pow(0.9, step));
  const float c2 = static_cast<float>(1.0 - std::pow(0.999, step));
  mlp_adam_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(th, g, m, v, NPARAM, lr, b1, b2, c1, c2, eps);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mlp_choose(const float* th, const float* x, float threshold, int* out, cudaStream_t st) {
  mlp_choose_kernel<<<1, NH, 0, st>>>(th, x, threshold, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace emu
