// K5: the learned job-cost model.  A 12 -> 64 -> 64 -> 1 ReLU network
// predicts log(job time) from features of the job; jobs are then queued by
// non-increasing prediction (an LPT order on predicted times, Section 2.4).
// Forward, backward and Adam are plain FP32 kernels:
//   H1 = relu(X W1^T + b1), H2 = relu(H1 W2^T + b2), P = H2 w3 + b3,
//   L = mean (P - y)^2,
//   D3 = 2 (P - y) / N, D2 = (D3 w3^T) o [H2 > 0], D1 = (D2 W2) o [H1 > 0],
//   gW2 = D2^T H1, gW1 = D1^T X, gw3 = H2^T D3, gb = column sums.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "internal.h"

namespace {

constexpr int F = PERM_MLP_FEATURES;
constexpr int H = PERM_MLP_HIDDEN;
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + H * F;
constexpr int OFF_W2 = OFF_B1 + H;
constexpr int OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H;
constexpr int OFF_B3 = OFF_W3 + H;
static_assert(OFF_B3 + 1 == PERM_MLP_PARAMS, "parameter layout");

// Features of a job: order, density, row-count histogram, KKLLL estimate,
// Ryser work of the job as a leaf.
__global__ void k_features(JobArrays jobs, int64_t njobs, const uint64_t* __restrict__ arena,
                           const float* __restrict__ log_ap, float* __restrict__ feats) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= njobs) return;
  const int m = jobs.m[j];
  const int nnz = jobs.nnz[j];
  CsrView v = csr_view(arena, jobs.off[j], m, nnz);
  float hist[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int r = 0; r < m; ++r) {
    const int k = v.rowptr[r + 1] - v.rowptr[r];
    const int b = k <= 4 ? (k < 1 ? 0 : k - 1) : (k <= 6 ? 4 : (k <= 9 ? 5 : (k <= 14 ? 6 : 7)));
    hist[b] += 1.0f;
  }
  float* f = feats + j * F;
  const float inv = m > 0 ? 1.0f / (float)m : 0.0f;
  f[0] = (float)m / 64.0f;
  f[1] = m > 0 ? (float)nnz * inv * inv : 0.0f;
  for (int b = 0; b < 8; ++b) f[2 + b] = hist[b] * inv;
  const float la = log_ap ? log_ap[j] : 0.0f;
  f[10] = isfinite(la) ? la / 64.0f : -1.0f;
  f[11] = m > 0 ? (log2f((float)m) + (float)(m - 1)) / 64.0f : 0.0f;
}

// forward for one sample per thread; weights staged in shared memory
__global__ void k_mlp_forward(const float* __restrict__ P, const float* __restrict__ X, int32_t n,
                              float* __restrict__ H1, float* __restrict__ H2, float* __restrict__ pred) {
  __shared__ float w[PERM_MLP_PARAMS];
  for (int k = threadIdx.x; k < PERM_MLP_PARAMS; k += blockDim.x) w[k] = P[k];
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x[F];
  for (int k = 0; k < F; ++k) x[k] = X[i * F + k];
  float h1[H];
  for (int a = 0; a < H; ++a) {
    float s = w[OFF_B1 + a];
#pragma unroll
    for (int k = 0; k < F; ++k) s = fmaf(w[OFF_W1 + a * F + k], x[k], s);
    h1[a] = s > 0.f ? s : 0.f;
    if (H1) H1[i * H + a] = h1[a];
  }
  float out = w[OFF_B3];
  for (int a = 0; a < H; ++a) {
    float s = w[OFF_B2 + a];
#pragma unroll 16
    for (int b = 0; b < H; ++b) s = fmaf(w[OFF_W2 + a * H + b], h1[b], s);
    s = s > 0.f ? s : 0.f;
    if (H2) H2[i * H + a] = s;
    out = fmaf(w[OFF_W3 + a], s, out);
  }
  pred[i] = out;
}

// per-sample deltas D2, D1 and the loss terms
__global__ void k_mlp_deltas(const float* __restrict__ P, const float* __restrict__ H1, const float* __restrict__ H2,
                             const float* __restrict__ pred, const float* __restrict__ y, int32_t n,
                             float* __restrict__ D3, float* __restrict__ D2, float* __restrict__ D1,
                             float* __restrict__ loss) {
  __shared__ float w2[H * H];
  __shared__ float w3[H];
  for (int k = threadIdx.x; k < H * H; k += blockDim.x) w2[k] = P[OFF_W2 + k];
  for (int k = threadIdx.x; k < H; k += blockDim.x) w3[k] = P[OFF_W3 + k];
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < n) {
    const float e = pred[i] - y[i];
    l = e * e / (float)n;
    const float d3 = 2.0f * e / (float)n;
    D3[i] = d3;
    float d2[H];
    for (int a = 0; a < H; ++a) {
      d2[a] = H2[i * H + a] > 0.f ? d3 * w3[a] : 0.f;
      D2[i * H + a] = d2[a];
    }
    for (int b = 0; b < H; ++b) {
      float s = 0.f;
#pragma unroll 16
      for (int a = 0; a < H; ++a) s = fmaf(w2[a * H + b], d2[a], s);
      D1[i * H + b] = H1[i * H + b] > 0.f ? s : 0.f;
    }
  }
  // block sum of the loss
  for (int d = 16; d > 0; d >>= 1) l += __shfl_xor_sync(0xffffffffu, l, d);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

// gradient of one parameter per thread, summed over a slice of samples:
// grad[p] = sum_i U[i][a] * V[i][b] for the parameter's (a, b)
__global__ void k_mlp_grads(const float* __restrict__ X, const float* __restrict__ H1, const float* __restrict__ H2,
                            const float* __restrict__ D3, const float* __restrict__ D2,
                            const float* __restrict__ D1, int32_t n, int32_t slice, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= PERM_MLP_PARAMS) return;
  const int64_t i0 = (int64_t)blockIdx.y * slice;
  int64_t i1 = i0 + slice;
  if (i1 > n) i1 = n;
  float s = 0.f;
  if (p < OFF_B1) {
    const int a = p / F, k = p % F;
    for (int64_t i = i0; i < i1; ++i) s = fmaf(D1[i * H + a], X[i * F + k], s);
  } else if (p < OFF_W2) {
    const int a = p - OFF_B1;
    for (int64_t i = i0; i < i1; ++i) s += D1[i * H + a];
  } else if (p < OFF_B2) {
    const int a = (p - OFF_W2) / H, b = (p - OFF_W2) % H;
    for (int64_t i = i0; i < i1; ++i) s = fmaf(D2[i * H + a], H1[i * H + b], s);
  } else if (p < OFF_W3) {
    const int a = p - OFF_B2;
    for (int64_t i = i0; i < i1; ++i) s += D2[i * H + a];
  } else if (p < OFF_B3) {
    const int a = p - OFF_W3;
    for (int64_t i = i0; i < i1; ++i) s = fmaf(D3[i], H2[i * H + a], s);
  } else {
    for (int64_t i = i0; i < i1; ++i) s += D3[i];
  }
  atomicAdd(grad + p, s);
}

__global__ void k_adam(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, int32_t step, float lr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= PERM_MLP_PARAMS) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float gi = g[p];
  const float a = b1 * m1[p] + (1.f - b1) * gi;
  const float b = b2 * m2[p] + (1.f - b2) * gi * gi;
  m1[p] = a;
  m2[p] = b;
  const float ah = a / (1.f - powf(b1, (float)step));
  const float bh = b / (1.f - powf(b2, (float)step));
  P[p] -= lr * ah / (sqrtf(bh) + eps);
}

}  // namespace

cudaError_t launch_features(const JobArrays& jobs, int64_t njobs, const uint64_t* arena, const float* log_ap,
                            float* feats, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  k_features<<<(unsigned)((njobs + 255) / 256), 256, 0, s>>>(jobs, njobs, arena, log_ap, feats);
  return cudaGetLastError();
}

// scratch layout (floats): H1[n*H], H2[n*H], D3[n], D2[n*H], D1[n*H], pred[n]
cudaError_t mlp_forward_backward(const float* params, const float* feats, const float* target, int32_t count,
                                 float* scratch, float* grad, float* loss, cudaStream_t s) {
  if (count <= 0) return cudaErrorInvalidValue;
  float* H1 = scratch;
  float* H2 = H1 + (size_t)count * H;
  float* D3 = H2 + (size_t)count * H;
  float* D2 = D3 + count;
  float* D1 = D2 + (size_t)count * H;
  float* pred = D1 + (size_t)count * H;
  const int tb = 128;
  const unsigned nb = (unsigned)((count + tb - 1) / tb);
  k_mlp_forward<<<nb, tb, 0, s>>>(params, feats, count, H1, H2, pred);
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(grad, 0, sizeof(float) * PERM_MLP_PARAMS, s);
  if (e != cudaSuccess) return e;
  k_mlp_deltas<<<nb, tb, 0, s>>>(params, H1, H2, pred, target, count, D3, D2, D1, loss);
  const int32_t slice = 2048;
  dim3 g((PERM_MLP_PARAMS + 255) / 256, (unsigned)((count + slice - 1) / slice));
  k_mlp_grads<<<g, 256, 0, s>>>(feats, H1, H2, D3, D2, D1, count, slice, grad);
  return cudaGetLastError();
}

cudaError_t mlp_predict(const float* params, const float* feats, int32_t count, float* pred, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int tb = 128;
  k_mlp_forward<<<(unsigned)((count + tb - 1) / tb), tb, 0, s>>>(params, feats, count, nullptr, nullptr, pred);
  return cudaGetLastError();
}

cudaError_t mlp_adam_step(float* params, const float* grad, float* m1, float* m2, int32_t step, float lr,
                          cudaStream_t s) {
  k_adam<<<(PERM_MLP_PARAMS + 255) / 256, 256, 0, s>>>(params, grad, m1, m2, step, lr);
  return cudaGetLastError();
}

size_t mlp_scratch_floats(int32_t count) { return (size_t)count * (4 * H + 2); }
