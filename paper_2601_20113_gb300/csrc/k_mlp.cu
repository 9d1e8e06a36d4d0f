// Training and batch inference of the block-rank MLP (32 -> 64 -> 64 -> 1,
// ReLU), BF16 weights with FP32 accumulation.  The MLP is not in the paper:
// it predicts the rank the bisection of Algorithm 1 would choose, from block
// features, so the compressor can test one candidate instead of searching.
//
// Parameter vector (FP32 master copy, kMlpNParam floats):
//   [mu 32][sigma 32][W1 64x32][b1 64][W2 64x64][b2 64][W3 64][b3 1]
// mu and sigma standardise the features and are not trained.  The forward
// and backward passes use the weights rounded to BF16 (round to nearest
// even); gradients update the FP32 masters (straight-through), with Adam.
//
// Training runs in one CTA: every gradient entry is one thread's sequential
// sum over the minibatch, so results are deterministic.
#include <cuda_bf16.h>

#include "dls_internal.cuh"

namespace dls {
namespace {

constexpr int kB = 128;             // largest minibatch
constexpr int kT = 256;             // threads
constexpr int kZs = kMlpF + 1;      // padded row strides (bank-conflict free)
constexpr int kHs = kMlpH + 1;

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

struct TrainSmem {
  float W[kMlpNParam];       // bf16-rounded weights (mu, sigma exact)
  float Z[kB * kZs];         // standardised features [b][f]
  float H1[kB * kHs];        // [b][h]
  float H2[kB * kHs];
  float D2[kB * kHs];        // dL/d(pre-activation 2)
  float D1[kB * kHs];        // dL/d(pre-activation 1)
  float y[kB], t[kB], dy[kB];
};

__device__ void load_weights(TrainSmem& S, const float* params) {
  for (int i = threadIdx.x; i < kMlpNParam; i += kT) {
    const float v = params[i];
    S.W[i] = (i < kMlpOffW1) ? v : bf16r(v);
  }
}

// Forward and backward over a minibatch of B samples `idx[b]`.  If grad_out is
// set, writes the gradient vector (zeros for mu, sigma) and the loss;
// otherwise applies one Adam step to params (m, v state) at step number `tstep`.
__device__ void minibatch(TrainSmem& S, const float* feat, const float* target, const int32_t* idx, int B,
                          float* params, float* m, float* v, int tstep, float lr, float* grad_out,
                          float* loss_out) {
  const int tid = threadIdx.x;
  __syncthreads();
  load_weights(S, params);
  for (int e = tid; e < B * kMlpF; e += kT) {
    const int b = e / kMlpF, f = e % kMlpF;
    const float x = feat[(int64_t)idx[b] * kMlpF + f];
    S.Z[b * kZs + f] = (x - S.W[kMlpOffMu + f]) / S.W[kMlpOffSig + f];
  }
  for (int b = tid; b < B; b += kT) S.t[b] = target[idx[b]];
  __syncthreads();
  // layer 1
  for (int e = tid; e < B * kMlpH; e += kT) {
    const int b = e % B, h = e / B;
    float acc = S.W[kMlpOffB1 + h];
    for (int f = 0; f < kMlpF; ++f) acc = fmaf(S.W[kMlpOffW1 + h * kMlpF + f], S.Z[b * kZs + f], acc);
    S.H1[b * kHs + h] = acc > 0.0f ? acc : 0.0f;
  }
  __syncthreads();
  // layer 2
  for (int e = tid; e < B * kMlpH; e += kT) {
    const int b = e % B, h = e / B;
    float acc = S.W[kMlpOffB2 + h];
    for (int k = 0; k < kMlpH; ++k) acc = fmaf(S.W[kMlpOffW2 + h * kMlpH + k], S.H1[b * kHs + k], acc);
    S.H2[b * kHs + h] = acc > 0.0f ? acc : 0.0f;
  }
  __syncthreads();
  for (int b = tid; b < B; b += kT) {
    float acc = S.W[kMlpOffB3];
    for (int k = 0; k < kMlpH; ++k) acc = fmaf(S.W[kMlpOffW3 + k], S.H2[b * kHs + k], acc);
    S.y[b] = acc;
    S.dy[b] = 2.0f * (acc - S.t[b]) / (float)B;
  }
  __syncthreads();
  if (tid == 0 && loss_out) {
    float l = 0.0f;
    for (int b = 0; b < B; ++b) { const float d = S.y[b] - S.t[b]; l = fmaf(d, d, l); }
    *loss_out = l / (float)B;
  }
  const float b1c = 1.0f - powf(0.9f, (float)tstep), b2c = 1.0f - powf(0.999f, (float)tstep);
  auto apply = [&](int i, float g) {
    if (grad_out) { grad_out[i] = g; return; }
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi / b1c) / (sqrtf(vi / b2c) + 1e-8f);
  };
  if (grad_out)
    for (int i = tid; i < kMlpOffW1; i += kT) grad_out[i] = 0.0f;
  // output layer gradients; dL/d(pre2)
  for (int k = tid; k <= kMlpH; k += kT) {
    float g = 0.0f;
    if (k < kMlpH) {
      for (int b = 0; b < B; ++b) g = fmaf(S.dy[b], S.H2[b * kHs + k], g);
      apply(kMlpOffW3 + k, g);
    } else {
      for (int b = 0; b < B; ++b) g += S.dy[b];
      apply(kMlpOffB3, g);
    }
  }
  for (int e = tid; e < B * kMlpH; e += kT) {
    const int b = e % B, k = e / B;
    S.D2[b * kHs + k] = S.H2[b * kHs + k] > 0.0f ? S.W[kMlpOffW3 + k] * S.dy[b] : 0.0f;
  }
  __syncthreads();
  // layer 2 weight gradients
  for (int e = tid; e < kMlpH * kMlpH; e += kT) {
    const int h = e / kMlpH, k = e % kMlpH;
    float g = 0.0f;
    for (int b = 0; b < B; ++b) g = fmaf(S.D2[b * kHs + h], S.H1[b * kHs + k], g);
    apply(kMlpOffW2 + e, g);
  }
  for (int h = tid; h < kMlpH; h += kT) {
    float g = 0.0f;
    for (int b = 0; b < B; ++b) g += S.D2[b * kHs + h];
    apply(kMlpOffB2 + h, g);
  }
  // dL/d(pre1)
  for (int e = tid; e < B * kMlpH; e += kT) {
    const int b = e % B, k = e / B;
    float acc = 0.0f;
    for (int h = 0; h < kMlpH; ++h) acc = fmaf(S.W[kMlpOffW2 + h * kMlpH + k], S.D2[b * kHs + h], acc);
    S.D1[b * kHs + k] = S.H1[b * kHs + k] > 0.0f ? acc : 0.0f;
  }
  __syncthreads();
  for (int e = tid; e < kMlpH * kMlpF; e += kT) {
    const int h = e / kMlpF, f = e % kMlpF;
    float g = 0.0f;
    for (int b = 0; b < B; ++b) g = fmaf(S.D1[b * kHs + h], S.Z[b * kZs + f], g);
    apply(kMlpOffW1 + e, g);
  }
  for (int h = tid; h < kMlpH; h += kT) {
    float g = 0.0f;
    for (int b = 0; b < B; ++b) g += S.D1[b * kHs + h];
    apply(kMlpOffB1 + h, g);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kT) k_mlp_train(float* params, float* adam, const float* feat, const float* target,
                                                  const int32_t* order, int64_t n_order, int steps, int B,
                                                  float lr, int step0, float* loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  __shared__ int32_t idx[kB];
  float* m = adam;
  float* v = adam + kMlpNParam;
  for (int s = 0; s < steps; ++s) {
    for (int b = threadIdx.x; b < B; b += kT) idx[b] = order[((int64_t)s * B + b) % n_order];
    minibatch(S, feat, target, idx, B, params, m, v, step0 + s + 1, lr, nullptr, loss ? loss + s : nullptr);
  }
}

__global__ void __launch_bounds__(kT) k_mlp_grad(const float* params, const float* feat, const float* target, int B,
                                                 float* grad, float* loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  __shared__ int32_t idx[kB];
  for (int b = threadIdx.x; b < B; b += kT) idx[b] = b;
  minibatch(S, feat, target, idx, B, const_cast<float*>(params), nullptr, nullptr, 1, 0.0f, grad, loss);
}

__global__ void k_mlp_forward(const float* params, const float* feat, int64_t n, float* y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float z[kMlpF], h1[kMlpH];
  for (int f = 0; f < kMlpF; ++f) z[f] = (feat[i * kMlpF + f] - params[kMlpOffMu + f]) / params[kMlpOffSig + f];
  for (int h = 0; h < kMlpH; ++h) {
    float acc = bf16r(params[kMlpOffB1 + h]);
    for (int f = 0; f < kMlpF; ++f) acc = fmaf(bf16r(params[kMlpOffW1 + h * kMlpF + f]), z[f], acc);
    h1[h] = acc > 0.0f ? acc : 0.0f;
  }
  float out = bf16r(params[kMlpOffB3]);
  for (int h = 0; h < kMlpH; ++h) {
    float acc = bf16r(params[kMlpOffB2 + h]);
    for (int k = 0; k < kMlpH; ++k) acc = fmaf(bf16r(params[kMlpOffW2 + h * kMlpH + k]), h1[k], acc);
    acc = acc > 0.0f ? acc : 0.0f;
    out = fmaf(bf16r(params[kMlpOffW3 + h]), acc, out);
  }
  y[i] = out;
}

}  // namespace

int launch_mlp_train(float* params, float* adam, const float* feat, const float* target, const int32_t* order,
                     int64_t n_order, int steps, int B, float lr, int step0, float* loss, cudaStream_t s) {
  const size_t smem = sizeof(TrainSmem);
  if (cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return DLS_ERR_CUDA;
  k_mlp_train<<<1, kT, smem, s>>>(params, adam, feat, target, order, n_order, steps, B, lr, step0, loss);
  return cudaGetLastError() == cudaSuccess ? DLS_OK : DLS_ERR_CUDA;
}

int launch_mlp_grad(const float* params, const float* feat, const float* target, int B, float* grad, float* loss,
                    cudaStream_t s) {
  const size_t smem = sizeof(TrainSmem);
  if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return DLS_ERR_CUDA;
  k_mlp_grad<<<1, kT, smem, s>>>(params, feat, target, B, grad, loss);
  return cudaGetLastError() == cudaSuccess ? DLS_OK : DLS_ERR_CUDA;
}

int launch_mlp_forward(const float* params, const float* feat, int64_t n, float* y, cudaStream_t s) {
  if (n <= 0) return DLS_OK;
  k_mlp_forward<<<(unsigned)cdiv(n, 128), 128, 0, s>>>(params, feat, n, y);
  return cudaGetLastError() == cudaSuccess ? DLS_OK : DLS_ERR_CUDA;
}

int mlp_max_batch() { return kB; }

}  // namespace dls
