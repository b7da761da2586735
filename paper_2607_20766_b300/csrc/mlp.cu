// Per-atom control-variate network: neighbour features, forward pass, fused
// forward/backward with a deterministic gradient reduction, Adam step.
//
// The network is small (6401 parameters, ~6.3k multiply-adds per atom); it
// runs on the CUDA cores with the weights rounded to BF16 and held in
// shared memory as FP32, activations and accumulation in FP32. Its cost is
// well under one percent of the sampling it serves.
#include <cmath>

#include <cuda_bf16.h>

#include "device.cuh"
#include "internal.h"

namespace shp {
namespace {

constexpr int kIn = SHP_MLP_IN, kH = SHP_MLP_HIDDEN, kP = SHP_MLP_PARAMS;
constexpr int oW1 = 0, oB1 = kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH;
static_assert(oB3 + 1 == kP, "parameter layout");

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.7071067811865476f)); }

__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.7071067811865476f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

__device__ void load_weights(float* W, const float* params) {
  for (int i = threadIdx.x; i < kP; i += blockDim.x) W[i] = bf16r(params[i]);
  __syncthreads();
}

// ---------------------------------------------------------------- features

__global__ void features_kernel(SetView S, int64_t n_atoms, float* feat) {
  // one thread per atom; binary search for its molecule
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_atoms) return;
  int32_t lo = 0, hi = S.n_mol;
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) >> 1;
    if (S.off[mid] <= a) lo = mid; else hi = mid;
  }
  const int32_t a0 = S.off[lo], n = S.off[lo + 1] - a0, i = (int32_t)(a - a0);
  const float4 ci = S.atom[a];
  float bd[16];
  int bi[16];
  int cnt = 0;
  for (int j = 0; j < n; ++j) {
    if (j == i) continue;
    const float4 cj = S.atom[a0 + j];
    const float dx = ci.x - cj.x, dy = ci.y - cj.y, dz = ci.z - cj.z;
    const float d = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    // insert (d, j) into the sorted list of the 16 nearest (ties keep lower j first)
    if (cnt == 16 && !(d < bd[15])) continue;
    int pos = cnt < 16 ? cnt : 15;
    while (pos > 0 && bd[pos - 1] > d) {
      bd[pos] = bd[pos - 1];
      bi[pos] = bi[pos - 1];
      --pos;
    }
    bd[pos] = d;
    bi[pos] = j;
    if (cnt < 16) ++cnt;
  }
  float* f = feat + (int64_t)kIn * a;
  for (int k = 0; k < 16; ++k) {
    if (k < cnt) {
      f[2 * k] = bd[k] * 0.25f;
      f[2 * k + 1] = S.radius[a0 + bi[k]] * (1.f / 1.7f);
    } else {
      f[2 * k] = 2.5f;
      f[2 * k + 1] = 0.f;
    }
  }
  f[32] = S.radius[a] * (1.f / 1.7f);
}

// ---------------------------------------------------------------- forward

constexpr int kFwdThreads = 128;

__global__ void __launch_bounds__(kFwdThreads) forward_kernel(const float* params, const float* x,
                                                              const int32_t* rows, int64_t n, float* y) {
  __shared__ float W[kP];
  load_weights(W, params);
  const int64_t k = (int64_t)blockIdx.x * kFwdThreads + threadIdx.x;
  if (k >= n) return;
  const int64_t r = rows ? rows[k] : k;
  const float* xr = x + kIn * r;
  float xv[kIn];
#pragma unroll
  for (int i = 0; i < kIn; ++i) xv[i] = xr[i];
  float h1[kH];
#pragma unroll 4
  for (int j = 0; j < kH; ++j) {
    float z = W[oB1 + j];
#pragma unroll
    for (int i = 0; i < kIn; ++i) z = fmaf(W[oW1 + kIn * j + i], xv[i], z);
    h1[j] = gelu(z);
  }
  float out = W[oB3];
  for (int j = 0; j < kH; ++j) {
    float z = W[oB2 + j];
#pragma unroll
    for (int i = 0; i < kH; ++i) z = fmaf(W[oW2 + kH * j + i], h1[i], z);
    out = fmaf(W[oW3 + j], gelu(z), out);
  }
  y[k] = out;
}

// ---------------------------------------------------------------- backward

constexpr int kBwdAtoms = 64;  // atoms (threads) per block

struct BwdSmem {
  float W[kP];
  float X[kIn][kBwdAtoms];
  float H1[kH][kBwdAtoms];
  float D1[kH][kBwdAtoms];  // gelu'(z1), then delta1
  float H2[kH][kBwdAtoms];
  float D2[kH][kBwdAtoms];  // gelu'(z2), then delta2
  float dy[kBwdAtoms];
  float loss[kBwdAtoms];
};

// Per block: forward of its atoms, dL/dy = 2 (y - t) / n, back-propagation,
// and the block's partial parameter gradient summed over its atoms, written
// to part[block][kP + 1] (last slot: the block's sum of squared errors).
__global__ void __launch_bounds__(kBwdAtoms) backward_kernel(const float* params, const float* x,
                                                             const float* target, const int32_t* rows, int64_t n,
                                                             float* part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BwdSmem& s = *reinterpret_cast<BwdSmem*>(smem_raw);
  load_weights(s.W, params);
  const int t = threadIdx.x;
  const int64_t k = (int64_t)blockIdx.x * kBwdAtoms + t;
  const bool valid = k < n;
  const int64_t r = valid ? (rows ? rows[k] : k) : 0;
  for (int i = 0; i < kIn; ++i) s.X[i][t] = valid ? x[kIn * r + i] : 0.f;
  for (int j = 0; j < kH; ++j) {
    float z = s.W[oB1 + j];
    for (int i = 0; i < kIn; ++i) z = fmaf(s.W[oW1 + kIn * j + i], s.X[i][t], z);
    s.H1[j][t] = gelu(z);
    s.D1[j][t] = gelu_grad(z);
  }
  float y = s.W[oB3];
  for (int j = 0; j < kH; ++j) {
    float z = s.W[oB2 + j];
    for (int i = 0; i < kH; ++i) z = fmaf(s.W[oW2 + kH * j + i], s.H1[i][t], z);
    const float h = gelu(z);
    s.H2[j][t] = h;
    s.D2[j][t] = gelu_grad(z);
    y = fmaf(s.W[oW3 + j], h, y);
  }
  const float err = valid ? y - target[r] : 0.f;
  const float dy = 2.f * err / (float)n;
  s.dy[t] = dy;
  s.loss[t] = err * err;
  for (int j = 0; j < kH; ++j) s.D2[j][t] *= dy * s.W[oW3 + j];  // delta2
  for (int i = 0; i < kH; ++i) {
    float acc = 0.f;
    for (int j = 0; j < kH; ++j) acc = fmaf(s.W[oW2 + kH * j + i], s.D2[j][t], acc);
    s.D1[i][t] *= acc;  // delta1
  }
  __syncthreads();
  float* out = part + (int64_t)blockIdx.x * (kP + 1);
  for (int e = t; e < kP + 1; e += kBwdAtoms) {
    float acc = 0.f;
    if (e < oB1) {
      const int j = e / kIn, i = e - j * kIn;
      for (int a = 0; a < kBwdAtoms; ++a) acc = fmaf(s.D1[j][a], s.X[i][a], acc);
    } else if (e < oW2) {
      const int j = e - oB1;
      for (int a = 0; a < kBwdAtoms; ++a) acc += s.D1[j][a];
    } else if (e < oB2) {
      const int j = (e - oW2) / kH, i = (e - oW2) - j * kH;
      for (int a = 0; a < kBwdAtoms; ++a) acc = fmaf(s.D2[j][a], s.H1[i][a], acc);
    } else if (e < oW3) {
      const int j = e - oB2;
      for (int a = 0; a < kBwdAtoms; ++a) acc += s.D2[j][a];
    } else if (e < oB3) {
      const int j = e - oW3;
      for (int a = 0; a < kBwdAtoms; ++a) acc = fmaf(s.dy[a], s.H2[j][a], acc);
    } else if (e == oB3) {
      for (int a = 0; a < kBwdAtoms; ++a) acc += s.dy[a];
    } else {
      for (int a = 0; a < kBwdAtoms; ++a) acc += s.loss[a];
    }
    out[e] = acc;
  }
}

// grad[e] = sum over blocks of part[b][e] (fixed order); loss = SSE / n.
__global__ void reduce_kernel(const float* part, int64_t n_blocks, int64_t n, float* grad, double* loss) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > kP) return;
  double acc = 0.0;
  for (int64_t b = 0; b < n_blocks; ++b) acc += (double)part[b * (kP + 1) + e];
  if (e < kP) grad[e] = (float)acc;
  else *loss = acc / (double)n;
}

__global__ void adam_kernel(float* p, float* m, float* v, const float* g, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
  const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace
}  // namespace shp

using namespace shp;

extern "C" int cv_features(shp_set S, float* feat, void* stream) {
  clear_error();
  if (!S || (!feat && S->n_atoms)) { set_error("cv_features: NULL argument"); return SHP_EINVAL; }
  if (S->n_atoms == 0) return SHP_OK;
  const int threads = 128;
  features_kernel<<<(unsigned)((S->n_atoms + threads - 1) / threads), threads, 0, (cudaStream_t)stream>>>(
      view(S), S->n_atoms, feat);
  SHP_CUDA(cudaGetLastError());
  return SHP_OK;
}

extern "C" int mlp_forward(const float* params, const float* x, const int32_t* rows, int64_t n, float* y,
                           void* stream) {
  clear_error();
  if (n < 0 || (n > 0 && (!params || !x || !y))) { set_error("mlp_forward: bad arguments"); return SHP_EINVAL; }
  if (n == 0) return SHP_OK;
  forward_kernel<<<(unsigned)((n + kFwdThreads - 1) / kFwdThreads), kFwdThreads, 0, (cudaStream_t)stream>>>(
      params, x, rows, n, y);
  SHP_CUDA(cudaGetLastError());
  return SHP_OK;
}

extern "C" int mlp_loss_grad(const float* params, const float* x, const float* target, const int32_t* rows,
                             int64_t n, float* grad, double* loss, void* stream) {
  clear_error();
  if (n <= 0 || !params || !x || !target || !grad || !loss) { set_error("mlp_loss_grad: bad arguments"); return SHP_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t blocks = (n + kBwdAtoms - 1) / kBwdAtoms;
  float* part = nullptr;
  SHP_CUDA(dev_alloc((void**)&part, sizeof(float) * (size_t)blocks * (kP + 1), st));
  cudaError_t e = cudaFuncSetAttribute(backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(BwdSmem));
  if (e == cudaSuccess) {
    backward_kernel<<<(unsigned)blocks, kBwdAtoms, sizeof(BwdSmem), st>>>(params, x, target, rows, n, part);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    reduce_kernel<<<(kP + 1 + 255) / 256, 256, 0, st>>>(part, blocks, n, grad, loss);
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaFreeAsync(part, st);
  if (e != cudaSuccess) return cuda_fail(e, "mlp_loss_grad");
  if (e2 != cudaSuccess) return cuda_fail(e2, "mlp_loss_grad: cudaFreeAsync");
  return SHP_OK;
}

namespace shp {

// The loss/gradient kernels writing their per-block partials to `part`
// (at least ceil(n / 64) x 6402 floats, caller-provided).
int mlp_loss_grad_into(const float* params, const float* x, const float* target, const int32_t* rows, int64_t n,
                       float* part, float* grad, double* loss, cudaStream_t st) {
  const int64_t blocks = (n + kBwdAtoms - 1) / kBwdAtoms;
  SHP_CUDA(cudaFuncSetAttribute(backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BwdSmem)));
  backward_kernel<<<(unsigned)blocks, kBwdAtoms, sizeof(BwdSmem), st>>>(params, x, target, rows, n, part);
  SHP_CUDA(cudaGetLastError());
  reduce_kernel<<<(kP + 1 + 255) / 256, 256, 0, st>>>(part, blocks, n, grad, loss);
  SHP_CUDA(cudaGetLastError());
  return SHP_OK;
}

}  // namespace shp

extern "C" int mlp_adam(float* params, float* m, float* v, const float* grad, int64_t n_params, int64_t step,
                        float lr, float beta1, float beta2, float eps, void* stream) {
  clear_error();
  if (!params || !m || !v || !grad || n_params <= 0 || step < 1) { set_error("mlp_adam: bad arguments"); return SHP_EINVAL; }
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  adam_kernel<<<(unsigned)((n_params + 255) / 256), 256, 0, (cudaStream_t)stream>>>(params, m, v, grad, n_params, lr,
                                                                                    beta1, beta2, eps, c1, c2);
  SHP_CUDA(cudaGetLastError());
  return SHP_OK;
}
