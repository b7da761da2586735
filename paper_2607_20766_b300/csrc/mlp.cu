// Per-atom control-variate network: neighbour features, forward pass, fused
// forward/backward with a deterministic gradient reduction, Adam step.
//
// The network is small (6401 parameters, ~6.3k multiply-adds per atom); it
// runs on the CUDA cores with the weights rounded to BF16 and held in
// shared memory as FP32, activations and accumulation in FP32, as
// register-tiled GEMMs over 32-atom tiles for training.
#include <cmath>
#include <cstddef>

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

// gelu(z) = z Phi(z) and gelu'(z) = Phi(z) + z phi(z) from one erf.
__device__ __forceinline__ void gelu_both(float z, float& h, float& d) {
  const float c = 1.f + erff(z * 0.7071067811865476f);
  h = 0.5f * z * c;
  d = 0.5f * c + z * 0.3989422804014327f * expf(-0.5f * z * z);
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

// Loss and gradient: persistent blocks of 256 threads, each over a fixed
// range of 32-atom tiles (so the result does not depend on scheduling). Per
// tile, four small GEMMs with 2x4 (forward, back-propagation) or 4x4
// (weight gradients) register tiles per thread, operands in shared memory
// in the layout each GEMM reads with vector loads:
//   z1 = X W1^T + b1, h1 = gelu(z1)          (X^T, W1^T)
//   z2 = h1 W2^T + b2, h2 = gelu(z2), y      (h1^T, W2^T)
//   d2 = dy w3 * gelu'(z2), d1 = (d2 W2) * gelu'(z1)   (d2^T, W2)
//   gW2 += d2^T h1, gW1 += d1^T [X 1]        (d2, h1, d1, X; the column of
//                                             ones gives gb1)
// with dy = 2 (y - t) / n. The weight gradients stay in registers over the
// block's tiles; each block writes one partial row of part[kP + 1] (last
// slot: its sum of squared errors).
constexpr int kTile = 32;       // atoms per tile
constexpr int kTrThreads = 256;
constexpr int kXP = 36;         // X row: 33 features, a one, two zeros

struct TrainSmem {
  float W1T[kIn][kH];           // W1^T (input, hidden)
  float W2T[kH][kH];            // W2^T (h1, h2)
  float W2N[kH][kH];            // W2 (h2, h1)
  float b1[kH], b2[kH], w3[kH];
  float b3[4];                  // b3 (padded: the arrays below take vector loads)
  float XT[kIn][kTile];         // the tile's features, atom-contiguous
  float XN[kTile][kXP];         // the same, feature-contiguous, with the ones column
  float AT[kH][kTile];          // h1^T, then d2^T
  float H1N[kTile][kH];
  float D2N[kTile][kH];
  float D1N[kTile][kH];
  float red[16][kH];            // block reductions at the end
  float sse[kTrThreads], sdy[kTrThreads];
};
// every array read with float2 / float4 loads starts on a 16-byte boundary,
// and its rows are whole multiples of 16 bytes
static_assert(offsetof(TrainSmem, W1T) % 16 == 0 && offsetof(TrainSmem, W2T) % 16 == 0, "alignment");
static_assert(offsetof(TrainSmem, W2N) % 16 == 0 && offsetof(TrainSmem, XT) % 16 == 0, "alignment");
static_assert(offsetof(TrainSmem, XN) % 16 == 0 && offsetof(TrainSmem, AT) % 16 == 0, "alignment");
static_assert(offsetof(TrainSmem, H1N) % 16 == 0 && offsetof(TrainSmem, D2N) % 16 == 0, "alignment");
static_assert(offsetof(TrainSmem, D1N) % 16 == 0, "alignment");
static_assert((kH * 4) % 16 == 0 && (kTile * 4) % 16 == 0 && (kXP * 4) % 16 == 0, "row sizes");

__global__ void __launch_bounds__(kTrThreads) train_kernel(const float* params, const float* x, const float* target,
                                                           const int32_t* rows, int64_t n, int64_t tiles_per_block,
                                                           float* part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& s = *reinterpret_cast<TrainSmem*>(smem_raw);
  const int tid = threadIdx.x;
  for (int e = tid; e < kH * kIn; e += kTrThreads) {
    const int h = e / kIn, i = e - h * kIn;
    s.W1T[i][h] = bf16r(params[oW1 + e]);
  }
  for (int e = tid; e < kH * kH; e += kTrThreads) {
    const int h2 = e / kH, h1 = e - h2 * kH;
    const float w = bf16r(params[oW2 + e]);
    s.W2T[h1][h2] = w;
    s.W2N[h2][h1] = w;
  }
  if (tid < kH) {
    s.b1[tid] = bf16r(params[oB1 + tid]);
    s.b2[tid] = bf16r(params[oB2 + tid]);
    s.w3[tid] = bf16r(params[oW3 + tid]);
  }
  if (tid == 0) s.b3[0] = bf16r(params[oB3]);
  // forward / back-propagation tile of this thread: atoms 2 ta, 2 ta + 1,
  // hidden units 4 th .. 4 th + 3; gradient tile: rows 4 gr .., columns 4 gc ..
  const int ta = tid >> 4, th = tid & 15;
  const int gr = tid >> 4, gc = tid & 15;
  float gW2[4][4] = {}, gW1[4][4] = {}, gw3[4] = {};
  float gb2 = 0.f, sse = 0.f, sdy = 0.f;
  const float inv_n = 2.f / (float)n;
  const int64_t n_tiles = (n + kTile - 1) / kTile;
  const int64_t t0 = (int64_t)blockIdx.x * tiles_per_block;
  const int64_t t1 = t0 + tiles_per_block < n_tiles ? t0 + tiles_per_block : n_tiles;
  // each tile's features (this thread's share of the kTile x kXP entries)
  // and the targets of this thread's two atoms are loaded one tile ahead, so
  // the gather's latency overlaps the previous tile's GEMMs
  constexpr int kXPer = (kTile * kXP + kTrThreads - 1) / kTrThreads;
  float xv[kXPer], tv[2];
  auto load_tile = [&](int64_t tile) {
    const int64_t a_base = tile * kTile;
#pragma unroll
    for (int j = 0; j < kXPer; ++j) {
      const int e = tid + j * kTrThreads;
      const int a = e / kXP, i = e - a * kXP;
      const int64_t k = a_base + a;
      float v = 0.f;
      if (e < kTile * kXP && k < n) {
        const int64_t r = rows ? rows[k] : k;
        v = i < kIn ? x[(int64_t)kIn * r + i] : (i == kIn ? 1.f : 0.f);
      }
      xv[j] = v;
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int64_t k = a_base + 2 * ta + r;
      tv[r] = k < n ? target[rows ? rows[k] : k] : 0.f;
    }
  };
  if (t0 < t1) load_tile(t0);
  for (int64_t tile = t0; tile < t1; ++tile) {
    __syncthreads();  // the previous tile's buffers (and the weights, first time) are done with
    const int64_t a_base = tile * kTile;
#pragma unroll
    for (int j = 0; j < kXPer; ++j) {
      const int e = tid + j * kTrThreads;
      if (e < kTile * kXP) {
        const int a = e / kXP, i = e - a * kXP;
        s.XN[a][i] = xv[j];
        if (i < kIn) s.XT[i][a] = xv[j];
      }
    }
    const float tcur[2] = {tv[0], tv[1]};
    __syncthreads();
    if (tile + 1 < t1) load_tile(tile + 1);
    // z1 and h1
    float z[2][4], d1g[2][4];
#pragma unroll
    for (int c = 0; c < 4; ++c) z[0][c] = z[1][c] = s.b1[4 * th + c];
#pragma unroll 3
    for (int i = 0; i < kIn; ++i) {
      const float2 xa = *reinterpret_cast<const float2*>(&s.XT[i][2 * ta]);
      const float4 w = *reinterpret_cast<const float4*>(&s.W1T[i][4 * th]);
      z[0][0] = fmaf(xa.x, w.x, z[0][0]); z[0][1] = fmaf(xa.x, w.y, z[0][1]);
      z[0][2] = fmaf(xa.x, w.z, z[0][2]); z[0][3] = fmaf(xa.x, w.w, z[0][3]);
      z[1][0] = fmaf(xa.y, w.x, z[1][0]); z[1][1] = fmaf(xa.y, w.y, z[1][1]);
      z[1][2] = fmaf(xa.y, w.z, z[1][2]); z[1][3] = fmaf(xa.y, w.w, z[1][3]);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      float h[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        gelu_both(z[r][c], h[c], d1g[r][c]);
        s.AT[4 * th + c][2 * ta + r] = h[c];
      }
      *reinterpret_cast<float4*>(&s.H1N[2 * ta + r][4 * th]) = make_float4(h[0], h[1], h[2], h[3]);
    }
    __syncthreads();
    // z2, h2 and y
#pragma unroll
    for (int c = 0; c < 4; ++c) z[0][c] = z[1][c] = s.b2[4 * th + c];
#pragma unroll 4
    for (int k = 0; k < kH; ++k) {
      const float2 ha = *reinterpret_cast<const float2*>(&s.AT[k][2 * ta]);
      const float4 w = *reinterpret_cast<const float4*>(&s.W2T[k][4 * th]);
      z[0][0] = fmaf(ha.x, w.x, z[0][0]); z[0][1] = fmaf(ha.x, w.y, z[0][1]);
      z[0][2] = fmaf(ha.x, w.z, z[0][2]); z[0][3] = fmaf(ha.x, w.w, z[0][3]);
      z[1][0] = fmaf(ha.y, w.x, z[1][0]); z[1][1] = fmaf(ha.y, w.y, z[1][1]);
      z[1][2] = fmaf(ha.y, w.z, z[1][2]); z[1][3] = fmaf(ha.y, w.w, z[1][3]);
    }
    float h2[2][4], d2[2][4], dy[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      float part_y = 0.f;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        gelu_both(z[r][c], h2[r][c], d2[r][c]);
        part_y = fmaf(s.w3[4 * th + c], h2[r][c], part_y);
      }
      // the 16 threads of an atom pair are one half-warp
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) part_y += __shfl_xor_sync(0xffffffffu, part_y, o);
      const int64_t k = a_base + 2 * ta + r;
      float err = 0.f;
      if (k < n) err = part_y + s.b3[0] - tcur[r];
      dy[r] = err * inv_n;
      if (th == 0) { sse = fmaf(err, err, sse); sdy += dy[r]; }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      gw3[c] = fmaf(dy[0], h2[0][c], fmaf(dy[1], h2[1][c], gw3[c]));
      d2[0][c] *= dy[0] * s.w3[4 * th + c];
      d2[1][c] *= dy[1] * s.w3[4 * th + c];
    }
    __syncthreads();  // every thread has read h1^T from AT
#pragma unroll
    for (int r = 0; r < 2; ++r) {
#pragma unroll
      for (int c = 0; c < 4; ++c) s.AT[4 * th + c][2 * ta + r] = d2[r][c];
      *reinterpret_cast<float4*>(&s.D2N[2 * ta + r][4 * th]) = make_float4(d2[r][0], d2[r][1], d2[r][2], d2[r][3]);
    }
    __syncthreads();
    // d1 = (d2 W2) * gelu'(z1)
    float g[2][4] = {};
#pragma unroll 4
    for (int k = 0; k < kH; ++k) {
      const float2 da = *reinterpret_cast<const float2*>(&s.AT[k][2 * ta]);
      const float4 w = *reinterpret_cast<const float4*>(&s.W2N[k][4 * th]);
      g[0][0] = fmaf(da.x, w.x, g[0][0]); g[0][1] = fmaf(da.x, w.y, g[0][1]);
      g[0][2] = fmaf(da.x, w.z, g[0][2]); g[0][3] = fmaf(da.x, w.w, g[0][3]);
      g[1][0] = fmaf(da.y, w.x, g[1][0]); g[1][1] = fmaf(da.y, w.y, g[1][1]);
      g[1][2] = fmaf(da.y, w.z, g[1][2]); g[1][3] = fmaf(da.y, w.w, g[1][3]);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
      *reinterpret_cast<float4*>(&s.D1N[2 * ta + r][4 * th]) =
          make_float4(g[r][0] * d1g[r][0], g[r][1] * d1g[r][1], g[r][2] * d1g[r][2], g[r][3] * d1g[r][3]);
    __syncthreads();
    // weight gradients over the tile's atoms
#pragma unroll 4
    for (int a = 0; a < kTile; ++a) {
      const float4 dv = *reinterpret_cast<const float4*>(&s.D2N[a][4 * gr]);
      const float4 hv = *reinterpret_cast<const float4*>(&s.H1N[a][4 * gc]);
      const float dd[4] = {dv.x, dv.y, dv.z, dv.w}, hh[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) gW2[u][v] = fmaf(dd[u], hh[v], gW2[u][v]);
    }
    if (gc < kXP / 4) {
#pragma unroll 4
      for (int a = 0; a < kTile; ++a) {
        const float4 dv = *reinterpret_cast<const float4*>(&s.D1N[a][4 * gr]);
        const float4 xv = *reinterpret_cast<const float4*>(&s.XN[a][4 * gc]);
        const float dd[4] = {dv.x, dv.y, dv.z, dv.w}, xx[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) gW1[u][v] = fmaf(dd[u], xx[v], gW1[u][v]);
      }
    }
    if (tid < kH)
      for (int a = 0; a < kTile; ++a) gb2 += s.D2N[a][tid];
  }
  // the block's partial row
  float* out = part + (int64_t)blockIdx.x * (kP + 1);
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) out[oW2 + kH * (4 * gr + u) + 4 * gc + v] = gW2[u][v];
  if (gc < kXP / 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int i = 4 * gc + v;
        if (i < kIn) out[oW1 + kIn * (4 * gr + u) + i] = gW1[u][v];
        else if (i == kIn) out[oB1 + 4 * gr + u] = gW1[u][v];
      }
  }
  if (tid < kH) out[oB2 + tid] = gb2;
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 4; ++c) s.red[ta][4 * th + c] = gw3[c];
  s.sse[tid] = sse;
  s.sdy[tid] = sdy;
  __syncthreads();
  if (tid < kH) {
    float acc = 0.f;
    for (int r = 0; r < 16; ++r) acc += s.red[r][tid];
    out[oW3 + tid] = acc;
  }
  if (tid == 0) {
    float a = 0.f, b = 0.f;
    for (int t = 0; t < kTrThreads; ++t) { a += s.sse[t]; b += s.sdy[t]; }
    out[kP] = a;
    out[oB3] = b;
  }
}

// Blocks of train_kernel for n rows: ranges of whole tiles, at most two
// blocks per SM and at most ceil(n / 64) (the partial rows callers provide).
int train_launch(const float* params, const float* x, const float* target, const int32_t* rows, int64_t n,
                 float* part, int64_t* n_blocks, cudaStream_t st) {
  int dev = 0, sms = 0;
  SHP_CUDA(cudaGetDevice(&dev));
  SHP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t n_tiles = (n + kTile - 1) / kTile;
  int64_t blocks = 2 * (int64_t)sms;
  const int64_t cap = (n + 63) / 64;
  if (blocks > cap) blocks = cap;
  if (blocks > n_tiles) blocks = n_tiles;
  const int64_t per = (n_tiles + blocks - 1) / blocks;
  blocks = (n_tiles + per - 1) / per;
  SHP_CUDA(cudaFuncSetAttribute(train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem)));
  train_kernel<<<(unsigned)blocks, kTrThreads, sizeof(TrainSmem), st>>>(params, x, target, rows, n, per, part);
  SHP_CUDA(cudaGetLastError());
  *n_blocks = blocks;
  return SHP_OK;
}

// grad[e] = sum over blocks of part[b][e] (fixed order); loss = SSE / n.
// Blocks of 32 columns x 8 row groups: row group r sums rows r, r + 8, ...
// in FP64, then the 8 group sums are added in order (a fixed order for every
// run).
constexpr int kRedCols = 32, kRedGroups = 8;

__global__ void __launch_bounds__(kRedCols * kRedGroups) reduce_kernel(const float* part, int64_t n_blocks, int64_t n,
                                                                      float* grad, double* loss) {
  __shared__ double sums[kRedGroups][kRedCols];
  const int c = threadIdx.x % kRedCols, r = threadIdx.x / kRedCols;
  const int e = blockIdx.x * kRedCols + c;
  double acc = 0.0;
  if (e <= kP)
    for (int64_t b = r; b < n_blocks; b += kRedGroups) acc += (double)part[b * (kP + 1) + e];
  sums[r][c] = acc;
  __syncthreads();
  if (r == 0 && e <= kP) {
    double t = 0.0;
    for (int g = 0; g < kRedGroups; ++g) t += sums[g][c];
    if (e < kP) grad[e] = (float)t;
    else *loss = t / (double)n;
  }
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
  const int64_t rows_max = (n + 63) / 64;
  float* part = nullptr;
  SHP_CUDA(dev_alloc((void**)&part, sizeof(float) * (size_t)rows_max * (kP + 1), st));
  const int rc = mlp_loss_grad_into(params, x, target, rows, n, part, grad, loss, st);
  const cudaError_t e2 = cudaFreeAsync(part, st);
  if (rc) return rc;
  if (e2 != cudaSuccess) return cuda_fail(e2, "mlp_loss_grad: cudaFreeAsync");
  return SHP_OK;
}

namespace shp {

// The loss/gradient kernels writing their per-block partials to `part`
// (at least ceil(n / 64) x 6402 floats, caller-provided).
int mlp_loss_grad_into(const float* params, const float* x, const float* target, const int32_t* rows, int64_t n,
                       float* part, float* grad, double* loss, cudaStream_t st) {
  int64_t blocks = 0;
  const int rc = train_launch(params, x, target, rows, n, part, &blocks, st);
  if (rc) return rc;
  reduce_kernel<<<(kP + 1 + kRedCols - 1) / kRedCols, kRedCols * kRedGroups, 0, st>>>(part, blocks, n, grad, loss);
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

extern "C" int mlp_train_epoch(float* params, float* m, float* v, const float* x, const float* target,
                               const int32_t* perm, int64_t n, int64_t batch, int64_t step0, float lr, float beta1,
                               float beta2, float eps, double* losses, void* stream) {
  clear_error();
  if (!params || !m || !v || !x || !target || !perm || !losses || n <= 0 || batch <= 0 || step0 < 0) {
    set_error("mlp_train_epoch: bad arguments");
    return SHP_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t b = batch < n ? batch : n;
  float* part = nullptr;
  float* grad = nullptr;
  cudaError_t e = dev_alloc((void**)&part, sizeof(float) * (size_t)((b + 63) / 64) * (kP + 1), st);
  if (e == cudaSuccess) e = dev_alloc((void**)&grad, sizeof(float) * kP, st);
  int rc = e == cudaSuccess ? SHP_OK : cuda_fail(e, "mlp_train_epoch: scratch");
  // the same launches, in the same order, as mlp_loss_grad then mlp_adam per
  // minibatch: the result is that of the step-by-step calls
  int64_t step = step0;
  for (int64_t s0 = 0; s0 < n && rc == SHP_OK; s0 += b) {
    const int64_t nb = n - s0 < b ? n - s0 : b;
    rc = mlp_loss_grad_into(params, x, target, perm + s0, nb, part, grad, losses + s0 / b, st);
    if (rc) break;
    ++step;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<(unsigned)((kP + 255) / 256), 256, 0, st>>>(params, m, v, grad, kP, lr, beta1, beta2, eps, c1, c2);
    const cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) rc = cuda_fail(le, "mlp_train_epoch: adam");
  }
  for (void* p : {(void*)part, (void*)grad})
    if (p) cudaFreeAsync(p, st);
  return rc;
}
