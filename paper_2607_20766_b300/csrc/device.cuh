// Device building blocks of the importance-sampling estimator (sm_103a).
//
// Counter-based random words (Philox4x32-10, Salmon et al. SC'11), the
// Box-Muller normals and alias pick of the sample layout, and the packed
// FP32x2 Gaussian evaluation of Eq. occ / Eq. union used by every kernel.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "shape.h"

namespace shp {

// ---------------------------------------------------------------- Philox

struct Key {
  uint32_t k0, k1;
};

__device__ __forceinline__ uint4 philox10(uint4 c, Key k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c = make_uint4(hi1 ^ c.y ^ k.k0, lo1, hi0 ^ c.w ^ k.k1, lo0);
    k.k0 += 0x9E3779B9u;
    k.k1 += 0xBB67AE85u;
  }
  return c;
}

// ---------------------------------------------------------------- math

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Box-Muller on two words: u1 = ((a >> 8) + 1) 2^-24 in (0, 1],
// t = 2 (b >> 8) 2^-24 - 1 in [-1, 1) (both exact in FP32),
// rho = sqrt(-2 ln u1), normals (rho cos(pi t), rho sin(pi t)).
// Uses the SFU approximations of log2, sin and cos.
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1) {
  const float u1 = __uint2float_rn((a >> 8) + 1u) * 5.9604644775390625e-08f;  // 2^-24
  const float t = __uint2float_rn(b >> 8) * 1.1920928955078125e-07f - 1.0f;  // 2^-23
  const float q = fmaxf(-1.3862943611198906f * __log2f(u1), 1e-30f);        // -2 ln u1
  const float rho = q * rsqrtf(q);
  const float ang = 3.14159265358979f * t;
  float s, c;
  __sincosf(ang, &s, &c);
  z0 = rho * c;
  z1 = rho * s;
}

// Per-atom constants of the closed-form first-order term (Eq. fo): with
// beta' = 1 / (alpha log2 e) and log2 w' = log2 p - (3/2) log2 alpha +
// (3/4) (log2 pi - log2 log2 e), the term of atoms i, j at distance d is
// w'_i w'_j r^3 2^(-r^2 d^2) with r = (beta'_i + beta'_j)^(-1/2)
// (r^2 = log2(e) alpha_i alpha_j / (alpha_i + alpha_j)).
__device__ __forceinline__ void fo_atom_consts(float alpha, float lp, float& beta, float& lw) {
  const float kLog2e = 1.4426950408889634f;
  const float kC = 0.8420473173955658f;  // (3/4) (log2 pi - log2 log2 e)
  beta = __fdividef(1.f, alpha * kLog2e);
  lw = fmaf(-1.5f, __log2f(alpha), lp + kC);
}

// ---------------------------------------------------------------- tables

struct Pose {
  float r[9];
  float t[3];
  bool identity;
};

__device__ __forceinline__ Pose make_pose(const float* p) {
  Pose P;
  if (p == nullptr) {
    P.identity = true;
    for (int i = 0; i < 9; ++i) P.r[i] = (i % 4 == 0) ? 1.f : 0.f;
    P.t[0] = P.t[1] = P.t[2] = 0.f;
    return P;
  }
  P.identity = false;
  float w = p[0], x = p[1], y = p[2], z = p[3];
  const float inv = rsqrtf(w * w + x * x + y * y + z * z);
  w *= inv; x *= inv; y *= inv; z *= inv;
  P.r[0] = 1.f - 2.f * (y * y + z * z); P.r[1] = 2.f * (x * y - w * z); P.r[2] = 2.f * (x * z + w * y);
  P.r[3] = 2.f * (x * y + w * z); P.r[4] = 1.f - 2.f * (x * x + z * z); P.r[5] = 2.f * (y * z - w * x);
  P.r[6] = 2.f * (x * z - w * y); P.r[7] = 2.f * (y * z + w * x); P.r[8] = 1.f - 2.f * (x * x + y * y);
  P.t[0] = p[4]; P.t[1] = p[5]; P.t[2] = p[6];
  return P;
}

__device__ __forceinline__ float3 apply_pose(const Pose& P, float3 c) {
  if (P.identity) return c;
  return make_float3(fmaf(P.r[0], c.x, fmaf(P.r[1], c.y, fmaf(P.r[2], c.z, P.t[0]))),
                     fmaf(P.r[3], c.x, fmaf(P.r[4], c.y, fmaf(P.r[5], c.z, P.t[1]))),
                     fmaf(P.r[6], c.x, fmaf(P.r[7], c.y, fmaf(P.r[8], c.z, P.t[2]))));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace shp
