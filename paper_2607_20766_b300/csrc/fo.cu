// Closed-form first-order overlap (Eq. fo, with heights p_i p_j): one warp
// per pair, lanes over A's atoms, B's atoms read as warp-wide broadcasts.
// Terms are evaluated in FP32 (SFU exp2) and each lane's partial sum is
// reduced over the warp in FP64.
#include "device.cuh"
#include "internal.h"

namespace shp {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fo_kernel(SetView A, const int32_t* ia, SetView B,
                                                      const int32_t* ib, const float* poses,
                                                      int64_t n_pairs, double* out) {
  const int64_t k = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= n_pairs) return;
  const int32_t xa = ia[k], xb = ib[k];
  if (xa < 0 || xa >= A.n_mol || xb < 0 || xb >= B.n_mol) {
    if (lane == 0) out[k] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  const Pose P = make_pose(poses ? poses + 7 * k : nullptr);
  const int32_t a0 = A.off[xa], na = A.off[xa + 1] - a0;
  const int32_t b0 = B.off[xb], nb = B.off[xb + 1] - b0;
  const float kLog2e = 1.4426950408889634f, kPi = 3.14159265358979f;
  float acc = 0.f;
  for (int i = lane; i < na; i += 32) {
    const float4 ai = A.atom[a0 + i];
    const float lpi = A.aux[a0 + i].y;
    for (int j = 0; j < nb; ++j) {
      const float4 bj = B.atom[b0 + j];
      const float3 c = apply_pose(P, make_float3(bj.x, bj.y, bj.z));
      const float dx = ai.x - c.x, dy = ai.y - c.y, dz = ai.z - c.z;
      const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      const float s = ai.w + bj.w;
      const float inv = 1.0f / s;
      const float t = kPi * inv;
      const float e = fmaf(-kLog2e * ai.w * bj.w * inv, d2, lpi + B.aux[b0 + j].y);
      acc = fmaf(t * sqrtf(t), ex2_approx(e), acc);
    }
  }
  const double tot = warp_sum((double)acc);
  if (lane == 0) out[k] = tot;
}

}  // namespace
}  // namespace shp

using namespace shp;

extern "C" int fo_overlap(shp_set A, const int32_t* ia, shp_set B, const int32_t* ib, int64_t n_pairs,
                          const float* poseB, double* out, void* stream) {
  clear_error();
  if (!A || !B) { set_error("fo_overlap: NULL set"); return SHP_EINVAL; }
  if (n_pairs < 0) { set_error("fo_overlap: negative n_pairs"); return SHP_EINVAL; }
  if (n_pairs == 0) return SHP_OK;
  if (!ia || !ib || !out) { set_error("fo_overlap: NULL array"); return SHP_EINVAL; }
  const int64_t blocks = (n_pairs * 32 + kThreads - 1) / kThreads;
  fo_kernel<<<(unsigned)blocks, kThreads, 0, (cudaStream_t)stream>>>(view(A), ia, view(B), ib, poseB, n_pairs,
                                                                       out);
  SHP_CUDA(cudaGetLastError());
  return SHP_OK;
}
