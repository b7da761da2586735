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

// First-order Tanimoto of every (query, database) pair: one thread per pair,
// the block's query atoms staged in shared memory (read as broadcasts), the
// thread's database atoms read once each from global memory. Terms in FP32
// with the SFU reciprocal, reciprocal square root and exp2; FP32 sum per
// pair (the prefilter ranks pairs; its values are not an estimate).
constexpr int kScreenThreads = 128;

__global__ void __launch_bounds__(kScreenThreads) fo_tanimoto_kernel(SetView Q, SetView D, const double* self_q,
                                                                     const double* self_db, float* T) {
  __shared__ float4 qa[SHP_MAX_ATOMS];
  __shared__ float qlp[SHP_MAX_ATOMS];
  const int32_t q = blockIdx.y;
  const int32_t q0 = Q.off[q], nq = Q.off[q + 1] - q0;
  for (int i = threadIdx.x; i < nq; i += kScreenThreads) {
    qa[i] = Q.atom[q0 + i];
    qlp[i] = Q.aux[q0 + i].y;
  }
  __syncthreads();
  const int64_t d = (int64_t)blockIdx.x * kScreenThreads + threadIdx.x;
  if (d >= D.n_mol) return;
  const int32_t d0 = D.off[d], nd = D.off[d + 1] - d0;
  const float kLog2e = 1.4426950408889634f, kPi = 3.14159265358979f;
  float acc = 0.f;
  for (int j = 0; j < nd; ++j) {
    const float4 b = D.atom[d0 + j];
    const float lpb = D.aux[d0 + j].y;
    for (int i = 0; i < nq; ++i) {
      const float4 a = qa[i];
      const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
      const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      const float r = __fdividef(1.f, a.w + b.w);
      const float t = kPi * r;
      const float e = fmaf(-kLog2e * a.w * b.w * r, d2, qlp[i] + lpb);
      acc = fmaf(t * t * rsqrtf(t), ex2_approx(e), acc);
    }
  }
  const double S = self_q[q] + self_db[d];
  T[(int64_t)q * D.n_mol + d] = (float)((double)acc / (S - (double)acc));
}

}  // namespace
}  // namespace shp

using namespace shp;

extern "C" int fo_tanimoto_screen(shp_set Q, shp_set D, const double* fo_self_q, const double* fo_self_db,
                                  float* T_fo, void* stream) {
  clear_error();
  if (!Q || !D) { set_error("fo_tanimoto_screen: NULL set"); return SHP_EINVAL; }
  if (Q->n_mol == 0 || D->n_mol == 0) return SHP_OK;
  if (!fo_self_q || !fo_self_db || !T_fo) { set_error("fo_tanimoto_screen: NULL array"); return SHP_EINVAL; }
  if (Q->n_mol > 65535) { set_error("fo_tanimoto_screen: at most 65535 queries per call"); return SHP_ERANGE; }
  const dim3 grid((unsigned)((D->n_mol + kScreenThreads - 1) / kScreenThreads), (unsigned)Q->n_mol);
  fo_tanimoto_kernel<<<grid, kScreenThreads, 0, (cudaStream_t)stream>>>(view(Q), view(D), fo_self_q, fo_self_db,
                                                                         T_fo);
  SHP_CUDA(cudaGetLastError());
  return SHP_OK;
}

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
