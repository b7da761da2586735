// Closed-form first-order overlap (Eq. fo, with heights p_i p_j): one warp
// per pair over its flattened atom pairs, and the first-order Tanimoto of
// every (query, database) pair for the screen's prefilter. Terms are
// evaluated in FP32 with per-atom constants (SFU rsqrt and exp2 per term).
#include "device.cuh"
#include "internal.h"

namespace shp {
namespace {

constexpr int kThreads = 256;
constexpr int kFoWarps = kThreads / 32;

struct FoAtom {
  float x, y, z, beta;  // centre, beta' = 1 / (alpha log2 e)
};

struct FoWarpStage {
  FoAtom a[SHP_MAX_ATOMS], b[SHP_MAX_ATOMS];
  float la[SHP_MAX_ATOMS], lb[SHP_MAX_ATOMS];  // log2 w'
};

// Warp per pair: both molecules staged in shared memory with their per-atom
// constants (fo_atom_consts; B's centres posed once), lanes over the
// flattened atom pairs (i, j) so that every lane has work for any atom
// counts, FP32 terms w'_i w'_j r^3 2^(-r^2 d^2) summed per lane, then over
// the warp in FP64.
__global__ void __launch_bounds__(kThreads) fo_kernel(SetView A, const int32_t* ia, SetView B,
                                                      const int32_t* ib, const float* poses,
                                                      int64_t n_pairs, double* out) {
  __shared__ FoWarpStage stage[kFoWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k = (int64_t)blockIdx.x * kFoWarps + warp;
  if (k >= n_pairs) return;
  const int32_t xa = ia[k], xb = ib[k];
  if (xa < 0 || xa >= A.n_mol || xb < 0 || xb >= B.n_mol) {
    if (lane == 0) out[k] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  FoWarpStage& S = stage[warp];
  const Pose P = make_pose(poses ? poses + 7 * k : nullptr);
  const int32_t a0 = A.off[xa], na = A.off[xa + 1] - a0;
  const int32_t b0 = B.off[xb], nb = B.off[xb + 1] - b0;
  for (int i = lane; i < na; i += 32) {
    const float4 c = A.atom[a0 + i];
    float beta, lw;
    fo_atom_consts(c.w, A.aux[a0 + i].y, beta, lw);
    S.a[i] = FoAtom{c.x, c.y, c.z, beta};
    S.la[i] = lw;
  }
  for (int j = lane; j < nb; j += 32) {
    const float4 c = B.atom[b0 + j];
    const float3 p = apply_pose(P, make_float3(c.x, c.y, c.z));
    float beta, lw;
    fo_atom_consts(c.w, B.aux[b0 + j].y, beta, lw);
    S.b[j] = FoAtom{p.x, p.y, p.z, beta};
    S.lb[j] = lw;
  }
  __syncwarp();
  float acc = 0.f;
  const int total = na * nb;
  int i = lane / nb, j = lane - i * nb;
  for (int t = lane; t < total; t += 32) {
    const FoAtom a = S.a[i], b = S.b[j];
    const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    const float r = rsqrtf(a.beta + b.beta), rn = -r * r;
    const float e = fmaf(rn, fmaf(dx, dx, fmaf(dy, dy, dz * dz)), S.la[i] + S.lb[j]);
    acc = fmaf(-rn * r, ex2_approx(e), acc);
    j += 32;
    while (j >= nb) { j -= nb; ++i; }
  }
  const double tot = warp_sum((double)acc);
  if (lane == 0) out[k] = tot;
}

// First-order Tanimoto of every (query, database) pair: one thread per pair,
// the block's query atoms staged in shared memory (read as broadcasts), the
// thread's database atoms read once each from global memory. Threads take
// database molecules in the set's size order (atom count descending), so a
// warp's molecules have nearly equal atom counts. Each term is rewritten with
// per-atom constants: with beta'_i = 1 / (alpha_i log2 e),
// r = (beta'_i + beta'_j)^{-1/2} (so r^2 = log2(e) alpha_i alpha_j /
// (alpha_i + alpha_j)) and w'_i = p_i pi^{3/4} alpha_i^{-3/2} log2(e)^{-3/4},
//   p_i p_j (pi / (alpha_i + alpha_j))^{3/2} exp(-a d^2) = w'_i w'_j r^3 2^{-r^2 d^2},
// one SFU rsqrt and one SFU exp2 per atom pair (log2 w'_i folded into the
// exponent), two query atoms per packed FP32x2 instruction. FP32 terms and
// sum per pair (the prefilter ranks pairs; its values are not an estimate).
constexpr int kScreenThreads = 128;

// Two query atoms i, i + 1 (x, y, z, beta', log2 w' each as a pair); an odd
// count is padded with an atom of weight 0 (log2 w' = -inf).
struct __align__(16) FoAtom2 {
  float4 xy;  // x_i, x_i+1, y_i, y_i+1
  float4 zb;  // z_i, z_i+1, beta'_i, beta'_i+1
  float2 lw;  // log2 w'_i, log2 w'_i+1
  float2 pad;
};

// Queries per block: each thread screens its database molecule against all
// of them, so every database atom is read, and its constants computed, once
// per group of queries.
constexpr int kQueryGroup = 16;

__global__ void __launch_bounds__(kScreenThreads) fo_tanimoto_kernel(SetView Q, SetView D, const int32_t* order,
                                                                     const double* self_q, const double* self_db,
                                                                     float* T) {
  __shared__ FoAtom2 qa[kQueryGroup * (SHP_MAX_ATOMS / 2)];
  __shared__ int32_t qs[kQueryGroup + 1];  // first atom pair of each query of the group, and the end
  __shared__ float sacc[kQueryGroup][kScreenThreads];  // each thread's first-order sums
  const int32_t g0 = blockIdx.y * kQueryGroup;
  const int ng = min(kQueryGroup, Q.n_mol - g0);
  if (threadIdx.x == 0) {
    int32_t t = 0;
    for (int k = 0; k < ng; ++k) {
      qs[k] = t;
      t += (Q.off[g0 + k + 1] - Q.off[g0 + k] + 1) / 2;
    }
    for (int k = ng; k <= kQueryGroup; ++k) qs[k] = t;
  }
  __syncthreads();
  for (int k = 0; k < ng; ++k) {
    const int32_t q0 = Q.off[g0 + k], nq = Q.off[g0 + k + 1] - q0;
    for (int i2 = threadIdx.x; 2 * i2 < nq; i2 += kScreenThreads) {
      float v[2][5];
      for (int h = 0; h < 2; ++h) {
        const int i = 2 * i2 + h;
        if (i < nq) {
          const float4 a = Q.atom[q0 + i];
          v[h][0] = a.x; v[h][1] = a.y; v[h][2] = a.z;
          fo_atom_consts(a.w, Q.aux[q0 + i].y, v[h][3], v[h][4]);
        } else {
          v[h][0] = v[h][1] = v[h][2] = 0.f;
          v[h][3] = 1.f;
          v[h][4] = -INFINITY;
        }
      }
      FoAtom2 A;
      A.xy = make_float4(v[0][0], v[1][0], v[0][1], v[1][1]);
      A.zb = make_float4(v[0][2], v[1][2], v[0][3], v[1][3]);
      A.lw = make_float2(v[0][4], v[1][4]);
      A.pad = make_float2(0.f, 0.f);
      qa[qs[k] + i2] = A;
    }
  }
  __syncthreads();
  const int64_t rank = (int64_t)blockIdx.x * kScreenThreads + threadIdx.x;
  if (rank >= D.n_mol) return;
  const int32_t d = order[rank];
  const int32_t d0 = D.off[d], nd = D.off[d + 1] - d0;
  for (int k = 0; k < kQueryGroup; ++k) sacc[k][threadIdx.x] = 0.f;
  for (int j = 0; j < nd; ++j) {
    const float4 b = D.atom[d0 + j];
    float bbeta, blw;
    fo_atom_consts(b.w, D.aux[d0 + j].y, bbeta, blw);
    const float wb = ex2_approx(blw);
    const float2 nbx = make_float2(-b.x, -b.x), nby = make_float2(-b.y, -b.y), nbz = make_float2(-b.z, -b.z);
    const float2 bb = make_float2(bbeta, bbeta);
    for (int k = 0; k < ng; ++k) {
      {
        float2 aj = make_float2(0.f, 0.f);  // minus the sum of r^3 2^e
#pragma unroll 4
        for (int i2 = qs[k]; i2 < qs[k + 1]; ++i2) {
          const FoAtom2 a = qa[i2];
          const float2 dx = __fadd2_rn(make_float2(a.xy.x, a.xy.y), nbx);
          const float2 dy = __fadd2_rn(make_float2(a.xy.z, a.xy.w), nby);
          const float2 dz = __fadd2_rn(make_float2(a.zb.x, a.zb.y), nbz);
          const float2 d2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
          const float2 sb = __fadd2_rn(make_float2(a.zb.z, a.zb.w), bb);
          const float2 r = make_float2(rsqrtf(sb.x), rsqrtf(sb.y));
          const float2 rn = __fmul2_rn(r, make_float2(-r.x, -r.y));  // -r^2
          const float2 e = __ffma2_rn(rn, d2, a.lw);
          const float2 r3n = __fmul2_rn(rn, r);                       // -r^3
          aj = __ffma2_rn(r3n, make_float2(ex2_approx(e.x), ex2_approx(e.y)), aj);
        }
        sacc[k][threadIdx.x] = fmaf(-wb, aj.x + aj.y, sacc[k][threadIdx.x]);
      }
    }
  }
  for (int k = 0; k < ng; ++k) {
    const double O = sacc[k][threadIdx.x];
    const double S = self_q[g0 + k] + self_db[d];
    T[(int64_t)(g0 + k) * D.n_mol + d] = (float)(O / (S - O));
  }
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
  const dim3 grid((unsigned)((D->n_mol + kScreenThreads - 1) / kScreenThreads),
                  (unsigned)((Q->n_mol + kQueryGroup - 1) / kQueryGroup));
  fo_tanimoto_kernel<<<grid, kScreenThreads, 0, (cudaStream_t)stream>>>(view(Q), view(D), D->order, fo_self_q,
                                                                         fo_self_db, T_fo);
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
  const int64_t blocks = (n_pairs + kFoWarps - 1) / kFoWarps;
  fo_kernel<<<(unsigned)blocks, kThreads, 0, (cudaStream_t)stream>>>(view(A), ia, view(B), ib, poseB, n_pairs,
                                                                       out);
  SHP_CUDA(cudaGetLastError());
  return SHP_OK;
}
