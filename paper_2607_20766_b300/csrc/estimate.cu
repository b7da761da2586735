// Importance-sampling estimators on sm_103a: pair overlaps (first order and
// union), union volumes / self-overlaps, and the fixed-budget Tanimoto
// screen (Eq. expectation, Eq. var, Eq. union-is, Sec. confidence-bounded
// screening).
//
// Work decomposition: one warp owns one work item (a molecule pair, or one
// molecule for volumes) and runs all of its samples; warps take items from a
// device queue (persistent kernel, items largest-first for screens). Per
// item and direction the warp stages, in shared memory, the sampled
// molecule's component table (centre, sigma, alias) and both molecules'
// Gaussian coefficients in the frame of the sampled molecule's centroid.
// Each lane then draws 4 sample pairs per batch (256 samples per warp) and
// evaluates every atom of both molecules with packed FP32x2 FMAs and one
// SFU exp2 per Gaussian; FP32 batch partials are folded into a hi/lo pair
// per lane and reduced over the warp in FP64.
#include <cmath>

#include "device.cuh"
#include "internal.h"

namespace shp {
namespace {

constexpr int kSP = 4;     // sample pairs per lane per batch
constexpr int kWarps = 8;  // warps per CTA
constexpr int kThreads = kWarps * 32;

struct __align__(16) WarpTables {
  Coef x[SHP_MAX_ATOMS];       // sampled molecule
  Coef y[SHP_MAX_ATOMS];       // other molecule
  float4 samp[SHP_MAX_ATOMS];  // sampled molecule: centre - origin, sigma
  uint32_t thr[SHP_MAX_ATOMS];
  uint8_t alias[SHP_MAX_ATOMS];
};
constexpr size_t kSmemBytes = sizeof(WarpTables) * kWarps;

struct MolRef {
  int32_t a0, n;
};

__device__ __forceinline__ MolRef mol_ref(const SetView& S, int32_t m) {
  const int32_t a0 = S.off[m];
  return MolRef{a0, S.off[m + 1] - a0};
}

__device__ float3 centroid(const SetView& S, MolRef M, const Pose& P, int lane) {
  float sx = 0.f, sy = 0.f, sz = 0.f;
  for (int i = lane; i < M.n; i += 32) {
    const float4 a = S.atom[M.a0 + i];
    const float3 c = apply_pose(P, make_float3(a.x, a.y, a.z));
    sx += c.x; sy += c.y; sz += c.z;
  }
  const float inv = 1.0f / (float)M.n;
  return make_float3(warp_sum(sx) * inv, warp_sum(sy) * inv, warp_sum(sz) * inv);
}

__device__ void stage_coef(Coef* dst, const SetView& S, MolRef M, const Pose& P, float3 o, int lane) {
  const float kLog2e = 1.4426950408889634f;
  for (int i = lane; i < M.n; i += 32) {
    const float4 a = S.atom[M.a0 + i];
    const float lp = S.aux[M.a0 + i].y;
    const float3 c = apply_pose(P, make_float3(a.x, a.y, a.z));
    const float dx = c.x - o.x, dy = c.y - o.y, dz = c.z - o.z;
    const float al = a.w * kLog2e;
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    Coef k;
    k.a = make_float2(-al, -al);
    const float bx = 2.f * al * dx, by = 2.f * al * dy, bz = 2.f * al * dz;
    k.bx = make_float2(bx, bx);
    k.by = make_float2(by, by);
    k.bz = make_float2(bz, bz);
    const float c0 = fmaf(-al, d2, lp);
    k.c0 = make_float2(c0, c0);
    k.pad = make_float2(0.f, 0.f);
    dst[i] = k;
  }
}

__device__ void stage_samp(WarpTables& T, const SetView& S, MolRef M, const Pose& P, float3 o, int lane) {
  for (int i = lane; i < M.n; i += 32) {
    const float4 a = S.atom[M.a0 + i];
    const float3 c = apply_pose(P, make_float3(a.x, a.y, a.z));
    T.samp[i] = make_float4(c.x - o.x, c.y - o.y, c.z - o.z, S.aux[M.a0 + i].x);
    T.thr[i] = S.thr[M.a0 + i];
    T.alias[i] = S.alias[M.a0 + i];
  }
}

// Alias pick: column j = hi32(x n); keep j if lo32(x n) < thr_j.
__device__ __forceinline__ int pick(const WarpTables& T, int n, uint32_t x) {
  const unsigned long long prod = (unsigned long long)x * (unsigned)n;
  const uint32_t j = (uint32_t)(prod >> 32), f = (uint32_t)prod;
  return f < T.thr[j] ? (int)j : (int)T.alias[j];
}

// m = sum g and q = prod (1 - g) over one molecule's Gaussians, for kSP
// sample pairs held as packed (even, odd) sample float2s.
__device__ __forceinline__ void eval_table(const Coef* __restrict__ tab, int n,
                                           const float2 (&rx)[kSP], const float2 (&ry)[kSP],
                                           const float2 (&rz)[kSP], const float2 (&rr)[kSP],
                                           float2 (&m)[kSP], float2 (&q)[kSP]) {
#pragma unroll 2
  for (int j = 0; j < n; ++j) {
    const float2 ka = tab[j].a, kbx = tab[j].bx, kby = tab[j].by, kbz = tab[j].bz, kc = tab[j].c0;
#pragma unroll
    for (int p = 0; p < kSP; ++p) {
      float2 e = __ffma2_rn(ka, rr[p], kc);
      e = __ffma2_rn(kbx, rx[p], e);
      e = __ffma2_rn(kby, ry[p], e);
      e = __ffma2_rn(kbz, rz[p], e);
      const float2 g = make_float2(ex2_approx(e.x), ex2_approx(e.y));
      m[p] = __fadd2_rn(m[p], g);
      q[p].x = fmaf(-g.x, q[p].x, q[p].x);
      q[p].y = fmaf(-g.y, q[p].y, q[p].y);
    }
  }
}

// One proposal direction: n samples from the staged molecule (T.x, T.samp)
// evaluated against itself and, unless kSelf, against T.y. Returns the warp
// totals of the shifted values, out = {sum (fa-Ka), sum (fa-Ka)^2,
// sum (fb-Kb), sum (fb-Kb)^2} with shift = {Ka, Kb} the first unit's values
// (a warp-uniform shift keeps the one-pass variance free of cancellation):
//   cross: fa = m_Y (first order), fb = (u_X / m_X) u_Y (union)
//   self:  fa = u_X / m_X (volume), fb = u_X^2 / m_X (self-overlap)
// With antithetic pairs the unit is the mean of a sample and its reflection.
template <bool kSelf>
__device__ void run_direction(const WarpTables& T, int nx, int ny, uint32_t n, Key key, uint64_t stream,
                              uint32_t tag, bool anti, int lane, double out[4], float shift[2]) {
  const uint32_t P = (n + 1u) >> 1;
  const uint32_t slo = (uint32_t)stream, shi = (uint32_t)(stream >> 32);
  float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
  for (uint32_t base = 0; base < P; base += 32u * kSP) {
    float2 rx[kSP], ry[kSP], rz[kSP], rr[kSP], valid[kSP];
#pragma unroll
    for (int p = 0; p < kSP; ++p) {
      const uint32_t s = base + (uint32_t)p * 32u + (uint32_t)lane;
      const bool ok0 = s < P;
      const bool ok1 = ok0 && (2u * s + 1u < n);
      const uint4 w0 = philox10(make_uint4(2u * s, slo, shi, tag), key);
      const uint4 w1 = philox10(make_uint4(2u * s + 1u, slo, shi, tag), key);
      float n0, n1, n2, n3, n4, n5;
      box_muller(w0.z, w0.w, n0, n1);
      box_muller(w1.x, w1.y, n2, n3);
      box_muller(w1.z, w1.w, n4, n5);
      const float4 c0 = T.samp[pick(T, nx, w0.x)];
      const float ax = fmaf(c0.w, n0, c0.x), ay = fmaf(c0.w, n1, c0.y), az = fmaf(c0.w, n4, c0.z);
      float bx, by, bz;
      if (anti) {
        bx = fmaf(-c0.w, n0, c0.x); by = fmaf(-c0.w, n1, c0.y); bz = fmaf(-c0.w, n4, c0.z);
      } else {
        const float4 c1 = T.samp[pick(T, nx, w0.y)];
        bx = fmaf(c1.w, n2, c1.x); by = fmaf(c1.w, n3, c1.y); bz = fmaf(c1.w, n5, c1.z);
      }
      rx[p] = make_float2(ax, bx);
      ry[p] = make_float2(ay, by);
      rz[p] = make_float2(az, bz);
      rr[p] = make_float2(fmaf(ax, ax, fmaf(ay, ay, az * az)), fmaf(bx, bx, fmaf(by, by, bz * bz)));
      valid[p] = make_float2(ok0 ? 1.f : 0.f, ok1 ? 1.f : 0.f);
    }
    float2 m[kSP], q[kSP], fa[kSP], fb[kSP];
#pragma unroll
    for (int p = 0; p < kSP; ++p) { m[p] = make_float2(0.f, 0.f); q[p] = make_float2(1.f, 1.f); }
    eval_table(T.x, nx, rx, ry, rz, rr, m, q);
    if (kSelf) {
#pragma unroll
      for (int p = 0; p < kSP; ++p) {
        const float ux = 1.f - q[p].x, uy = 1.f - q[p].y;
        const float wx = __fdividef(ux, m[p].x), wy = __fdividef(uy, m[p].y);
        fa[p] = make_float2(wx, wy);
        fb[p] = make_float2(wx * ux, wy * uy);
      }
    } else {
      float2 w[kSP];
#pragma unroll
      for (int p = 0; p < kSP; ++p) {
        w[p] = make_float2(__fdividef(1.f - q[p].x, m[p].x), __fdividef(1.f - q[p].y, m[p].y));
        m[p] = make_float2(0.f, 0.f);
        q[p] = make_float2(1.f, 1.f);
      }
      eval_table(T.y, ny, rx, ry, rz, rr, m, q);
#pragma unroll
      for (int p = 0; p < kSP; ++p) {
        fa[p] = m[p];
        fb[p] = make_float2(w[p].x * (1.f - q[p].x), w[p].y * (1.f - q[p].y));
      }
    }
    if (base == 0) {
      // sample 0 (lane 0, pair 0) always exists since n >= 2
      shift[0] = __shfl_sync(0xffffffffu, anti ? 0.5f * (fa[0].x + fa[0].y) : fa[0].x, 0);
      shift[1] = __shfl_sync(0xffffffffu, anti ? 0.5f * (fb[0].x + fb[0].y) : fb[0].x, 0);
    }
    float b[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int p = 0; p < kSP; ++p) {
      if (anti) {
        const float ga = 0.5f * (fa[p].x + fa[p].y) - shift[0], gb = 0.5f * (fb[p].x + fb[p].y) - shift[1];
        const float v = valid[p].x;
        b[0] = fmaf(v, ga, b[0]);
        b[1] = fmaf(v * ga, ga, b[1]);
        b[2] = fmaf(v, gb, b[2]);
        b[3] = fmaf(v * gb, gb, b[3]);
      } else {
        const float2 v = valid[p];
        const float a0 = fa[p].x - shift[0], a1 = fa[p].y - shift[0];
        const float b0 = fb[p].x - shift[1], b1 = fb[p].y - shift[1];
        b[0] += v.x * a0 + v.y * a1;
        b[1] += v.x * a0 * a0 + v.y * a1 * a1;
        b[2] += v.x * b0 + v.y * b1;
        b[3] += v.x * b0 * b0 + v.y * b1 * b1;
      }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) acc2(hi[t], lo[t], b[t]);
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) out[t] = warp_sum((double)hi[t] + (double)lo[t]);
}

// est = Z mean, se = Z sqrt(s^2 / n) (n-1 sample variance, Eq. var) from
// sums s, s2 of the values shifted by K.
__device__ __forceinline__ void finish(double Z, double s, double s2, double K, double n, double& est,
                                       double& se) {
  const double dm = s / n;
  double var = n > 1.0 ? (s2 - s * dm) / (n - 1.0) : 0.0;
  var = var > 0.0 ? var : 0.0;
  est = Z * (K + dm);
  se = Z * sqrt(var / n);
}

struct CrossArgs {
  SetView A, B;
  // pair mode
  const int32_t* ia;
  const int32_t* ib;
  const float* pose;
  double* est;
  double* se;
  // screen mode
  const int32_t* order_b;
  int32_t n_q, n_db;
  const double* self_q;
  const double* self_db;
  float* T;
  float* seT;
  double* O;
  double* seO;
  // common
  int64_t n_items;
  Key key;
  uint64_t stream_base;
  uint32_t n;
  bool anti, symmetric;
  unsigned long long* queue;
};

template <bool kScreen>
__global__ void __launch_bounds__(kThreads, 2) cross_kernel(const CrossArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpTables& T = reinterpret_cast<WarpTables*>(smem_raw)[warp];
  const double n_eff = args.anti ? (double)(args.n / 2u) : (double)args.n;
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(args.queue, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= (unsigned long long)args.n_items) break;
    int32_t xa, xb;
    int64_t out_idx;
    const float* pose = nullptr;
    if (kScreen) {
      const int64_t rank = (int64_t)item / args.n_q;
      xa = (int32_t)((int64_t)item - rank * args.n_q);
      xb = args.order_b[rank];
      out_idx = (int64_t)xa * args.n_db + xb;
    } else {
      xa = args.ia[item];
      xb = args.ib[item];
      out_idx = (int64_t)item;
      if (args.pose) pose = args.pose + 7 * (int64_t)item;
    }
    if (xa < 0 || xa >= args.A.n_mol || xb < 0 || xb >= args.B.n_mol) {
      if (lane == 0 && !kScreen) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        args.est[2 * out_idx] = nan; args.est[2 * out_idx + 1] = nan;
        args.se[2 * out_idx] = nan; args.se[2 * out_idx + 1] = nan;
      }
      continue;
    }
    const uint64_t stream = args.stream_base + (uint64_t)out_idx;
    const MolRef MA = mol_ref(args.A, xa), MB = mol_ref(args.B, xb);
    const Pose PA = make_pose(nullptr), PB = make_pose(pose);
    double s0[4], s1[4] = {0.0, 0.0, 0.0, 0.0};
    float k0[2], k1[2] = {0.f, 0.f};
    {
      const float3 o = centroid(args.A, MA, PA, lane);
      __syncwarp();
      stage_coef(T.x, args.A, MA, PA, o, lane);
      stage_coef(T.y, args.B, MB, PB, o, lane);
      stage_samp(T, args.A, MA, PA, o, lane);
      __syncwarp();
      run_direction<false>(T, MA.n, MB.n, args.n, args.key, stream, SHP_TAG_AB, args.anti, lane, s0, k0);
    }
    if (args.symmetric) {
      const float3 o = centroid(args.B, MB, PB, lane);
      __syncwarp();
      stage_coef(T.x, args.B, MB, PB, o, lane);
      stage_coef(T.y, args.A, MA, PA, o, lane);
      stage_samp(T, args.B, MB, PB, o, lane);
      __syncwarp();
      run_direction<false>(T, MB.n, MA.n, args.n, args.key, stream, SHP_TAG_BA, args.anti, lane, s1, k1);
    }
    __syncwarp();
    if (lane == 0) {
      const double ZA = args.A.Z[xa], ZB = args.B.Z[xb];
      double e[2], sd[2];
      for (int slot = 0; slot < 2; ++slot) {
        double e0, se0;
        finish(ZA, s0[2 * slot], s0[2 * slot + 1], k0[slot], n_eff, e0, se0);
        if (args.symmetric) {
          double e1, se1;
          finish(ZB, s1[2 * slot], s1[2 * slot + 1], k1[slot], n_eff, e1, se1);
          e[slot] = 0.5 * (e0 + e1);
          sd[slot] = 0.5 * sqrt(se0 * se0 + se1 * se1);
        } else {
          e[slot] = e0;
          sd[slot] = se0;
        }
      }
      if (kScreen) {
        for (int slot = 0; slot < 2; ++slot) {
          const double S = args.self_q[2 * (int64_t)xa + slot] + args.self_db[2 * (int64_t)xb + slot];
          const double den = S - e[slot];
          args.T[2 * out_idx + slot] = (float)(e[slot] / den);
          args.seT[2 * out_idx + slot] = (float)(fabs(S / (den * den)) * sd[slot]);
          if (args.O) args.O[2 * out_idx + slot] = e[slot];
          if (args.seO) args.seO[2 * out_idx + slot] = sd[slot];
        }
      } else {
        args.est[2 * out_idx] = e[0]; args.est[2 * out_idx + 1] = e[1];
        args.se[2 * out_idx] = sd[0]; args.se[2 * out_idx + 1] = sd[1];
      }
    }
  }
}

struct SelfArgs {
  SetView S;
  const int32_t* idx;
  int64_t n_items;
  Key key;
  uint64_t stream_base;
  uint32_t n;
  bool anti;
  double* vol;
  double* vol_se;
  double* self_ov;
  double* self_se;
  unsigned long long* queue;
};

__global__ void __launch_bounds__(kThreads, 2) self_kernel(const SelfArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpTables& T = reinterpret_cast<WarpTables*>(smem_raw)[warp];
  const double n_eff = args.anti ? (double)(args.n / 2u) : (double)args.n;
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(args.queue, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= (unsigned long long)args.n_items) break;
    const int32_t xm = args.idx ? args.idx[item] : (int32_t)item;
    if (xm < 0 || xm >= args.S.n_mol) {
      if (lane == 0) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        args.vol[item] = nan;
        if (args.vol_se) args.vol_se[item] = nan;
        if (args.self_ov) args.self_ov[item] = nan;
        if (args.self_se) args.self_se[item] = nan;
      }
      continue;
    }
    const MolRef M = mol_ref(args.S, xm);
    const Pose P = make_pose(nullptr);
    const float3 o = centroid(args.S, M, P, lane);
    __syncwarp();
    stage_coef(T.x, args.S, M, P, o, lane);
    stage_samp(T, args.S, M, P, o, lane);
    __syncwarp();
    double s[4];
    float k[2];
    run_direction<true>(T, M.n, 0, args.n, args.key, args.stream_base + item, SHP_TAG_SELF, args.anti, lane, s,
                        k);
    __syncwarp();
    if (lane == 0) {
      const double Z = args.S.Z[xm];
      double e, sd;
      finish(Z, s[0], s[1], k[0], n_eff, e, sd);
      args.vol[item] = e;
      if (args.vol_se) args.vol_se[item] = sd;
      finish(Z, s[2], s[3], k[1], n_eff, e, sd);
      if (args.self_ov) args.self_ov[item] = e;
      if (args.self_se) args.self_se[item] = sd;
    }
  }
}

template <class Kernel>
int persistent_grid(Kernel k, int64_t n_items, int* grid) {
  static int sms = 0;
  int dev = 0;
  SHP_CUDA(cudaGetDevice(&dev));
  SHP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SHP_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
  int per_sm = 0;
  SHP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, kSmemBytes));
  if (per_sm < 1) per_sm = 1;
  const int64_t need = (n_items + kWarps - 1) / kWarps;
  int64_t g = (int64_t)sms * per_sm;
  if (need < g) g = need;
  *grid = (int)(g < 1 ? 1 : g);
  return SHP_OK;
}

int check_mc(const shp_mc* mc, const char* who) {
  if (!mc) { set_error("%s: NULL shp_mc", who); return SHP_EINVAL; }
  if (mc->n_samples < 2) { set_error("%s: n_samples must be >= 2", who); return SHP_EINVAL; }
  if ((mc->flags & SHP_ANTITHETIC) && (mc->n_samples & 1u)) {
    set_error("%s: antithetic sampling needs an even n_samples", who);
    return SHP_EINVAL;
  }
  if (mc->flags & ~(SHP_SYMMETRIC | SHP_ANTITHETIC)) { set_error("%s: unknown flags", who); return SHP_EINVAL; }
  return SHP_OK;
}

// Launch a persistent kernel with a stream-ordered queue counter.
template <class Kernel, class Args>
int launch_queued(Kernel k, Args args, int64_t n_items, cudaStream_t st) {
  int grid = 0;
  int rc = persistent_grid(k, n_items, &grid);
  if (rc) return rc;
  unsigned long long* q = nullptr;
  SHP_CUDA(cudaMallocAsync((void**)&q, sizeof(unsigned long long), st));
  cudaError_t e = cudaMemsetAsync(q, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    args.queue = q;
    k<<<grid, kThreads, kSmemBytes, st>>>(args);
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaFreeAsync(q, st);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
  return SHP_OK;
}

}  // namespace
}  // namespace shp

using namespace shp;

extern "C" int overlap_estimate(shp_set A, const int32_t* ia, shp_set B, const int32_t* ib, int64_t n_pairs,
                                const float* poseB, const shp_mc* mc, double* est, double* se, void* stream) {
  clear_error();
  if (!A || !B) { set_error("overlap_estimate: NULL set"); return SHP_EINVAL; }
  int rc = check_mc(mc, "overlap_estimate");
  if (rc) return rc;
  if (n_pairs < 0) { set_error("overlap_estimate: negative n_pairs"); return SHP_EINVAL; }
  if (n_pairs == 0) return SHP_OK;
  if (!ia || !ib || !est || !se) { set_error("overlap_estimate: NULL array"); return SHP_EINVAL; }
  CrossArgs a{};
  a.A = view(A);
  a.B = view(B);
  a.ia = ia;
  a.ib = ib;
  a.pose = poseB;
  a.est = est;
  a.se = se;
  a.n_items = n_pairs;
  a.key = Key{(uint32_t)mc->seed, (uint32_t)(mc->seed >> 32)};
  a.stream_base = mc->stream_base;
  a.n = mc->n_samples;
  a.anti = (mc->flags & SHP_ANTITHETIC) != 0;
  a.symmetric = (mc->flags & SHP_SYMMETRIC) != 0;
  return launch_queued(cross_kernel<false>, a, n_pairs, (cudaStream_t)stream);
}

extern "C" int union_volume_estimate(shp_set S, const int32_t* idx, int64_t n, const shp_mc* mc, double* vol,
                                     double* vol_se, double* self_ov, double* self_se, void* stream) {
  clear_error();
  if (!S) { set_error("union_volume_estimate: NULL set"); return SHP_EINVAL; }
  int rc = check_mc(mc, "union_volume_estimate");
  if (rc) return rc;
  if (mc->flags & SHP_SYMMETRIC) { set_error("union_volume_estimate: SHP_SYMMETRIC does not apply"); return SHP_EINVAL; }
  if (n < 0) { set_error("union_volume_estimate: negative n"); return SHP_EINVAL; }
  if (n == 0) return SHP_OK;
  if (!vol) { set_error("union_volume_estimate: NULL vol"); return SHP_EINVAL; }
  if (!idx && n > S->n_mol) { set_error("union_volume_estimate: n exceeds the set size"); return SHP_ERANGE; }
  SelfArgs a{};
  a.S = view(S);
  a.idx = idx;
  a.n_items = n;
  a.key = Key{(uint32_t)mc->seed, (uint32_t)(mc->seed >> 32)};
  a.stream_base = mc->stream_base;
  a.n = mc->n_samples;
  a.anti = (mc->flags & SHP_ANTITHETIC) != 0;
  a.vol = vol;
  a.vol_se = vol_se;
  a.self_ov = self_ov;
  a.self_se = self_se;
  return launch_queued(self_kernel, a, n, (cudaStream_t)stream);
}

extern "C" int tanimoto_screen(shp_set Q, shp_set D, const shp_screen* cfg, const double* self_q,
                               const double* self_db, float* T, float* seT, double* O_out, double* seO_out,
                               void* stream) {
  clear_error();
  if (!Q || !D || !cfg) { set_error("tanimoto_screen: NULL set or config"); return SHP_EINVAL; }
  if (cfg->n_fixed < 2) { set_error("tanimoto_screen: n_fixed must be >= 2"); return SHP_EINVAL; }
  if ((cfg->flags & SHP_ANTITHETIC) && (cfg->n_fixed & 1u)) {
    set_error("tanimoto_screen: antithetic sampling needs an even n_fixed");
    return SHP_EINVAL;
  }
  if (cfg->flags & ~SHP_ANTITHETIC) { set_error("tanimoto_screen: unknown flags"); return SHP_EINVAL; }
  const int64_t n_items = (int64_t)Q->n_mol * D->n_mol;
  if (n_items == 0) return SHP_OK;
  if (!self_q || !self_db || !T || !seT) { set_error("tanimoto_screen: NULL array"); return SHP_EINVAL; }
  CrossArgs a{};
  a.A = view(Q);
  a.B = view(D);
  a.order_b = D->order;
  a.n_q = Q->n_mol;
  a.n_db = D->n_mol;
  a.self_q = self_q;
  a.self_db = self_db;
  a.T = T;
  a.seT = seT;
  a.O = O_out;
  a.seO = seO_out;
  a.n_items = n_items;
  a.key = Key{(uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32)};
  a.stream_base = cfg->stream_base;
  a.n = cfg->n_fixed;
  a.anti = (cfg->flags & SHP_ANTITHETIC) != 0;
  a.symmetric = true;
  return launch_queued(cross_kernel<true>, a, n_items, (cudaStream_t)stream);
}
