// Importance-sampling estimators on sm_103a: pair overlaps (first order and
// union), union volumes / self-overlaps, and the fixed-budget and adaptive
// Tanimoto screens (Eq. expectation, Eq. var, Eq. union-is, Sec.
// confidence-bounded screening).
//
// Work decomposition: one warp owns one work item (a molecule pair, or one
// molecule for volumes) and runs all of its samples; warps take items from a
// device queue (persistent kernel; screens take pairs largest-first). Per
// item and direction the warp stages, in shared memory, the sampled
// molecule's component table (centre, sigma, alias) and both molecules'
// Gaussian coefficients in the frame of the sampled molecule's centroid.
// Each lane then draws SP sample pairs per batch (64 SP samples per warp)
// and evaluates every atom of both molecules: four FP32 FMAs for the
// exponent, one SFU exp2, a packed FP32x2 add for the first-order sum and an
// FMA for the union product. FP32 batch partials (the lane's 2 SP samples) of
// values shifted by a warp-uniform constant are added to FP64 running sums
// per lane, reduced over the warp in FP64; the epilogue runs in FP64.
//
// Launch variants (SP, exponent form, warps per CTA, CTAs per SM) are
// template instances; tanimoto_screen_tune times them and keeps the fastest.
#include <cmath>
#include <mutex>

#include "device.cuh"
#include "internal.h"

namespace shp {
namespace {

// Gaussian coefficients of one atom in the frame of the sampled molecule:
// log2 g(r) = a |r'|^2 + b . r' + c0 with r' = r - o, a = -alpha log2(e),
// b = 2 alpha log2(e) (c - o), c0 = -alpha log2(e) |c - o|^2 + log2 p; every
// scalar is stored twice so the packed form evaluates two samples per
// instruction; om is the control-variate weight of the atom (0 if unused).
struct __align__(16) CoefT {
  float4 ac;   // a, a, c0, c0
  float4 bxy;  // bx, bx, by, by
  float4 bzw;  // bz, bz, om, om
};

// Running per-lane sums of one proposal direction: FP64 sums of the shifted
// values {fa, fa^2, fb, fb^2}, the FP32 partial of the batches not yet added
// to them (a batch's partial covers the lane's 2 SP samples; fixed-budget
// runs add two batches' partials at a time), and the warp-uniform shifts.
struct DirState {
  double s[4];
  float p[4];
  float K[2];
};

struct __align__(16) WarpTables {
  CoefT x[SHP_MAX_ATOMS];      // sampled molecule
  CoefT y[SHP_MAX_ATOMS];      // other molecule
  float4 samp[SHP_MAX_ATOMS];  // sampled molecule: centre - origin, sigma
  uint32_t thr[SHP_MAX_ATOMS];
  uint8_t alias[SHP_MAX_ATOMS];
  DirState st[2][32];          // per-lane running sums of both directions
  float4 origin;               // frame shared by both directions (adaptive screen)
};

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

// log2 g(r) = a |r'|^2 + b . r' + c0 with r' = r - o (expanded form).
__device__ void stage_coef(CoefT* dst, const SetView& S, MolRef M, const Pose& P, float3 o, const float* omega,
                           int lane) {
  const float kLog2e = 1.4426950408889634f;
  for (int i = lane; i < M.n; i += 32) {
    const float4 a = S.atom[M.a0 + i];
    const float lp = S.aux[M.a0 + i].y;
    const float3 c = apply_pose(P, make_float3(a.x, a.y, a.z));
    const float dx = c.x - o.x, dy = c.y - o.y, dz = c.z - o.z;
    const float al = a.w * kLog2e;
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float c0 = fmaf(-al, d2, lp);
    const float bx = 2.f * al * dx, by = 2.f * al * dy, bz = 2.f * al * dz;
    const float om = omega ? omega[M.a0 + i] : 0.f;
    CoefT k;
    k.ac = make_float4(-al, -al, c0, c0);
    k.bxy = make_float4(bx, bx, by, by);
    k.bzw = make_float4(bz, bz, om, om);
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

// Stage one direction: X sampled (its coefficients, centres and alias
// table), Y evaluated, in the frame of X's centroid. Poses (NULL =
// identity) are rebuilt here so no pose is held in registers while sampling.
__device__ __noinline__ void stage_direction(WarpTables& T, const SetView& SX, MolRef MX, const float* pose_x,
                                             const SetView* SY, MolRef MY, const float* pose_y, int lane,
                                             const float* omega_x = nullptr, const float* omega_y = nullptr) {
  const Pose PX = make_pose(pose_x), PY = make_pose(pose_y);
  const float3 o = centroid(SX, MX, PX, lane);
  __syncwarp();
  stage_coef(T.x, SX, MX, PX, o, omega_x, lane);
  if (SY) stage_coef(T.y, *SY, MY, PY, o, omega_y, lane);
  stage_samp(T, SX, MX, PX, o, lane);
  __syncwarp();
}

// Both molecules' coefficient tables (A into x, B into y) in one frame for
// both proposal directions, when their centroids lie within 2 A of each
// other (the frame is then their midpoint, which keeps every sample as close
// to the origin as a per-direction frame would). Returns false, staging
// nothing, otherwise. Later rounds restage only the sampled molecule's
// component table (stage_samp_in_frame).
__device__ __noinline__ bool stage_pair_frame(WarpTables& T, const SetView& SA, MolRef MA, const SetView& SB,
                                              MolRef MB, int lane, const float* omega_a, const float* omega_b) {
  const Pose P = make_pose(nullptr);
  const float3 oa = centroid(SA, MA, P, lane), ob = centroid(SB, MB, P, lane);
  const float dx = oa.x - ob.x, dy = oa.y - ob.y, dz = oa.z - ob.z;
  if (dx * dx + dy * dy + dz * dz > 4.f) return false;
  const float3 o = make_float3(0.5f * (oa.x + ob.x), 0.5f * (oa.y + ob.y), 0.5f * (oa.z + ob.z));
  __syncwarp();
  stage_coef(T.x, SA, MA, P, o, omega_a, lane);
  stage_coef(T.y, SB, MB, P, o, omega_b, lane);
  if (lane == 0) T.origin = make_float4(o.x, o.y, o.z, 0.f);
  __syncwarp();
  return true;
}

__device__ __noinline__ void stage_samp_in_frame(WarpTables& T, const SetView& S, MolRef M, int lane) {
  const float4 o = T.origin;
  __syncwarp();
  stage_samp(T, S, M, make_pose(nullptr), make_float3(o.x, o.y, o.z), lane);
  __syncwarp();
}

// Alias pick: column j = hi32(x n); keep j if lo32(x n) < thr_j. The alias
// is masked to the table size, a no-op for a staged table (alias < n <= 64).
__device__ __forceinline__ int pick(const uint32_t* thr, const uint8_t* alias, int n, uint32_t x) {
  const unsigned long long prod = (unsigned long long)x * (unsigned)n;
  const uint32_t j = (uint32_t)(prod >> 32), f = (uint32_t)prod;
  return f < thr[j] ? (int)j : (int)(alias[j] & (SHP_MAX_ATOMS - 1));
}

// One atom's contribution to m = sum g, q = prod (1 - g) (and with kCV
// ut = sum om g) for SP sample pairs (even sample in .x, odd in .y). kForm 0:
// four scalar FMAs for the exponent; kForm >= 2: four packed FP32x2 FMAs
// (two samples per instruction); kForm >= 5 also updates q with one packed
// FMA per sample pair.
template <int SP, int kForm, bool kCV>
__device__ __forceinline__ void eval_atom(const float4 k0, const float4 k1, const float4 k2, const float2 (&rx)[SP],
                                          const float2 (&ry)[SP], const float2 (&rz)[SP], const float2 (&rr)[SP],
                                          float2 (&m)[SP], float2 (&q)[SP], float2 (&ut)[SP]) {
#pragma unroll
  for (int p = 0; p < SP; ++p) {
    float2 g;
    if (kForm == 0) {
      const float ex = fmaf(k2.x, rz[p].x, fmaf(k1.z, ry[p].x, fmaf(k1.x, rx[p].x, fmaf(k0.x, rr[p].x, k0.z))));
      const float ey = fmaf(k2.x, rz[p].y, fmaf(k1.z, ry[p].y, fmaf(k1.x, rx[p].y, fmaf(k0.x, rr[p].y, k0.z))));
      g = make_float2(ex2_approx(ex), ex2_approx(ey));
    } else {
      float2 e = __ffma2_rn(make_float2(k0.x, k0.y), rr[p], make_float2(k0.z, k0.w));
      e = __ffma2_rn(make_float2(k1.x, k1.y), rx[p], e);
      e = __ffma2_rn(make_float2(k1.z, k1.w), ry[p], e);
      e = __ffma2_rn(make_float2(k2.x, k2.y), rz[p], e);
      g = make_float2(ex2_approx(e.x), ex2_approx(e.y));
    }
    m[p] = __fadd2_rn(m[p], g);
    if (kForm >= 5) {
      q[p] = __ffma2_rn(make_float2(-g.x, -g.y), q[p], q[p]);
    } else {
      q[p].x = fmaf(-g.x, q[p].x, q[p].x);
      q[p].y = fmaf(-g.y, q[p].y, q[p].y);
    }
    if (kCV) ut[p] = __ffma2_rn(make_float2(k2.z, k2.w), g, ut[p]);
  }
}

// m, q (and ut) over one molecule's n >= 1 Gaussians. The atom loop is
// unrolled 2 (forms 0, 2, 6), 1 (forms 3, 5, 7) or 4 (form 4) times; form 7
// loads the next atom's coefficients before evaluating the current one.
template <int SP, int kForm, bool kCV = false>
__device__ __forceinline__ void eval_table(const CoefT* __restrict__ tab, int n, const float2 (&rx)[SP],
                                           const float2 (&ry)[SP], const float2 (&rz)[SP],
                                           const float2 (&rr)[SP], float2 (&m)[SP], float2 (&q)[SP],
                                           float2 (&ut)[SP]) {
  if (kForm == 7) {
    float4 k0 = tab[0].ac, k1 = tab[0].bxy, k2 = tab[0].bzw;
#pragma unroll 1
    for (int j = 0; j < n; ++j) {
      const int jn = j + 1 < n ? j + 1 : j;  // stays inside the staged table
      const float4 n0 = tab[jn].ac, n1 = tab[jn].bxy, n2 = tab[jn].bzw;
      eval_atom<SP, kForm, kCV>(k0, k1, k2, rx, ry, rz, rr, m, q, ut);
      k0 = n0; k1 = n1; k2 = n2;
    }
    return;
  }
  constexpr int kUnroll = (kForm == 3 || kForm == 5) ? 1 : (kForm == 4 ? 4 : 2);
#pragma unroll kUnroll
  for (int j = 0; j < n; ++j) eval_atom<SP, kForm, kCV>(tab[j].ac, tab[j].bxy, tab[j].bzw, rx, ry, rz, rr, m, q, ut);
}

__device__ __forceinline__ void dir_init(DirState& s) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    s.s[t] = 0.0;
    s.p[t] = 0.f;
  }
  s.K[0] = s.K[1] = 0.f;
}

// Draws sample pairs [b * 32 SP, (b + 1) * 32 SP) of one direction from the
// sampled molecule's component table (centres relative to the frame origin,
// sigma, alias): pair s = base + 32 p + lane of this lane goes to slot p,
// even sample in .x, odd sample (or the reflection) in .y; rr = |r|^2.
template <int SP>
__device__ __forceinline__ void draw_batch(const float4* __restrict__ samp, const uint32_t* thr, const uint8_t* alias,
                                           int nx, uint32_t b, Key key, uint32_t slo, uint32_t shi, uint32_t tag,
                                           bool anti, int lane, float2 (&rx)[SP], float2 (&ry)[SP],
                                           float2 (&rz)[SP], float2 (&rr)[SP]) {
  const uint32_t base = b * 32u * SP;
#pragma unroll
  for (int p = 0; p < SP; ++p) {
    const uint32_t s = base + (uint32_t)p * 32u + (uint32_t)lane;
    const uint4 w0 = philox10(make_uint4(2u * s, slo, shi, tag), key);
    const uint4 w1 = philox10(make_uint4(2u * s + 1u, slo, shi, tag), key);
    float n0, n1, n2, n3, n4, n5;
    box_muller(w0.z, w0.w, n0, n1);
    box_muller(w1.x, w1.y, n2, n3);
    box_muller(w1.z, w1.w, n4, n5);
    const float4 c0 = samp[pick(thr, alias, nx, w0.x)];
    const float ax = fmaf(c0.w, n0, c0.x), ay = fmaf(c0.w, n1, c0.y), az = fmaf(c0.w, n4, c0.z);
    float bx, by, bz;
    if (anti) {
      bx = fmaf(-c0.w, n0, c0.x); by = fmaf(-c0.w, n1, c0.y); bz = fmaf(-c0.w, n4, c0.z);
    } else {
      const float4 c1 = samp[pick(thr, alias, nx, w0.y)];
      bx = fmaf(c1.w, n2, c1.x); by = fmaf(c1.w, n3, c1.y); bz = fmaf(c1.w, n5, c1.z);
    }
    rx[p] = make_float2(ax, bx);
    ry[p] = make_float2(ay, by);
    rz[p] = make_float2(az, bz);
    rr[p] = make_float2(fmaf(ax, ax, fmaf(ay, ay, az * az)), fmaf(bx, bx, fmaf(by, by, bz * bz)));
  }
}

// Evaluates and accumulates one batch of drawn sample pairs (P sample pairs
// in total, n samples). Values:
//   cross: fa = m_Y (first order), fb = (u_X / m_X) u_Y (union), with kCV
//          fb = (u_X u_Y - ut_X ut_Y) / m_X (union residual, ut = sum om g)
//   self:  fa = u_X / m_X (volume), with kCV (u_X - ut_X) / m_X,
//          fb = u_X^2 / m_X (self-overlap), with kCV (u_X^2 - ut_X^2) / m_X
// With antithetic pairs the unit is the mean of a sample and its
// reflection. The first batch sets the shifts from sample 0.
// The batch's FP32 partial is added to the FP64 sums when `flush` (with the
// partial carried from an unflushed batch before it), else carried.
template <bool kSelf, int SP, int kForm, bool kCV = false>
__device__ __forceinline__ void eval_batch(const CoefT* __restrict__ tx, const CoefT* __restrict__ ty, int nx,
                                           int ny, uint32_t b, uint32_t n, bool anti, int lane, DirState& st,
                                           const float2 (&rx)[SP], const float2 (&ry)[SP], const float2 (&rz)[SP],
                                           const float2 (&rr)[SP], bool flush = true) {
  const uint32_t P = (n + 1u) >> 1;
  const uint32_t base = b * 32u * SP;
  float2 m[SP], q[SP], ut[SP], fa[SP], fb[SP];
#pragma unroll
  for (int p = 0; p < SP; ++p) {
    m[p] = make_float2(0.f, 0.f);
    q[p] = make_float2(1.f, 1.f);
    ut[p] = make_float2(0.f, 0.f);
  }
  eval_table<SP, kForm, kCV>(tx, nx, rx, ry, rz, rr, m, q, ut);
  if (kSelf) {
    // volume: fa = u/m (or (u - ut)/m with the control variate), self-overlap:
    // fb = u^2/m (or (u^2 - ut^2)/m)
#pragma unroll
    for (int p = 0; p < SP; ++p) {
      const float ux = 1.f - q[p].x, uy = 1.f - q[p].y;
      const float ix = __fdividef(1.f, m[p].x), iy = __fdividef(1.f, m[p].y);
      fa[p] = kCV ? make_float2((ux - ut[p].x) * ix, (uy - ut[p].y) * iy) : make_float2(ux * ix, uy * iy);
      fb[p] = kCV ? make_float2(fmaf(ux, ux, -ut[p].x * ut[p].x) * ix, fmaf(uy, uy, -ut[p].y * ut[p].y) * iy)
                  : make_float2(ux * ux * ix, uy * uy * iy);
    }
  } else {
    float2 w[SP], wt[SP];
#pragma unroll
    for (int p = 0; p < SP; ++p) {
      w[p] = make_float2(__fdividef(1.f - q[p].x, m[p].x), __fdividef(1.f - q[p].y, m[p].y));
      if (kCV) {
        wt[p] = make_float2(__fdividef(ut[p].x, m[p].x), __fdividef(ut[p].y, m[p].y));
        ut[p] = make_float2(0.f, 0.f);
      }
      m[p] = make_float2(0.f, 0.f);
      q[p] = make_float2(1.f, 1.f);
    }
    eval_table<SP, kForm, kCV>(ty, ny, rx, ry, rz, rr, m, q, ut);
#pragma unroll
    for (int p = 0; p < SP; ++p) {
      fa[p] = m[p];
      if (kCV)
        fb[p] = make_float2(fmaf(-wt[p].x, ut[p].x, w[p].x * (1.f - q[p].x)),
                            fmaf(-wt[p].y, ut[p].y, w[p].y * (1.f - q[p].y)));
      else
        fb[p] = make_float2(w[p].x * (1.f - q[p].x), w[p].y * (1.f - q[p].y));
    }
  }
  if (b == 0) {
    // sample 0 (lane 0, pair 0) always exists since n >= 2
    st.K[0] = __shfl_sync(0xffffffffu, anti ? 0.5f * (fa[0].x + fa[0].y) : fa[0].x, 0);
    st.K[1] = __shfl_sync(0xffffffffu, anti ? 0.5f * (fb[0].x + fb[0].y) : fb[0].x, 0);
  }
  const float Ka = st.K[0], Kb = st.K[1];
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  if (!anti && 2u * (base + 32u * SP) <= n) {
    // every sample of the batch exists (all but a ragged last batch): packed
    // sums without the validity masks
    float2 s1 = make_float2(0.f, 0.f), s2 = s1, t1 = s1, t2 = s1;
#pragma unroll
    for (int p = 0; p < SP; ++p) {
      const float2 a = __fadd2_rn(fa[p], make_float2(-Ka, -Ka));
      const float2 c = __fadd2_rn(fb[p], make_float2(-Kb, -Kb));
      s1 = __fadd2_rn(s1, a);
      s2 = __ffma2_rn(a, a, s2);
      t1 = __fadd2_rn(t1, c);
      t2 = __ffma2_rn(c, c, t2);
    }
    acc[0] = s1.x + s1.y;
    acc[1] = s2.x + s2.y;
    acc[2] = t1.x + t1.y;
    acc[3] = t2.x + t2.y;
  } else {
#pragma unroll
  for (int p = 0; p < SP; ++p) {
    const uint32_t s = base + (uint32_t)p * 32u + (uint32_t)lane;
    const float v0 = s < P ? 1.f : 0.f;
    const float v1 = 2u * s + 1u < n ? 1.f : 0.f;  // implies s < P
    if (anti) {
      const float ga = 0.5f * (fa[p].x + fa[p].y) - Ka, gb = 0.5f * (fb[p].x + fb[p].y) - Kb;
      acc[0] = fmaf(v0, ga, acc[0]);
      acc[1] = fmaf(v0 * ga, ga, acc[1]);
      acc[2] = fmaf(v0, gb, acc[2]);
      acc[3] = fmaf(v0 * gb, gb, acc[3]);
    } else {
      const float a0 = fa[p].x - Ka, a1 = fa[p].y - Ka;
      const float b0 = fb[p].x - Kb, b1 = fb[p].y - Kb;
      acc[0] += v0 * a0 + v1 * a1;
      acc[1] += v0 * a0 * a0 + v1 * a1 * a1;
      acc[2] += v0 * b0 + v1 * b1;
      acc[3] += v0 * b0 * b0 + v1 * b1 * b1;
    }
  }
  }
  if (flush) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      st.s[t] += (double)(st.p[t] + acc[t]);
      st.p[t] = 0.f;
    }
  } else {
#pragma unroll
    for (int t = 0; t < 4; ++t) st.p[t] += acc[t];
  }
}

// One batch of one direction (draw, evaluate, accumulate) by a single warp;
// tx/ty are the sampled and the other molecule's coefficient tables (T.x and
// T.y unless given).
template <bool kSelf, int SP, int kForm, bool kCV = false>
__device__ __forceinline__ void run_batch(WarpTables& T, int nx, int ny, uint32_t b, uint32_t n, Key key,
                                          uint32_t slo, uint32_t shi, uint32_t tag, bool anti, int lane,
                                          DirState& st, const CoefT* tx = nullptr, const CoefT* ty = nullptr,
                                          bool flush = true) {
  float2 rx[SP], ry[SP], rz[SP], rr[SP];
  draw_batch<SP>(T.samp, T.thr, T.alias, nx, b, key, slo, shi, tag, anti, lane, rx, ry, rz, rr);
  eval_batch<kSelf, SP, kForm, kCV>(tx ? tx : T.x, ty ? ty : T.y, nx, ny, b, n, anti, lane, st, rx, ry, rz, rr,
                                    flush);
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

// Warp totals of a direction (in every lane): sums[4] in FP64.
__device__ __forceinline__ void dir_totals(const DirState& st, double sums[4]) {
#pragma unroll
  for (int t = 0; t < 4; ++t) sums[t] = warp_sum(st.s[t]);
}

enum Mode { kPairs = 0, kScreen = 1, kAdaptive = 2 };

struct CrossArgs {
  SetView A, B;
  // pair mode
  const int32_t* ia;
  const int32_t* ib;
  const float* pose;
  double* est;
  double* se;
  // screen modes
  const int32_t* order_b;
  const int32_t* list_q;   // explicit pair list (screen modes), or NULL
  const int32_t* list_b;
  int32_t n_q, n_db;
  uint64_t stream_stride;  // pair (q, d) uses stream stream_base + q * stream_stride + d
  const double* self_q;
  const double* self_db;
  const double* self_se_q;   // standard errors of self_q / self_db, or NULL (exact)
  const double* self_se_db;
  float* T;
  float* seT;
  double* O;
  double* seO;
  uint32_t* n_used;
  // control variate of the union slot (screen modes): per-atom weights
  const float* omega_a;
  const float* omega_b;
  // adaptive
  float tau;
  uint32_t round_b, min_b, cap_b;  // in batches
  int watch;
  // common
  int64_t n_items;
  int64_t item_stride;
  int64_t stream_group;  // pair mode: item k uses stream stream_base + k / stream_group
  Key key;
  uint64_t stream_base;
  uint32_t n;
  bool anti, symmetric;
  unsigned long long* queue;
};

// Closed-form integral of the control variate for one pair,
// C = sum_ij om_i om_j integral g_i g_j (Eq. fo with weights): lanes over A's
// atoms, FP32 terms (SFU exp2), FP64 warp sum, valid in every lane.
__device__ double weighted_fo(const SetView& A, MolRef MA, const float* wa, const SetView& B, MolRef MB,
                             const float* wb, int lane) {
  const float kLog2e = 1.4426950408889634f, kPi = 3.14159265358979f;
  float acc = 0.f;
  for (int i = lane; i < MA.n; i += 32) {
    const float4 ai = A.atom[MA.a0 + i];
    const float lpi = A.aux[MA.a0 + i].y, wi = wa[MA.a0 + i];
    for (int j = 0; j < MB.n; ++j) {
      const float4 bj = B.atom[MB.a0 + j];
      const float dx = ai.x - bj.x, dy = ai.y - bj.y, dz = ai.z - bj.z;
      const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      const float inv = 1.0f / (ai.w + bj.w);
      const float t = kPi * inv;
      const float e = fmaf(-kLog2e * ai.w * bj.w * inv, d2, lpi + B.aux[MB.a0 + j].y);
      acc = fmaf(wi * wb[MB.a0 + j] * t * sqrtf(t), ex2_approx(e), acc);
    }
  }
  return warp_sum((double)acc);
}

// Pair epilogue: symmetrised estimates, Tanimoto and SEs; lane 0 only. C is
// the control variate's closed-form part of the union slot (0 without it).
template <int MODE>
__device__ void pair_epilogue(const CrossArgs& args, int32_t xa, int32_t xb, int64_t out_idx, const double s0[4],
                              const float k0[2], const double s1[4], const float k1[2], double n_eff,
                              double C = 0.0) {
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
  e[1] += C;
  if (MODE == kPairs) {
    args.est[2 * out_idx] = e[0]; args.est[2 * out_idx + 1] = e[1];
    args.se[2 * out_idx] = sd[0]; args.se[2 * out_idx + 1] = sd[1];
  } else {
    for (int slot = 0; slot < 2; ++slot) {
      const double S = args.self_q[2 * (int64_t)xa + slot] + args.self_db[2 * (int64_t)xb + slot];
      const double den = S - e[slot];
      args.T[2 * out_idx + slot] = (float)(e[slot] / den);
      // delta method: dT/dO = S / den^2 (the paper's term) and, for
      // estimated self-overlaps, dT/dO_QQ = dT/dO_DD = -O / den^2
      const double dO = S / (den * den);
      double var_t = dO * dO * sd[slot] * sd[slot];
      if (args.self_se_q) {
        const double sq = args.self_se_q[2 * (int64_t)xa + slot], sdb = args.self_se_db[2 * (int64_t)xb + slot];
        const double dS = e[slot] / (den * den);
        var_t += dS * dS * (sq * sq + sdb * sdb);
      }
      args.seT[2 * out_idx + slot] = (float)sqrt(var_t);
      if (args.O) args.O[2 * out_idx + slot] = e[slot];
      if (args.seO) args.seO[2 * out_idx + slot] = sd[slot];
    }
  }
}

// FP32 SE(T) of the watched slot from the running sums (adaptive stop rule),
// with the self-overlaps' own errors when their SEs are given. The lanes'
// FP64 sums are reduced over the warp in FP32: the rule needs no more, and a
// warp-wide FP64 add occupies the SM's FP64 unit ~16 cycles.
__device__ __forceinline__ float watched_se_t(const CrossArgs& args, const DirState& sa, const DirState& sb, int32_t xa,
                                              int32_t xb, float n, float C = 0.f) {
  const bool w = args.watch != 0;
  float h[4] = {(float)(w ? sa.s[2] : sa.s[0]), (float)(w ? sa.s[3] : sa.s[1]), (float)(w ? sb.s[2] : sb.s[0]),
                (float)(w ? sb.s[3] : sb.s[1])};
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = warp_sum(h[i]);
  const float ZA = (float)args.A.Z[xa], ZB = (float)args.B.Z[xb];
  const float s1a = (float)h[0], s2a = (float)h[1], s1b = (float)h[2], s2b = (float)h[3];
  const float va = fmaxf((s2a - s1a * s1a / n) / (n - 1.f), 0.f);
  const float vb = fmaxf((s2b - s1b * s1b / n) / (n - 1.f), 0.f);
  const float ea = ZA * ((w ? sa.K[1] : sa.K[0]) + s1a / n), eb = ZB * ((w ? sb.K[1] : sb.K[0]) + s1b / n);
  const float O = 0.5f * (ea + eb) + (w ? C : 0.f);
  const float seO = 0.5f * sqrtf((ZA * ZA * va + ZB * ZB * vb) / n);
  const float S = (float)(args.self_q[2 * (int64_t)xa + args.watch] + args.self_db[2 * (int64_t)xb + args.watch]);
  const float den = S - O;
  const float dO = S / (den * den);
  float var_t = dO * dO * seO * seO;
  if (args.self_se_q) {
    const float sq = (float)args.self_se_q[2 * (int64_t)xa + args.watch];
    const float sdb = (float)args.self_se_db[2 * (int64_t)xb + args.watch];
    const float dS = O / (den * den);
    var_t = fmaf(dS * dS, fmaf(sq, sq, sdb * sdb), var_t);
  }
  return sqrtf(var_t);
}

// Stages direction dir of a pair (0: A sampled and B evaluated, 1: the
// reverse; the pose, if any, moves B) and runs its batches [b0, b1) into the
// direction's running sums. With a shared frame (both coefficient tables
// already staged, A in x and B in y) only the component table is restaged.
template <int SP, int kForm, bool kCV>
__device__ __forceinline__ void run_direction(WarpTables& T, const CrossArgs& args, int dir, bool shared, MolRef MA,
                                              MolRef MB, const float* pose, const float* wa, const float* wb,
                                              uint32_t b0, uint32_t b1, uint32_t n, bool anti, uint32_t slo,
                                              uint32_t shi, int lane) {
  const SetView& SX = dir ? args.B : args.A;
  const SetView& SY = dir ? args.A : args.B;
  const MolRef MX = dir ? MB : MA, MY = dir ? MA : MB;
  if (shared)
    stage_samp_in_frame(T, SX, MX, lane);
  else
    stage_direction(T, SX, MX, dir ? pose : nullptr, &SY, MY, dir ? nullptr : pose, lane, dir ? wb : wa,
                    dir ? wa : wb);
  const CoefT* tx = (shared && dir) ? T.y : T.x;
  const CoefT* ty = (shared && dir) ? T.x : T.y;
  DirState& st = T.st[dir][lane];
  // batches in twos: the FP64 sums take every second batch's partial (and
  // the last one's); an adaptive round's single batch is always added
  for (uint32_t k = b0; k < b1; ++k)
    run_batch<false, SP, kForm, kCV>(T, MX.n, MY.n, k, n, args.key, slo, shi, dir ? SHP_TAG_BA : SHP_TAG_AB, anti,
                                     lane, st, tx, ty, ((k - b0) & 1u) || k + 1u == b1);
}

// kCV (screen modes): union slot with the weighted-Gaussian control variate.
template <int MODE, int SP, int kForm, int kWarps, int kMinBlocks, bool kCV = false>
__global__ void __launch_bounds__(kWarps * 32, kMinBlocks) cross_kernel(const CrossArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpTables& T = reinterpret_cast<WarpTables*>(smem_raw)[warp];
  const uint32_t batch = 32u * SP;  // sample pairs per batch
  // lane 0 holds the next item, taken from the queue while the current one
  // runs so the atomic's latency is hidden
  unsigned long long next = 0;
  if (lane == 0) next = atomicAdd(args.queue, 1ull);
  for (;;) {
    const unsigned long long item = __shfl_sync(0xffffffffu, next, 0);
    if (item >= (unsigned long long)args.n_items) break;
    if (lane == 0) next = atomicAdd(args.queue, 1ull);
    int32_t xa, xb;
    int64_t out_idx;
    const float* pose = nullptr;
    if (MODE == kPairs) {
      xa = args.ia[item];
      xb = args.ib[item];
      out_idx = (int64_t)item;
      if (args.pose) pose = args.pose + 7 * (int64_t)item;
    } else if (args.list_q) {
      const int64_t t = (int64_t)item * args.item_stride;
      xa = args.list_q[t];
      xb = args.list_b[t];
      out_idx = t;
    } else {
      const int64_t t = (int64_t)item * args.item_stride;
      const int64_t rank = t / args.n_q;
      if (rank >= args.n_db) continue;
      xa = (int32_t)(t - rank * args.n_q);
      xb = args.order_b[rank];
      out_idx = (int64_t)xa * args.n_db + xb;
    }
    if (xa < 0 || xa >= args.A.n_mol || xb < 0 || xb >= args.B.n_mol) {
      if (lane == 0 && MODE == kPairs) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        args.est[2 * out_idx] = nan; args.est[2 * out_idx + 1] = nan;
        args.se[2 * out_idx] = nan; args.se[2 * out_idx + 1] = nan;
      }
      continue;
    }
    const uint64_t sid = args.stream_base + (MODE == kPairs ? (uint64_t)(out_idx / args.stream_group)
                                                            : (uint64_t)xa * args.stream_stride + (uint64_t)xb);
    const uint32_t slo = (uint32_t)sid, shi = (uint32_t)(sid >> 32);
    const MolRef MA = mol_ref(args.A, xa), MB = mol_ref(args.B, xb);
    DirState& sa = T.st[0][lane];
    DirState& sb = T.st[1][lane];
    dir_init(sa);
    dir_init(sb);
    const float* wa = kCV ? args.omega_a : nullptr;
    const float* wb = kCV ? args.omega_b : nullptr;
    const double Ccv = kCV ? weighted_fo(args.A, MA, wa, args.B, MB, wb, lane) : 0.0;
    uint32_t n_dir;
    // one inlined copy of the evaluation serves both directions (a loop, not
    // two copies: the adaptive rounds alternate directions every batch)
    if (MODE != kAdaptive) {
      const uint32_t nb = ((args.n + 1u) / 2u + batch - 1u) / batch;
      // screens (no poses, both directions): one shared frame when possible
      const bool shared = MODE == kScreen && stage_pair_frame(T, args.A, MA, args.B, MB, lane, wa, wb);
      const int ndir = args.symmetric ? 2 : 1;
#pragma unroll 1
      for (int dir = 0; dir < ndir; ++dir)
        run_direction<SP, kForm, kCV>(T, args, dir, shared, MA, MB, pose, wa, wb, 0, nb, args.n, args.anti, slo, shi,
                                      lane);
      n_dir = args.n;
    } else {
      // rounds of round_b batches per direction until SE(T) <= tau or cap;
      // with a shared frame only the sampled molecule's component table is
      // restaged per direction and round
      const bool shared = stage_pair_frame(T, args.A, MA, args.B, MB, lane, wa, wb);
      uint32_t b = 0;
      for (;;) {
        const uint32_t nxt = b + args.round_b;
        const uint32_t n_now = nxt * batch * 2u;
#pragma unroll 1
        for (int dir = 0; dir < 2; ++dir)
          run_direction<SP, kForm, kCV>(T, args, dir, shared, MA, MB, nullptr, wa, wb, b, nxt, n_now, false, slo, shi,
                                        lane);
        b = nxt;
        if (b >= args.cap_b) break;
        if (b >= args.min_b) {
          const float se_t = watched_se_t(args, sa, sb, xa, xb, (float)n_now, (float)Ccv);
          const int stop = __shfl_sync(0xffffffffu, (int)(se_t <= args.tau), 0);
          if (stop) break;
        }
      }
      n_dir = b * batch * 2u;
    }
    double s0[4], s1[4] = {0.0, 0.0, 0.0, 0.0};
    dir_totals(sa, s0);
    if (args.symmetric) dir_totals(sb, s1);
    if (lane == 0) {
      const double n_eff = args.anti ? (double)(n_dir / 2u) : (double)n_dir;
      pair_epilogue<MODE>(args, xa, xb, out_idx, s0, sa.K, s1, sb.K, n_eff, Ccv);
      if (MODE != kPairs && args.n_used) args.n_used[out_idx] = n_dir;
    }
    __syncwarp();
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
  bool by_id;  // stream stream_base + molecule id instead of + item
  double* vol;
  double* vol_se;
  double* self_ov;
  double* self_se;
  unsigned long long* queue;
};

template <int SP, int kForm, int kWarps, int kMinBlocks>
__global__ void __launch_bounds__(kWarps * 32, kMinBlocks) self_kernel(const SelfArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpTables& T = reinterpret_cast<WarpTables*>(smem_raw)[warp];
  const uint32_t batch = 32u * SP;
  unsigned long long next = 0;  // the next item, taken while the current one runs
  if (lane == 0) next = atomicAdd(args.queue, 1ull);
  for (;;) {
    const unsigned long long item = __shfl_sync(0xffffffffu, next, 0);
    if (item >= (unsigned long long)args.n_items) break;
    if (lane == 0) next = atomicAdd(args.queue, 1ull);
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
    const uint64_t stream = args.stream_base + (args.by_id ? (uint64_t)xm : (uint64_t)item);
    stage_direction(T, args.S, M, nullptr, nullptr, M, nullptr, lane);
    DirState& st = T.st[0][lane];
    dir_init(st);
    const uint32_t nb = ((args.n + 1u) / 2u + batch - 1u) / batch;
    for (uint32_t b = 0; b < nb; ++b)
      run_batch<true, SP, kForm>(T, M.n, 0, b, args.n, args.key, (uint32_t)stream, (uint32_t)(stream >> 32),
                                 SHP_TAG_SELF, args.anti, lane, st, nullptr, nullptr, (b & 1u) || b + 1u == nb);
    double s[4];
    dir_totals(st, s);
    if (lane == 0) {
      const double n_eff = args.anti ? (double)(args.n / 2u) : (double)args.n;
      const double Z = args.S.Z[xm];
      double e, sd;
      finish(Z, s[0], s[1], st.K[0], n_eff, e, sd);
      args.vol[item] = e;
      if (args.vol_se) args.vol_se[item] = sd;
      finish(Z, s[2], s[3], st.K[1], n_eff, e, sd);
      if (args.self_ov) args.self_ov[item] = e;
      if (args.self_se) args.self_se[item] = sd;
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------ roofline calibration

struct ProbeArgs {
  SetView A, B;
  int32_t xa, xb;
  uint32_t batches;  // per direction per warp
  int draw;
  Key key;
  double* sink;
};

// Synthetic sample pairs for the calibration without draws: slot p of a lane
// sits at staged component centres k0[p], k1[p] (advanced through the table
// by one per batch) moved by sigma times a warp-uniform offset of the batch:
// the position arithmetic of a drawn sample, without its Philox words, alias
// picks and normals.
template <int SP>
__device__ __forceinline__ void synth_batch(const float4* __restrict__ samp, int nx, uint32_t b, int (&k0)[SP],
                                            int (&k1)[SP], float2 (&rx)[SP], float2 (&ry)[SP], float2 (&rz)[SP],
                                            float2 (&rr)[SP]) {
  const float ox = 0.31f * (float)(b % 13u) - 1.9f, oy = 0.23f * (float)(b % 17u) - 1.8f;
  const float oz = 0.17f * (float)(b % 19u) - 1.5f;
#pragma unroll
  for (int p = 0; p < SP; ++p) {
    k0[p] = k0[p] + 1 < nx ? k0[p] + 1 : 0;
    k1[p] = k1[p] + 1 < nx ? k1[p] + 1 : 0;
    const float4 c0 = samp[k0[p]], c1 = samp[k1[p]];
    const float ax = fmaf(c0.w, ox, c0.x), ay = fmaf(c0.w, oy, c0.y), az = fmaf(c0.w, oz, c0.z);
    const float bx = fmaf(c1.w, oy, c1.x), by = fmaf(c1.w, oz, c1.y), bz = fmaf(c1.w, ox, c1.z);
    rx[p] = make_float2(ax, bx);
    ry[p] = make_float2(ay, by);
    rz[p] = make_float2(az, bz);
    rr[p] = make_float2(fmaf(ax, ax, fmaf(ay, ay, az * az)), fmaf(bx, bx, fmaf(by, by, bz * bz)));
  }
}

// The screen variant's per-sample work on one pair, both directions, a fixed
// number of batches per warp: no queue, no per-pair staging beyond the
// first, no epilogue.
template <int SP, int kForm, int kWarps, int kMinBlocks>
__global__ void __launch_bounds__(kWarps * 32, kMinBlocks) probe_kernel(const ProbeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpTables& T = reinterpret_cast<WarpTables*>(smem_raw)[warp];
  const MolRef MA = mol_ref(a.A, a.xa), MB = mol_ref(a.B, a.xb);
  const uint32_t gw = blockIdx.x * kWarps + warp;  // stream of this warp
  DirState& st = T.st[0][lane];
  double check = 0.0;
#pragma unroll 1
  for (int dir = 0; dir < 2; ++dir) {
    const SetView& SX = dir ? a.B : a.A;
    const SetView& SY = dir ? a.A : a.B;
    const MolRef MX = dir ? MB : MA, MY = dir ? MA : MB;
    stage_direction(T, SX, MX, nullptr, &SY, MY, nullptr, lane);
    dir_init(st);
    const uint32_t n = a.batches * 64u * SP;
    if (a.draw) {
      for (uint32_t b = 0; b < a.batches; ++b)
        run_batch<false, SP, kForm>(T, MX.n, MY.n, b, n, a.key, gw, 0u, (uint32_t)dir, false, lane, st, nullptr,
                                    nullptr, (b & 1u) || b + 1u == a.batches);
    } else {
      int k0[SP], k1[SP];
#pragma unroll
      for (int p = 0; p < SP; ++p) {
        k0[p] = (lane + 32 * p) % MX.n;
        k1[p] = (lane + 32 * p + 7) % MX.n;
      }
      for (uint32_t b = 0; b < a.batches; ++b) {
        float2 rx[SP], ry[SP], rz[SP], rr[SP];
        synth_batch<SP>(T.samp, MX.n, b, k0, k1, rx, ry, rz, rr);
        eval_batch<false, SP, kForm>(T.x, T.y, MX.n, MY.n, b, n, false, lane, st, rx, ry, rz, rr,
                                     (b & 1u) || b + 1u == a.batches);
      }
    }
    double sums[4];
    dir_totals(st, sums);
    check += sums[0] + sums[2];
    __syncwarp();
  }
  if (lane == 0) atomicAdd(a.sink, check);
}

// ------------------------------------------------------------ variants

// sample pairs per lane, exponent form, warps per CTA, CTAs per SM (the
// register budget follows: 2 x 8 or 4 x 4 warps -> 128, 5 x 4 -> 102; shared
// memory, about 10 KB per warp, caps an SM at 20 warps)
struct Variant {
  int sp, form, warps, min_blocks;
};
constexpr Variant kVariants[] = {{4, 0, 8, 2}, {4, 2, 8, 2}, {4, 0, 4, 5}, {4, 2, 4, 5}, {4, 3, 8, 2},
                                 {4, 4, 8, 2}, {8, 0, 4, 4}, {8, 2, 4, 4}, {4, 5, 8, 2}, {4, 6, 8, 2},
                                 {4, 7, 8, 2}, {4, 5, 4, 5}, {2, 5, 4, 5}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

// Variants also built with the control variate of the union slot (one more
// FMA per evaluation, packed over the sample pair, and two more values per
// sample pair in registers).
constexpr bool cv_variant(int v) {
  return kVariants[v].sp == 4 && kVariants[v].warps == 8 && kVariants[v].min_blocks == 2 &&
         (kVariants[v].form == 2 || kVariants[v].form == 3 || kVariants[v].form == 4 || kVariants[v].form == 5);
}

template <int V>
struct VariantTraits {
  static constexpr int sp = kVariants[V].sp, form = kVariants[V].form, warps = kVariants[V].warps;
  static constexpr int min_blocks = kVariants[V].min_blocks;
  static constexpr size_t smem = sizeof(WarpTables) * warps;
};

int sm_count(int* sms) {
  int dev = 0;
  SHP_CUDA(cudaGetDevice(&dev));
  SHP_CUDA(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
  return SHP_OK;
}

// Persistent launch: as many CTAs of `warps` warps as fit on the GPU (at
// most one per `warps` items), pulling items from a zeroed device queue
// counter (stream-ordered scratch unless given).
template <class Kernel, class Args>
int launch_persistent(Kernel k, Args args, int64_t n_items, int warps, size_t smem, cudaStream_t st,
                      unsigned long long* queue_in = nullptr) {
  int sms = 0;
  int rc = sm_count(&sms);
  if (rc) return rc;
  SHP_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SHP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, warps * 32, smem));
  if (per_sm < 1) per_sm = 1;
  const int64_t need = (n_items + warps - 1) / warps;
  int64_t g = (int64_t)sms * per_sm;
  if (need < g) g = need;
  const int grid = (int)(g < 1 ? 1 : g);
  unsigned long long* q = queue_in;
  if (!q) SHP_CUDA(dev_alloc((void**)&q, sizeof(unsigned long long), st));
  cudaError_t e = cudaMemsetAsync(q, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    args.queue = q;
    k<<<grid, warps * 32, smem, st>>>(args);
    e = cudaGetLastError();
  }
  cudaError_t e2 = queue_in ? cudaSuccess : cudaFreeAsync(q, st);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
  return SHP_OK;
}

template <int MODE, int V, bool kCV>
int launch_cross_v(const CrossArgs& a, int64_t n_items, cudaStream_t st) {
  using Tr = VariantTraits<V>;
  if constexpr (MODE == kAdaptive && Tr::sp != 4) {
    set_error("adaptive screen: launch variant %d does not run rounds of 256 samples", V);
    return SHP_EINVAL;
  } else if constexpr (kCV && (MODE == kPairs || !cv_variant(V))) {
    set_error("screen with control variate: launch variant %d is not built with it", V);
    return SHP_EINVAL;
  } else {
    return launch_persistent(cross_kernel<MODE, Tr::sp, Tr::form, Tr::warps, Tr::min_blocks, kCV>, a, n_items,
                             Tr::warps, Tr::smem, st);
  }
}

template <int MODE, bool kCV = false, int V = 0>
int launch_cross(int v, const CrossArgs& a, int64_t n_items, cudaStream_t st) {
  if constexpr (V + 1 < kNumVariants) {
    return v == V ? launch_cross_v<MODE, V, kCV>(a, n_items, st) : launch_cross<MODE, kCV, V + 1>(v, a, n_items, st);
  } else {
    return launch_cross_v<MODE, V, kCV>(a, n_items, st);
  }
}

template <int V>
int launch_probe_v(const ProbeArgs& a, cudaStream_t st, int64_t* warps) {
  using Tr = VariantTraits<V>;
  auto k = probe_kernel<Tr::sp, Tr::form, Tr::warps, Tr::min_blocks>;
  int sms = 0;
  int rc = sm_count(&sms);
  if (rc) return rc;
  SHP_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Tr::smem));
  int per_sm = 0;
  SHP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, Tr::warps * 32, Tr::smem));
  if (per_sm < 1) per_sm = 1;
  *warps = (int64_t)sms * per_sm * Tr::warps;
  k<<<sms * per_sm, Tr::warps * 32, Tr::smem, st>>>(a);
  SHP_CUDA(cudaGetLastError());
  return SHP_OK;
}

template <int V = 0>
int launch_probe(int v, const ProbeArgs& a, cudaStream_t st, int64_t* warps) {
  if constexpr (V + 1 < kNumVariants) {
    return v == V ? launch_probe_v<V>(a, st, warps) : launch_probe<V + 1>(v, a, st, warps);
  } else {
    return launch_probe_v<V>(a, st, warps);
  }
}

int launch_self(const SelfArgs& a, int64_t n_items, cudaStream_t st) {
  using Tr = VariantTraits<5>;  // packed exponent, atom loop unrolled 4, 4 sample pairs per lane, 8 warps x 2 CTAs
                                // (6% ahead of the loop unrolled 2 on 100k molecules of 18-60 atoms)
  return launch_persistent(self_kernel<Tr::sp, Tr::form, Tr::warps, Tr::min_blocks>, a, n_items, Tr::warps,
                           Tr::smem, st);
}

// Tuned defaults per (device, mode, control variate); -1 = not tuned, then
// variant 4 (4 sample pairs per lane, packed exponent, valid everywhere).
constexpr int kDefaultVariant = 4;
std::mutex g_tune_mu;
int g_tuned[64][3][2];
bool g_tuned_init = false;

int default_variant(int mode, bool cv = false) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (!g_tuned_init) {
    for (auto& dev : g_tuned)
      for (auto& row : dev) row[0] = row[1] = -1;
    g_tuned_init = true;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  const int v = (dev >= 0 && dev < 64) ? g_tuned[dev][mode][cv] : -1;
  return v >= 0 ? v : kDefaultVariant;
}

void set_default_variant(int mode, bool cv, int v) {
  default_variant(mode, cv);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64) g_tuned[dev][mode][cv] = v;
}

bool variant_valid(int mode, bool cv, int v) {
  if (v < 0 || v >= kNumVariants) return false;
  if (cv && !cv_variant(v)) return false;
  return mode != kAdaptive || kVariants[v].sp == 4;
}

static_assert(cv_variant(kDefaultVariant), "the default variant must be built with the control variate");

int check_mc(const shp_mc* mc, const char* who, uint32_t allowed = SHP_SYMMETRIC | SHP_ANTITHETIC) {
  if (!mc) { set_error("%s: NULL shp_mc", who); return SHP_EINVAL; }
  if (mc->n_samples < 2) { set_error("%s: n_samples must be >= 2", who); return SHP_EINVAL; }
  if ((mc->flags & SHP_ANTITHETIC) && (mc->n_samples & 1u)) {
    set_error("%s: antithetic sampling needs an even n_samples", who);
    return SHP_EINVAL;
  }
  if (mc->flags & ~allowed) { set_error("%s: unknown flags", who); return SHP_EINVAL; }
  return SHP_OK;
}

// Validates a screen config and fills the mode-specific arguments.
int screen_args(shp_set Q, shp_set D, const shp_screen* cfg, const double* self_q, const double* self_db, float* T,
                float* seT, double* O, double* seO, uint32_t* n_used, CrossArgs& a, int& mode, const char* who) {
  if (!Q || !D || !cfg) { set_error("%s: NULL set or config", who); return SHP_EINVAL; }
  if (cfg->flags & ~SHP_ANTITHETIC) { set_error("%s: unknown flags", who); return SHP_EINVAL; }
  a = CrossArgs{};
  if (cfg->n_fixed > 0) {
    mode = kScreen;
    if (cfg->n_fixed < 2) { set_error("%s: n_fixed must be >= 2", who); return SHP_EINVAL; }
    if ((cfg->flags & SHP_ANTITHETIC) && (cfg->n_fixed & 1u)) {
      set_error("%s: antithetic sampling needs an even n_fixed", who);
      return SHP_EINVAL;
    }
    a.n = cfg->n_fixed;
  } else {
    mode = kAdaptive;
    if (cfg->flags & SHP_ANTITHETIC) { set_error("%s: adaptive screens do not take SHP_ANTITHETIC", who); return SHP_EINVAL; }
    const uint32_t bs = 256;  // samples per direction per batch of the SP 4 variants
    if (cfg->round == 0 || cfg->round % bs || cfg->min_n < cfg->round || cfg->min_n % cfg->round ||
        cfg->cap < cfg->min_n || cfg->cap % cfg->round) {
      set_error("%s: adaptive round/min_n/cap must be multiples of 256 with round <= min_n <= cap", who);
      return SHP_EINVAL;
    }
    if (!(cfg->tau > 0.f) || cfg->watch > 1) { set_error("%s: tau must be > 0 and watch 0 or 1", who); return SHP_EINVAL; }
    a.round_b = cfg->round / bs;
    a.min_b = cfg->min_n / bs;
    a.cap_b = cfg->cap / bs;
    a.tau = cfg->tau;
    a.watch = (int)cfg->watch;
  }
  if (Q->n_mol > 0 && D->n_mol > 0 && (!self_q || !self_db || !T || !seT)) {
    set_error("%s: NULL array", who);
    return SHP_EINVAL;
  }
  a.A = view(Q);
  a.B = view(D);
  a.order_b = D->order;
  a.n_q = Q->n_mol;
  a.n_db = D->n_mol;
  a.self_q = self_q;
  a.self_db = self_db;
  a.T = T;
  a.seT = seT;
  a.O = O;
  a.seO = seO;
  a.n_used = n_used;
  a.n_items = (int64_t)Q->n_mol * D->n_mol;
  a.item_stride = 1;
  a.key = Key{(uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32)};
  a.stream_base = cfg->stream_base;
  a.stream_stride = cfg->stream_stride ? cfg->stream_stride : (uint64_t)D->n_mol;
  a.anti = (cfg->flags & SHP_ANTITHETIC) != 0;
  a.symmetric = true;
  if ((cfg->omega_q == nullptr) != (cfg->omega_db == nullptr)) {
    set_error("%s: give both control-variate weight arrays or neither", who);
    return SHP_EINVAL;
  }
  a.omega_a = cfg->omega_q;
  a.omega_b = cfg->omega_db;
  if ((cfg->self_se_q == nullptr) != (cfg->self_se_db == nullptr)) {
    set_error("%s: give both self-overlap SE arrays or neither", who);
    return SHP_EINVAL;
  }
  a.self_se_q = cfg->self_se_q;
  a.self_se_db = cfg->self_se_db;
  if ((cfg->pairs_q == nullptr) != (cfg->pairs_db == nullptr) || cfg->n_pairs < 0 ||
      (cfg->pairs_q == nullptr && cfg->n_pairs != 0)) {
    set_error("%s: give both pair-list arrays with n_pairs >= 0, or neither (n_pairs 0)", who);
    return SHP_EINVAL;
  }
  if (cfg->pairs_q) {
    a.list_q = cfg->pairs_q;
    a.list_b = cfg->pairs_db;
    a.n_items = cfg->n_pairs;
  }
  return SHP_OK;
}

int launch_screen(int mode, int v, const CrossArgs& a, int64_t n_items, cudaStream_t st) {
  if (a.omega_a)
    return mode == kScreen ? launch_cross<kScreen, true>(v, a, n_items, st)
                           : launch_cross<kAdaptive, true>(v, a, n_items, st);
  return mode == kScreen ? launch_cross<kScreen>(v, a, n_items, st) : launch_cross<kAdaptive>(v, a, n_items, st);
}

}  // namespace
}  // namespace shp

using namespace shp;

namespace shp {

int overlap_estimate_grouped(shp_set A, const int32_t* ia, shp_set B, const int32_t* ib, int64_t n_pairs,
                             const float* poseB, const shp_mc* mc, double* est, double* se, int64_t group,
                             cudaStream_t stream) {
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
  a.item_stride = 1;
  a.stream_group = group < 1 ? 1 : group;
  a.key = Key{(uint32_t)mc->seed, (uint32_t)(mc->seed >> 32)};
  a.stream_base = mc->stream_base;
  a.n = mc->n_samples;
  a.anti = (mc->flags & SHP_ANTITHETIC) != 0;
  a.symmetric = (mc->flags & SHP_SYMMETRIC) != 0;
  return launch_cross<kPairs>(default_variant(kPairs), a, n_pairs, stream);
}

}  // namespace shp

extern "C" int overlap_estimate(shp_set A, const int32_t* ia, shp_set B, const int32_t* ib, int64_t n_pairs,
                                const float* poseB, const shp_mc* mc, double* est, double* se, void* stream) {
  clear_error();
  return overlap_estimate_grouped(A, ia, B, ib, n_pairs, poseB, mc, est, se, 1, (cudaStream_t)stream);
}

extern "C" int union_volume_estimate(shp_set S, const int32_t* idx, int64_t n, const shp_mc* mc, double* vol,
                                     double* vol_se, double* self_ov, double* self_se, void* stream) {
  clear_error();
  if (!S) { set_error("union_volume_estimate: NULL set"); return SHP_EINVAL; }
  int rc = check_mc(mc, "union_volume_estimate", SHP_SYMMETRIC | SHP_ANTITHETIC | SHP_ID_STREAMS);
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
  a.by_id = idx && (mc->flags & SHP_ID_STREAMS);
  a.vol = vol;
  a.vol_se = vol_se;
  a.self_ov = self_ov;
  a.self_se = self_se;
  return launch_self(a, n, (cudaStream_t)stream);
}

extern "C" int tanimoto_screen(shp_set Q, shp_set D, const shp_screen* cfg, const double* self_q,
                               const double* self_db, float* T, float* seT, double* O_out, double* seO_out,
                               uint32_t* n_used, void* stream) {
  clear_error();
  CrossArgs a;
  int mode = 0;
  int rc = screen_args(Q, D, cfg, self_q, self_db, T, seT, O_out, seO_out, n_used, a, mode, "tanimoto_screen");
  if (rc) return rc;
  if (a.n_items == 0) return SHP_OK;
  int v = cfg->variant;
  const bool cv = a.omega_a != nullptr;
  if (v < 0) v = default_variant(mode, cv);
  if (!variant_valid(mode, cv, v)) { set_error("tanimoto_screen: variant %d not valid for this mode", v); return SHP_EINVAL; }
  return launch_screen(mode, v, a, a.n_items, (cudaStream_t)stream);
}

extern "C" int shp_screen_variants(void) { return kNumVariants; }

extern "C" int shp_screen_variant_info(int32_t v, int32_t info[4]) {
  clear_error();
  if (!info) { set_error("shp_screen_variant_info: NULL info"); return SHP_EINVAL; }
  if (v < 0 || v >= kNumVariants) { set_error("shp_screen_variant_info: no variant %d", v); return SHP_ERANGE; }
  info[0] = kVariants[v].sp;
  info[1] = kVariants[v].form;
  info[2] = kVariants[v].warps;
  info[3] = kVariants[v].min_blocks;
  return SHP_OK;
}

extern "C" int tanimoto_screen_tune(shp_set Q, shp_set D, const shp_screen* cfg, const double* self_q,
                                    const double* self_db, float* T, float* seT, uint32_t* n_used, int64_t n_sample,
                                    float* timings_ms, int32_t* best, void* stream) {
  clear_error();
  CrossArgs a;
  int mode = 0;
  int rc = screen_args(Q, D, cfg, self_q, self_db, T, seT, nullptr, nullptr, n_used, a, mode, "tanimoto_screen_tune");
  if (rc) return rc;
  if (a.n_items == 0 || n_sample <= 0) { set_error("tanimoto_screen_tune: nothing to time"); return SHP_EINVAL; }
  if (n_sample > a.n_items) n_sample = a.n_items;
  a.item_stride = a.n_items / n_sample;
  a.n_items = n_sample;  // the kernel visits items 0 .. n_sample-1, pair = item * stride
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  SHP_CUDA(cudaEventCreate(&e0));
  SHP_CUDA(cudaEventCreate(&e1));
  int best_v = -1;
  float best_ms = 0.f;
  for (int v = 0; v < kNumVariants; ++v) {
    if (timings_ms) timings_ms[v] = -1.f;
    if (!variant_valid(mode, a.omega_a != nullptr, v)) continue;
    rc = launch_screen(mode, v, a, n_sample, st);  // warm-up (first launch pays set-up)
    if (!rc) {
      cudaEventRecord(e0, st);
      rc = launch_screen(mode, v, a, n_sample, st);
      cudaEventRecord(e1, st);
    }
    if (rc) break;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) { rc = cuda_fail(e, "tanimoto_screen_tune: cudaEventSynchronize"); break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (timings_ms) timings_ms[v] = ms;
    if (best_v < 0 || ms < best_ms) { best_v = v; best_ms = ms; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  set_default_variant(mode, a.omega_a != nullptr, best_v);
  if (best) *best = best_v;
  return SHP_OK;
}

// ------------------------------------------------------------------------
// Learned control variate for the union volume
// ------------------------------------------------------------------------
namespace shp {
namespace {

constexpr int kCVWarps = 8;

struct AttrArgs {
  SetView S;
  Key key;
  uint64_t stream_base;
  uint32_t M;  // samples per atom, a multiple of 256
  float* omega;
  unsigned long long* queue;
};

// omega*_i = E_{N(c_i, I/(2 alpha_i))}[u/m]: atom i of molecule k uses sample
// pairs i M/2 .. (i+1) M/2 - 1 of stream stream_base + k, tag 5 (normals only).
__global__ void __launch_bounds__(kCVWarps * 32, 2) attribution_kernel(const AttrArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpTables& T = reinterpret_cast<WarpTables*>(smem_raw)[warp];
  constexpr int SP = 4;
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(a.queue, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= (unsigned long long)a.S.n_mol) break;
    const MolRef M = mol_ref(a.S, (int32_t)item);
    stage_direction(T, a.S, M, nullptr, nullptr, M, nullptr, lane);
    const uint64_t stream = a.stream_base + item;
    const uint32_t slo = (uint32_t)stream, shi = (uint32_t)(stream >> 32);
    for (int i = 0; i < M.n; ++i) {
      const float4 ci = T.samp[i];
      float acc = 0.f;
      for (uint32_t b = 0; b < a.M / 256u; ++b) {
        float2 rx[SP], ry[SP], rz[SP], rr[SP], m[SP], q[SP], ut[SP];
#pragma unroll
        for (int p = 0; p < SP; ++p) {
          const uint32_t s = (uint32_t)i * (a.M / 2u) + b * 128u + (uint32_t)p * 32u + (uint32_t)lane;
          const uint4 w0 = philox10(make_uint4(2u * s, slo, shi, SHP_TAG_ATTR), a.key);
          const uint4 w1 = philox10(make_uint4(2u * s + 1u, slo, shi, SHP_TAG_ATTR), a.key);
          float n0, n1, n2, n3, n4, n5;
          box_muller(w0.z, w0.w, n0, n1);
          box_muller(w1.x, w1.y, n2, n3);
          box_muller(w1.z, w1.w, n4, n5);
          const float ax = fmaf(ci.w, n0, ci.x), ay = fmaf(ci.w, n1, ci.y), az = fmaf(ci.w, n4, ci.z);
          const float bx = fmaf(ci.w, n2, ci.x), by = fmaf(ci.w, n3, ci.y), bz = fmaf(ci.w, n5, ci.z);
          rx[p] = make_float2(ax, bx);
          ry[p] = make_float2(ay, by);
          rz[p] = make_float2(az, bz);
          rr[p] = make_float2(fmaf(ax, ax, fmaf(ay, ay, az * az)), fmaf(bx, bx, fmaf(by, by, bz * bz)));
          m[p] = make_float2(0.f, 0.f);
          q[p] = make_float2(1.f, 1.f);
        }
        eval_table<SP, 0, false>(T.x, M.n, rx, ry, rz, rr, m, q, ut);
#pragma unroll
        for (int p = 0; p < SP; ++p)
          acc += __fdividef(1.f - q[p].x, m[p].x) + __fdividef(1.f - q[p].y, m[p].y);
      }
      acc = warp_sum(acc);
      if (lane == 0) a.omega[M.a0 + i] = acc / (float)a.M;
    }
    __syncwarp();
  }
}

struct CVArgs {
  SetView S;
  const int32_t* idx;
  const float* omega;  // per set atom, or NULL (plain estimator)
  int64_t n_items;
  Key key;
  uint64_t stream_base;
  uint32_t n;          // fixed budget (samples), or the cap when adaptive
  float target;        // > 0: stop once SE / estimate <= target for the watched
                       // estimand (checked every round_b batches)
  uint32_t round_b;
  int watch;           // 0: volume, 1: self-overlap
  bool by_id;          // stream stream_base + molecule id instead of + item
  double* vol;
  double* vol_se;
  double* self_ov;
  double* self_se;
  uint32_t* n_used;
  unsigned long long* queue;
};

// Union volume and union self-overlap, optionally with the weighted-Gaussian
// control variate ut = sum_i om_i g_i:
//   V    = sum_i om_i v_i                   + Z mean((u - ut) / m)
//   O_XX = sum_ij om_i om_j integral g_i g_j + Z mean((u^2 - ut^2) / m)
// same samples as union_volume_estimate; fixed budget or rounds until the
// watched estimate reaches a relative SE.
template <bool kCV>
__global__ void __launch_bounds__(kCVWarps * 32, 2) cv_volume_kernel(const CVArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpTables& T = reinterpret_cast<WarpTables*>(smem_raw)[warp];
  constexpr int SP = 4;
  const uint32_t batch = 32u * SP;
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(a.queue, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= (unsigned long long)a.n_items) break;
    const int32_t xm = a.idx ? a.idx[item] : (int32_t)item;
    if (xm < 0 || xm >= a.S.n_mol) {
      if (lane == 0) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        if (a.vol) a.vol[item] = nan;
        if (a.vol_se) a.vol_se[item] = nan;
        if (a.self_ov) a.self_ov[item] = nan;
        if (a.self_se) a.self_se[item] = nan;
        if (a.n_used) a.n_used[item] = 0;
      }
      continue;
    }
    const MolRef M = mol_ref(a.S, xm);
    stage_direction(T, a.S, M, nullptr, nullptr, M, nullptr, lane, kCV ? a.omega : nullptr);
    // closed-form parts: sum_i om_i v_i, v_i = p_i (pi / alpha_i)^{3/2}, in
    // FP64, and sum_ij om_i om_j integral g_i g_j (Eq. fo with weights)
    double closed = 0.0, closed_s = 0.0;
    if (kCV) {
      for (int i = lane; i < M.n; i += 32) {
        const double t = 3.141592653589793 / (double)a.S.atom[M.a0 + i].w;
        closed += (double)a.omega[M.a0 + i] * exp2((double)a.S.aux[M.a0 + i].y) * t * sqrt(t);
      }
      closed = warp_sum(closed);
      closed_s = weighted_fo(a.S, M, a.omega, a.S, M, a.omega, lane);
    }
    const double Z = a.S.Z[xm];
    DirState& st = T.st[0][lane];
    dir_init(st);
    const uint64_t stream = a.stream_base + (a.by_id ? (uint64_t)xm : (uint64_t)item);
    const uint32_t slo = (uint32_t)stream, shi = (uint32_t)(stream >> 32);
    uint32_t n_done;
    if (a.target <= 0.f) {
      const uint32_t nb = ((a.n + 1u) / 2u + batch - 1u) / batch;
      for (uint32_t b = 0; b < nb; ++b)
        run_batch<true, SP, 2, kCV>(T, M.n, 0, b, a.n, a.key, slo, shi, SHP_TAG_SELF, false, lane, st, nullptr,
                                    nullptr, (b & 1u) || b + 1u == nb);
      n_done = a.n;
    } else {
      const uint32_t cap_b = a.n / (2u * batch);
      uint32_t b = 0;
      for (;;) {
        const uint32_t nxt = b + a.round_b;
        const uint32_t n_now = nxt * batch * 2u;
        for (uint32_t k = b; k < nxt; ++k)
          run_batch<true, SP, 2, kCV>(T, M.n, 0, k, n_now, a.key, slo, shi, SHP_TAG_SELF, false, lane, st, nullptr,
                                      nullptr, ((k - b) & 1u) || k + 1u == nxt);
        b = nxt;
        if (b >= cap_b) break;
        const int w = a.watch;
        // the stop rule in FP32 (the lanes' FP64 sums reduced in FP32)
        const float nf = (float)n_now, s1 = warp_sum((float)st.s[2 * w]), s2 = warp_sum((float)st.s[2 * w + 1]);
        const float var = fmaxf((s2 - s1 * s1 / nf) / (nf - 1.f), 0.f);
        const float V = (float)(w ? closed_s : closed) + (float)Z * (st.K[w] + s1 / nf);
        const float se = (float)Z * sqrtf(var / nf);
        const int stop = __shfl_sync(0xffffffffu, (int)(se <= a.target * fabsf(V)), 0);
        if (stop) break;
      }
      n_done = b * batch * 2u;
    }
    double s[4];
    dir_totals(st, s);
    if (lane == 0) {
      double e, sd;
      finish(Z, s[0], s[1], st.K[0], (double)n_done, e, sd);
      if (a.vol) a.vol[item] = closed + e;
      if (a.vol_se) a.vol_se[item] = sd;
      finish(Z, s[2], s[3], st.K[1], (double)n_done, e, sd);
      if (a.self_ov) a.self_ov[item] = closed_s + e;
      if (a.self_se) a.self_se[item] = sd;
      if (a.n_used) a.n_used[item] = n_done;
    }
    __syncwarp();
  }
}

struct FitArgs {
  SetView S;
  const int32_t* idx;
  int64_t n_items;
  Key key;
  uint64_t stream_base;
  uint32_t nb;    // batches of 256 samples per molecule
  float ridge;
  float* omega;
  bool by_id;     // stream stream_base + molecule id instead of + item
  unsigned long long* queue;
};

// Closed-form overlap integral of two atomic Gaussians (Eq. fo term), FP32.
__device__ __forceinline__ float gauss_overlap(float4 ci, float lpi, float4 cj, float lpj) {
  const float kLog2e = 1.4426950408889634f, kPi = 3.14159265358979f;
  const float dx = ci.x - cj.x, dy = ci.y - cj.y, dz = ci.z - cj.z;
  const float inv = 1.0f / (ci.w + cj.w);
  const float t = kPi * inv;
  const float aa = ci.w * cj.w;  // every operation is symmetric in (i, j): G_ij == G_ji bit for bit
  return t * sqrtf(t) * ex2_approx(fmaf(-kLog2e * aa * inv, fmaf(dx, dx, fmaf(dy, dy, dz * dz)), lpi + lpj));
}

// Least-squares control-variate weights, one warp per molecule: the
// projection of u onto the molecule's own Gaussians, (G + lambda I) w = b
// with b_j = Z E_q[(u/m) g_j] from nb batches of the molecule's own samples
// (tag 6) and G_ij the closed-form overlaps, solved by conjugate gradients
// (lanes own rows j and j + 32; G's lower triangle, N (N + 1) / 2 floats, is
// formed once into the warp's staging tables, free after the sampling; at
// most 4 N iterations, stopping at a relative residual of
// 1e-6).
__global__ void __launch_bounds__(kCVWarps * 32, 2) cv_fit_kernel(const FitArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float s_b[kCVWarps][SHP_MAX_ATOMS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpTables& T = reinterpret_cast<WarpTables*>(smem_raw)[warp];
  float* bsum = s_b[warp];
  constexpr int SP = 4;
  unsigned long long next = 0;
  if (lane == 0) next = atomicAdd(a.queue, 1ull);
  for (;;) {
    const unsigned long long item = __shfl_sync(0xffffffffu, next, 0);
    if (item >= (unsigned long long)a.n_items) break;
    if (lane == 0) next = atomicAdd(a.queue, 1ull);
    const int32_t xm = a.idx ? a.idx[item] : (int32_t)item;
    if (xm < 0 || xm >= a.S.n_mol) continue;  // an id outside the set has no atoms to write
    const MolRef M = mol_ref(a.S, xm);
    const uint64_t stream = a.stream_base + (a.by_id ? (uint64_t)xm : (uint64_t)item);
    stage_direction(T, a.S, M, nullptr, nullptr, M, nullptr, lane);
    for (int j = lane; j < SHP_MAX_ATOMS; j += 32) bsum[j] = 0.f;
    __syncwarp();
    for (uint32_t bt = 0; bt < a.nb; ++bt) {
      float2 rx[SP], ry[SP], rz[SP], rr[SP], m[SP], q[SP], ut[SP], w[SP];
      draw_batch<SP>(T.samp, T.thr, T.alias, M.n, bt, a.key, (uint32_t)stream, (uint32_t)(stream >> 32), SHP_TAG_FIT,
                     false, lane, rx, ry, rz, rr);
#pragma unroll
      for (int p = 0; p < SP; ++p) {
        m[p] = make_float2(0.f, 0.f);
        q[p] = make_float2(1.f, 1.f);
      }
      eval_table<SP, 5, false>(T.x, M.n, rx, ry, rz, rr, m, q, ut);
#pragma unroll
      for (int p = 0; p < SP; ++p)
        w[p] = make_float2(__fdividef(1.f - q[p].x, m[p].x), __fdividef(1.f - q[p].y, m[p].y));
      // b_j += sum over the batch of (u/m) g_j, g_j from the same packed expression
#pragma unroll 1
      for (int j = 0; j < M.n; ++j) {
        const float4 k0 = T.x[j].ac, k1 = T.x[j].bxy, k2 = T.x[j].bzw;
        float c = 0.f;
#pragma unroll
        for (int p = 0; p < SP; ++p) {
          float2 e = __ffma2_rn(make_float2(k0.x, k0.y), rr[p], make_float2(k0.z, k0.w));
          e = __ffma2_rn(make_float2(k1.x, k1.y), rx[p], e);
          e = __ffma2_rn(make_float2(k1.z, k1.w), ry[p], e);
          e = __ffma2_rn(make_float2(k2.x, k2.y), rz[p], e);
          c = fmaf(w[p].x, ex2_approx(e.x), fmaf(w[p].y, ex2_approx(e.y), c));
        }
        c = warp_sum(c);
        if (lane == 0) bsum[j] += c;
      }
    }
    __syncwarp();
    // conjugate gradients on (G + lambda I) x = b; lane owns rows i0, i1
    const int N = M.n;
    const int i0 = lane, i1 = lane + 32;
    const bool h0 = i0 < N, h1 = i1 < N;
    const float scale = (float)(a.S.Z[xm] / (256.0 * a.nb));
    const float4 c0 = h0 ? a.S.atom[M.a0 + i0] : make_float4(0.f, 0.f, 0.f, 1.f);
    const float4 c1 = h1 ? a.S.atom[M.a0 + i1] : make_float4(0.f, 0.f, 0.f, 1.f);
    const float l0 = h0 ? a.S.aux[M.a0 + i0].y : 0.f, l1 = h1 ? a.S.aux[M.a0 + i1].y : 0.f;
    const float trace =
        warp_sum((h0 ? gauss_overlap(c0, l0, c0, l0) : 0.f) + (h1 ? gauss_overlap(c1, l1, c1, l1) : 0.f));
    const float lambda = a.ridge * trace / (float)N;
    // G's lower triangle, G_ij at i (i + 1) / 2 + j for j <= i, in the staging
    // tables (the sampling is done with them)
    float* G = reinterpret_cast<float*>(&T);
    static_assert(sizeof(WarpTables) >= sizeof(float) * SHP_MAX_ATOMS * (SHP_MAX_ATOMS + 1) / 2,
                  "the Gram triangle must fit the staging tables");
    __syncwarp();
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
      const float4 ci = a.S.atom[M.a0 + i];
      const float li = a.S.aux[M.a0 + i].y;
      for (int j = lane; j <= i; j += 32)
        G[i * (i + 1) / 2 + j] = gauss_overlap(ci, li, a.S.atom[M.a0 + j], a.S.aux[M.a0 + j].y);
    }
    __syncwarp();
    auto gram = [&](int i, int j) { return i >= j ? G[i * (i + 1) / 2 + j] : G[j * (j + 1) / 2 + i]; };
    float x0 = 0.f, x1 = 0.f;
    float r0 = h0 ? bsum[i0] * scale : 0.f, r1 = h1 ? bsum[i1] * scale : 0.f;
    float p0 = r0, p1 = r1;
    float rs = warp_sum(r0 * r0 + r1 * r1);
    const float tol = 1e-12f * rs;
    for (int it = 0; it < 4 * N && rs > tol; ++it) {
      float y0 = lambda * p0, y1 = lambda * p1;
#pragma unroll 4
      for (int j = 0; j < N; ++j) {
        const float pj = __shfl_sync(0xffffffffu, j < 32 ? p0 : p1, j & 31);
        if (h0) y0 = fmaf(gram(i0, j), pj, y0);
        if (h1) y1 = fmaf(gram(i1, j), pj, y1);
      }
      // warp_sum leaves the same bits in every lane, so these exits are
      // warp-uniform
      const float pap = warp_sum(p0 * y0 + p1 * y1);
      const float al = rs / pap;
      // a non-positive curvature or a non-finite step (possible with ridge 0
      // and nearly coincident atoms) ends the iteration at the last finite x
      if (!(pap > 0.f) || !isfinite(al)) break;
      const float nx0 = fmaf(al, p0, x0), nx1 = fmaf(al, p1, x1);
      if (!__all_sync(0xffffffffu, isfinite(nx0) && isfinite(nx1))) break;
      x0 = nx0; x1 = nx1;
      r0 = fmaf(-al, y0, r0); r1 = fmaf(-al, y1, r1);
      const float rs_new = warp_sum(r0 * r0 + r1 * r1);
      const float be = rs_new / rs;
      p0 = fmaf(be, p0, r0); p1 = fmaf(be, p1, r1);
      rs = rs_new;
    }
    if (h0) a.omega[M.a0 + i0] = x0;
    if (h1) a.omega[M.a0 + i1] = x1;
    __syncwarp();
  }
}

}  // namespace
}  // namespace shp

extern "C" int union_attributions(shp_set S, uint64_t seed, uint64_t stream_base, uint32_t M, float* omega,
                                  void* stream) {
  clear_error();
  if (!S || !omega) { set_error("union_attributions: NULL argument"); return SHP_EINVAL; }
  if (M == 0 || M % 256u) { set_error("union_attributions: M must be a positive multiple of 256"); return SHP_EINVAL; }
  if (S->n_mol == 0) return SHP_OK;
  AttrArgs a{};
  a.S = view(S);
  a.key = Key{(uint32_t)seed, (uint32_t)(seed >> 32)};
  a.stream_base = stream_base;
  a.M = M;
  a.omega = omega;
  return launch_persistent(attribution_kernel, a, S->n_mol, kCVWarps, sizeof(WarpTables) * kCVWarps,
                           (cudaStream_t)stream);
}

extern "C" int cv_fit_weights(shp_set S, const int32_t* idx, int64_t n, const shp_mc* mc, float ridge, float* omega,
                              void* stream) {
  clear_error();
  if (!S || !mc || !omega) { set_error("cv_fit_weights: NULL argument"); return SHP_EINVAL; }
  if (mc->n_samples == 0 || mc->n_samples % 256u || (mc->flags & ~SHP_ID_STREAMS)) {
    set_error("cv_fit_weights: n_samples must be a positive multiple of 256, no flags but SHP_ID_STREAMS");
    return SHP_EINVAL;
  }
  if (!(ridge >= 0.f)) { set_error("cv_fit_weights: ridge must be >= 0"); return SHP_EINVAL; }
  if (n < 0) { set_error("cv_fit_weights: negative n"); return SHP_EINVAL; }
  if (!idx && n > S->n_mol) { set_error("cv_fit_weights: n exceeds the set size"); return SHP_ERANGE; }
  if (n == 0) return SHP_OK;
  FitArgs a{};
  a.S = view(S);
  a.idx = idx;
  a.n_items = n;
  a.key = Key{(uint32_t)mc->seed, (uint32_t)(mc->seed >> 32)};
  a.stream_base = mc->stream_base;
  a.nb = mc->n_samples / 256u;
  a.ridge = ridge;
  a.omega = omega;
  a.by_id = idx && (mc->flags & SHP_ID_STREAMS);
  return launch_persistent(cv_fit_kernel, a, n, kCVWarps, sizeof(WarpTables) * kCVWarps, (cudaStream_t)stream);
}

namespace shp {
namespace {

int self_estimate(const char* who, shp_set S, const int32_t* idx, int64_t n, const shp_mc* mc, const float* omega,
                  float target_rel_se, uint32_t round, int watch, double* vol, double* vol_se, double* self_ov,
                  double* self_se, uint32_t* n_used, cudaStream_t stream) {
  if (!S || !mc) { set_error("%s: NULL argument", who); return SHP_EINVAL; }
  if (mc->n_samples < 2 || (mc->flags & ~SHP_ID_STREAMS)) {
    set_error("%s: n_samples >= 2 and no flags but SHP_ID_STREAMS", who);
    return SHP_EINVAL;
  }
  if (n < 0) { set_error("%s: negative n", who); return SHP_EINVAL; }
  if (watch != 0 && watch != 1) { set_error("%s: watch must be 0 (volume) or 1 (self-overlap)", who); return SHP_EINVAL; }
  if (n == 0) return SHP_OK;
  if (!vol && !self_ov) { set_error("%s: NULL outputs", who); return SHP_EINVAL; }
  if (!idx && n > S->n_mol) { set_error("%s: n exceeds the set size", who); return SHP_ERANGE; }
  CVArgs a{};
  if (target_rel_se > 0.f) {
    if (round == 0 || round % 256u || mc->n_samples % round) {
      set_error("%s: round must be a multiple of 256 dividing n_samples (the cap)", who);
      return SHP_EINVAL;
    }
    a.round_b = round / 256u;
  }
  a.S = view(S);
  a.idx = idx;
  a.omega = omega;
  a.n_items = n;
  a.key = Key{(uint32_t)mc->seed, (uint32_t)(mc->seed >> 32)};
  a.stream_base = mc->stream_base;
  a.n = mc->n_samples;
  a.target = target_rel_se;
  a.watch = watch;
  a.by_id = idx && (mc->flags & SHP_ID_STREAMS);
  a.vol = vol;
  a.vol_se = vol_se;
  a.self_ov = self_ov;
  a.self_se = self_se;
  a.n_used = n_used;
  const size_t smem = sizeof(WarpTables) * kCVWarps;
  return omega ? launch_persistent(cv_volume_kernel<true>, a, n, kCVWarps, smem, stream)
               : launch_persistent(cv_volume_kernel<false>, a, n, kCVWarps, smem, stream);
}

}  // namespace
}  // namespace shp

extern "C" int union_volume_cv(shp_set S, const int32_t* idx, int64_t n, const shp_mc* mc, const float* omega,
                               float target_rel_se, uint32_t round, double* vol, double* vol_se, uint32_t* n_used,
                               void* stream) {
  clear_error();
  if (n > 0 && !vol) { set_error("union_volume_cv: NULL vol"); return SHP_EINVAL; }
  return self_estimate("union_volume_cv", S, idx, n, mc, omega, target_rel_se, round, 0, vol, vol_se, nullptr,
                       nullptr, n_used, (cudaStream_t)stream);
}

extern "C" int union_self_estimate(shp_set S, const int32_t* idx, int64_t n, const shp_mc* mc, const float* omega,
                                   float target_rel_se, uint32_t round, uint32_t watch, double* vol, double* vol_se,
                                   double* self_ov, double* self_se, uint32_t* n_used, void* stream) {
  clear_error();
  return self_estimate("union_self_estimate", S, idx, n, mc, omega, target_rel_se, round, (int)watch, vol, vol_se,
                       self_ov, self_se, n_used, (cudaStream_t)stream);
}

extern "C" int shp_eval_probe(shp_set Q, int32_t iq, shp_set D, int32_t id, int32_t variant, int32_t draw,
                              uint32_t batches, double* sink, int64_t* evals, void* stream) {
  clear_error();
  if (!Q || !D || !sink || !evals) { set_error("shp_eval_probe: NULL argument"); return SHP_EINVAL; }
  if (iq < 0 || iq >= Q->n_mol || id < 0 || id >= D->n_mol) { set_error("shp_eval_probe: molecule index out of range"); return SHP_ERANGE; }
  if (variant < 0) variant = default_variant(kScreen);
  if (variant >= kNumVariants) { set_error("shp_eval_probe: no variant %d", variant); return SHP_ERANGE; }
  if (batches == 0 || batches > (1u << 20)) { set_error("shp_eval_probe: batches must be in 1 .. 2^20"); return SHP_EINVAL; }
  ProbeArgs a{};
  a.A = view(Q);
  a.B = view(D);
  a.xa = iq;
  a.xb = id;
  a.batches = batches;
  a.draw = draw != 0;
  a.key = Key{0x5A17u, 0x0C0FFEEu};
  a.sink = sink;
  int64_t warps = 0;
  const int rc = launch_probe(variant, a, (cudaStream_t)stream, &warps);
  if (rc) return rc;
  const int64_t na = Q->h_off_count(iq), nb = D->h_off_count(id);
  *evals = warps * 2 * (int64_t)batches * 64 * kVariants[variant].sp * (na + nb);
  return SHP_OK;
}
