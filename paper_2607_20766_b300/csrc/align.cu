// Differentiable rigid alignment (Sec. differentiable alignment, Eq. pose,
// Eq. grad): common-random-number (CRN) points from the query, a fused
// forward/adjoint kernel for the CRN overlap and its gradient with respect
// to B's pose (raw quaternion w,x,y,z normalised inside, translation), and a
// persistent multi-start Adam optimiser built on the same device routine.
//
// Objective with points r_k drawn once from the query's mixture:
//   first order  F = (Z_Q / n) sum_k m_B(r_k)
//   union        F = (Z_Q / n) sum_k w_k u_B(r_k),   w_k = u_Q(r_k) / m_Q(r_k)
// dF/dc'_j = (Z_Q / n) sum_k c_jk 2 alpha_j g_j(r_k) (r_k - c'_j) with
// c_jk = 1 (first order) or w_k prod_{l != j} (1 - g_l(r_k)) (union); the
// product over l != j is w_k q_k g_j / f_j in one pass over the atoms, with
// f_j = 1 - g_j rounded once and q_k the product of those same f: the
// rounded factor cancels exactly (g_j can reach 1 when p > 1: an f_j of
// exactly 0 is replaced by 2^-100, which keeps the other factors' product).
// The pose gradient is carried as the force
// f = dF/dt = sum_j dF/dc'_j and the torque tau = sum_j (c'_j - t) x dF/dc'_j
// (dF = tau . omega for the rotation c'_j - t -> (I + [omega]x)(c'_j - t)).
// With u_k = sum_j (dF/dc'_j)_k, point k's share of the force, and
// c'_j - t = (r_k - t) - (r_k - c'_j), tau = sum_k (r_k - t) x u_k. With
// h_jk the scalar factor of dF/dc'_j's k term and o the query centroid,
// u_k = (r_k - o) sum_j h_jk - sum_j h_jk (c'_j - o): four FMAs per point and
// atom, against the expanded exponent's b_j = 2 alpha_j log2(e) (c'_j - o). For q = (w, v) = p / |p| the left perturbation
// q -> (1, omega / 2) q gives dF/dw = -2 tau . v, dF/dv = 2 (w tau + tau x v),
// orthogonal to q, so dF/dp is that vector over |p|.
#include <cmath>

#include "device.cuh"
#include "internal.h"

namespace shp {
namespace {

constexpr int kAlignWarps = 4;
constexpr int kAlignThreads = kAlignWarps * 32;

// Expanded exponent of one posed atom about the origin o, every scalar twice
// (two CRN points per packed FP32x2 instruction): b = 2 alpha log2(e)
// (R c + t - o), c0 = -alpha log2(e) |R c + t - o|^2 + log2 p, a = -alpha log2(e).
struct __align__(16) CoefA {
  float4 bxy;  // bx, bx, by, by
  float4 bzc;  // bz, bz, c0, c0
  float2 a;    // a, a
  float2 pad;
};

// Two posed atoms j, j + 1 of B for the closed-form objective: minus their
// centres less t (y = R c), their beta' and log2 w' (fo_atom_consts); an odd
// count is padded with an atom of weight 0.
struct __align__(16) FoPairB {
  float4 nxy;  // -y_j.x, -y_j+1.x, -y_j.y, -y_j+1.y
  float4 nzb;  // -y_j.z, -y_j+1.z, beta'_j, beta'_j+1
  float2 lw;   // log2 w'_j, log2 w'_j+1
  float2 pad;
};

struct __align__(16) AlignTables {
  float4 body[SHP_MAX_ATOMS];   // B's centres (own frame), alpha
  float4 posed[SHP_MAX_ATOMS];  // R c (the posed centre less t), -alpha log2(e)
  CoefA coef[SHP_MAX_ATOMS];
  float lp[SHP_MAX_ATOMS];      // log2 p
  // closed-form objective
  float4 qatom[SHP_MAX_ATOMS];     // the query's centres, beta'
  float qlp[SHP_MAX_ATOMS];        // the query's log2 w'
  float2 fob[SHP_MAX_ATOMS];       // B's beta', log2 w'
  FoPairB fo2[SHP_MAX_ATOMS / 2];  // B's posed atoms in pairs
  float4 origin;                // o: the query's atom centroid
};
constexpr size_t kAlignSmem = sizeof(AlignTables) * kAlignWarps;

__device__ __forceinline__ void quat_to_rot(const float q[4], float R[9]) {
  const float w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

// Rotation matrix (row-major) to a unit quaternion (w, x, y, z), w >= 0
// branch chosen by the largest diagonal combination.
__device__ void rot_to_quat(const float R[9], float q[4]) {
  const float tr = R[0] + R[4] + R[8];
  if (tr > 0.f) {
    const float s = 2.f * sqrtf(tr + 1.f);
    q[0] = 0.25f * s; q[1] = (R[7] - R[5]) / s; q[2] = (R[2] - R[6]) / s; q[3] = (R[3] - R[1]) / s;
  } else if (R[0] > R[4] && R[0] > R[8]) {
    const float s = 2.f * sqrtf(1.f + R[0] - R[4] - R[8]);
    q[0] = (R[7] - R[5]) / s; q[1] = 0.25f * s; q[2] = (R[1] + R[3]) / s; q[3] = (R[2] + R[6]) / s;
  } else if (R[4] > R[8]) {
    const float s = 2.f * sqrtf(1.f + R[4] - R[0] - R[8]);
    q[0] = (R[2] - R[6]) / s; q[1] = (R[1] + R[3]) / s; q[2] = 0.25f * s; q[3] = (R[5] + R[7]) / s;
  } else {
    const float s = 2.f * sqrtf(1.f + R[8] - R[0] - R[4]);
    q[0] = (R[3] - R[1]) / s; q[1] = (R[2] + R[6]) / s; q[2] = (R[5] + R[7]) / s; q[3] = 0.25f * s;
  }
}

__device__ void stage_body(AlignTables& T, const SetView& B, int32_t a0, int nb, bool closed, int lane) {
  for (int i = lane; i < nb; i += 32) {
    const float4 c = B.atom[a0 + i];
    T.body[i] = c;
    T.lp[i] = B.aux[a0 + i].y;
    if (closed) {
      float beta, lw;
      fo_atom_consts(c.w, T.lp[i], beta, lw);
      T.fob[i] = make_float2(beta, lw);
    }
  }
  __syncwarp();
}

// Posed centres c' = R c + t and, for the CRN objectives, the expanded
// exponent log2 g(r) = a |r - o|^2 + b . (r - o) + c0 with a = -alpha log2(e)
// (the posed table's w), b = -2 a (c' - o), c0 = a |c' - o|^2 + log2 p.
__device__ void stage_posed(AlignTables& T, int nb, const float pose[7], bool closed, int lane) {
  const float kLog2e = 1.4426950408889634f;
  const float4 o = T.origin;
  float q[4] = {pose[0], pose[1], pose[2], pose[3]};
  const float inv = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) q[k] *= inv;
  float R[9];
  quat_to_rot(q, R);
  __syncwarp();
  for (int i = lane; i < nb; i += 32) {
    const float4 c = T.body[i];
    const float a = -c.w * kLog2e;
    const float yx = fmaf(R[0], c.x, fmaf(R[1], c.y, R[2] * c.z));
    const float yy = fmaf(R[3], c.x, fmaf(R[4], c.y, R[5] * c.z));
    const float yz = fmaf(R[6], c.x, fmaf(R[7], c.y, R[8] * c.z));
    T.posed[i] = make_float4(yx, yy, yz, a);
    if (closed) continue;  // the closed form uses the posed centres only
    const float dx = yx + pose[4] - o.x, dy = yy + pose[5] - o.y, dz = yz + pose[6] - o.z;
    const float bx = -2.f * a * dx, by = -2.f * a * dy, bz = -2.f * a * dz;
    const float c0 = fmaf(a, fmaf(dx, dx, fmaf(dy, dy, dz * dz)), T.lp[i]);
    CoefA k;
    k.bxy = make_float4(bx, bx, by, by);
    k.bzc = make_float4(bz, bz, c0, c0);
    k.a = make_float2(a, a);
    k.pad = make_float2(0.f, 0.f);
    T.coef[i] = k;
  }
  __syncwarp();
  if (closed) {
    for (int p = lane; 2 * p < nb; p += 32) {
      const int j = 2 * p;
      const bool two = j + 1 < nb;
      const float4 y0 = T.posed[j], y1 = two ? T.posed[j + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float2 f0 = T.fob[j], f1 = two ? T.fob[j + 1] : make_float2(1.f, -INFINITY);
      FoPairB P;
      P.nxy = make_float4(-y0.x, -y1.x, -y0.y, -y1.y);
      P.nzb = make_float4(-y0.z, -y1.z, f0.x, f1.x);
      P.lw = make_float2(f0.y, f1.y);
      P.pad = make_float2(0.f, 0.f);
      T.fo2[p] = P;
    }
    __syncwarp();
  }
}

// g_j at two points r' = r - o (one per half) with rr = |r'|^2: the expanded
// exponent in four packed FMAs, two SFU exp2.
__device__ __forceinline__ float2 g_expanded2(const CoefA& k, float2 rx, float2 ry, float2 rz, float2 rr) {
  float2 e = __ffma2_rn(make_float2(k.bzc.x, k.bzc.y), rz, make_float2(k.bzc.z, k.bzc.w));
  e = __ffma2_rn(make_float2(k.bxy.z, k.bxy.w), ry, e);
  e = __ffma2_rn(make_float2(k.bxy.x, k.bxy.y), rx, e);
  e = __ffma2_rn(k.a, rr, e);
  return make_float2(ex2_approx(e.x), ex2_approx(e.y));
}

// Adjoint sums of one atom j for two points: ha += a_j e, v += b_j e.
__device__ __forceinline__ void adj_add(const CoefA& k, float2 e, float2& ha, float2& vx, float2& vy, float2& vz) {
  ha = __ffma2_rn(k.a, e, ha);
  vx = __ffma2_rn(make_float2(k.bxy.x, k.bxy.y), e, vx);
  vy = __ffma2_rn(make_float2(k.bxy.z, k.bxy.w), e, vy);
  vz = __ffma2_rn(make_float2(k.bzc.x, k.bzc.y), e, vz);
}

// The query's atoms for the closed-form objective: centres, beta', log2 w'.
__device__ void stage_query(AlignTables& T, const SetView& Q, int32_t iq, int lane) {
  const int32_t a0 = Q.off[iq], na = Q.off[iq + 1] - a0;
  for (int i = lane; i < na; i += 32) {
    const float4 c = Q.atom[a0 + i];
    float beta, lw;
    fo_atom_consts(c.w, Q.aux[a0 + i].y, beta, lw);
    T.qatom[i] = make_float4(c.x, c.y, c.z, beta);
    T.qlp[i] = lw;
  }
  __syncwarp();
}

// The frame origin of the expanded exponent: the query's atom centroid.
__device__ void stage_origin(AlignTables& T, const SetView& Q, int32_t iq, int lane) {
  const int32_t a0 = Q.off[iq], na = Q.off[iq + 1] - a0;
  float sx = 0.f, sy = 0.f, sz = 0.f;
  for (int i = lane; i < na; i += 32) {
    const float4 a = Q.atom[a0 + i];
    sx += a.x; sy += a.y; sz += a.z;
  }
  sx = warp_sum(sx); sy = warp_sum(sy); sz = warp_sum(sz);
  const float inv = 1.f / (float)na;
  __syncwarp();
  if (lane == 0) T.origin = make_float4(sx * inv, sy * inv, sz * inv, 0.f);
  __syncwarp();
}

// Objective and gradient at the staged pose (translation t). acc = {F, force
// f = dF/dt (3), torque tau (3)}, reduced over the warp (every lane gets lane
// 0's totals). CRN objectives are returned before their Z_Q / n factor; the
// closed-form first order (Eq. fo) is exact:
//   F = sum_ij K_ij,  K_ij = p_i p_j (pi/s)^{3/2} exp(-a d^2), s = alpha_i +
//   alpha_j, a = alpha_i alpha_j / s, dF/dc'_j = sum_i 2 a K_ij (c_i - c'_j);
// lanes over the query's atoms i: with x_i = c_i - t, y_j = c'_j - t and
// h_ij = a K_ij, f = 2 sum_i (x_i H_i - W_i) and tau = 2 sum_i W_i x x_i for
// H_i = sum_j h_ij, W_i = sum_j h_ij y_j.
__device__ __forceinline__ void add_cross(float acc[7], float ax, float ay, float az, float bx, float by, float bz) {
  acc[4] = fmaf(ay, bz, fmaf(-az, by, acc[4]));
  acc[5] = fmaf(az, bx, fmaf(-ax, bz, acc[5]));
  acc[6] = fmaf(ax, by, fmaf(-ay, bx, acc[6]));
}

__device__ void value_grad(AlignTables& T, int nb, int na, const float4* __restrict__ pts, int n, int objective,
                           const float t[3], int lane, float acc[7]) {
#pragma unroll
  for (int i = 0; i < 7; ++i) acc[i] = 0.f;
  if (objective == SHP_OBJ_FO_CLOSED) {
    // K_ij = w'_i w'_j r^3 2^(-r^2 d^2) (fo_atom_consts) and h_ij = a K_ij =
    // ln 2 r^5 2^(...) w'_i w'_j; two database atoms per packed instruction
    const float kLn2 = 0.6931471805599453f;
    const int nb2 = (nb + 1) / 2;
    for (int i = lane; i < na; i += 32) {
      const float4 qa = T.qatom[i];
      const float xi = qa.x - t[0], yi = qa.y - t[1], zi = qa.z - t[2];
      const float2 x2 = make_float2(xi, xi), y2 = make_float2(yi, yi), z2 = make_float2(zi, zi);
      const float2 b2 = make_float2(qa.w, qa.w), l2 = make_float2(T.qlp[i], T.qlp[i]);
      float2 Fn = make_float2(0.f, 0.f), Hs = Fn, Wx = Fn, Wy = Fn, Wz = Fn;  // -F, H / ln 2, -W / ln 2
#pragma unroll 2
      for (int p = 0; p < nb2; ++p) {
        const FoPairB& P = T.fo2[p];
        const float2 ny = make_float2(P.nxy.z, P.nxy.w), nx = make_float2(P.nxy.x, P.nxy.y);
        const float2 nz = make_float2(P.nzb.x, P.nzb.y);
        const float2 dx = __fadd2_rn(x2, nx), dy = __fadd2_rn(y2, ny), dz = __fadd2_rn(z2, nz);
        const float2 d2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
        const float2 sb = __fadd2_rn(b2, make_float2(P.nzb.z, P.nzb.w));
        const float2 r = make_float2(rsqrtf(sb.x), rsqrtf(sb.y));
        const float2 rn = __fmul2_rn(r, make_float2(-r.x, -r.y));  // -r^2
        const float2 e = __ffma2_rn(rn, d2, __fadd2_rn(l2, P.lw));
        const float2 Kn = __fmul2_rn(__fmul2_rn(rn, r), make_float2(ex2_approx(e.x), ex2_approx(e.y)));  // -K
        Fn = __fadd2_rn(Fn, Kn);
        const float2 hp = __fmul2_rn(rn, Kn);  // h / ln 2
        Hs = __fadd2_rn(Hs, hp);
        Wx = __ffma2_rn(hp, nx, Wx); Wy = __ffma2_rn(hp, ny, Wy); Wz = __ffma2_rn(hp, nz, Wz);
      }
      const float H = kLn2 * (Hs.x + Hs.y);
      const float Wxs = -kLn2 * (Wx.x + Wx.y), Wys = -kLn2 * (Wy.x + Wy.y), Wzs = -kLn2 * (Wz.x + Wz.y);
      acc[0] -= Fn.x + Fn.y;
      acc[1] += 2.f * fmaf(xi, H, -Wxs); acc[2] += 2.f * fmaf(yi, H, -Wys); acc[3] += 2.f * fmaf(zi, H, -Wzs);
      add_cross(acc, 2.f * Wxs, 2.f * Wys, 2.f * Wzs, xi, yi, zi);
    }
  }
  // CRN objectives: each lane takes kPairs packed point pairs per pass,
  // points k + 64 p and k + 64 p + 32 of every 64 kPairs (those past n with
  // weight 0, skipped in the sums), in the halves of packed FP32x2 values.
  // ha = sum_j a_j e_jk, v = sum_j b_j e_jk with e_jk = h_jk /
  // (2 alpha_j ln 2): u_k = -ln 2 (2 ha (r_k - o) + v).
  constexpr int kPairs = 2;
  const float4 o = T.origin;
  for (int k0 = lane; k0 < n && objective != SHP_OBJ_FO_CLOSED; k0 += 64 * kPairs) {
    float4 rs[kPairs][2];
    bool has[kPairs][2];
    float2 ox[kPairs], oy[kPairs], oz[kPairs], rr[kPairs], w[kPairs];
    float2 ha[kPairs], vx[kPairs], vy[kPairs], vz[kPairs], F[kPairs];
#pragma unroll
    for (int p = 0; p < kPairs; ++p) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = k0 + 64 * p + 32 * h;
        has[p][h] = k < n;
        rs[p][h] = pts[has[p][h] ? k : k0];
      }
      ox[p] = make_float2(rs[p][0].x - o.x, rs[p][1].x - o.x);
      oy[p] = make_float2(rs[p][0].y - o.y, rs[p][1].y - o.y);
      oz[p] = make_float2(rs[p][0].z - o.z, rs[p][1].z - o.z);
      rr[p] = __ffma2_rn(ox[p], ox[p], __ffma2_rn(oy[p], oy[p], __fmul2_rn(oz[p], oz[p])));
      w[p] = make_float2(has[p][0] ? rs[p][0].w : 0.f, has[p][1] ? rs[p][1].w : 0.f);
      ha[p] = make_float2(0.f, 0.f); vx[p] = ha[p]; vy[p] = ha[p]; vz[p] = ha[p];
    }
    if (objective == SHP_OBJ_FO) {
      float2 m[kPairs];
#pragma unroll
      for (int p = 0; p < kPairs; ++p) m[p] = make_float2(0.f, 0.f);
#pragma unroll 2
      for (int j = 0; j < nb; ++j) {
        const CoefA& k = T.coef[j];
#pragma unroll
        for (int p = 0; p < kPairs; ++p) {
          const float2 g = g_expanded2(k, ox[p], oy[p], oz[p], rr[p]);  // h = 2 alpha g
          m[p] = __fadd2_rn(m[p], g);
          adj_add(k, g, ha[p], vx[p], vy[p], vz[p]);
        }
      }
#pragma unroll
      for (int p = 0; p < kPairs; ++p) F[p] = m[p];
    } else {
      // one pass: with f_j = 1 - g_j (rounded once) and q = prod_j f_j, the
      // adjoint weight of atom j is w prod_{l != j} f_l g_j = w q g_j / f_j;
      // the same rounded f_j enters the product and the quotient, so they
      // cancel exactly. An f_j of exactly 0 is replaced by 2^-100: q then
      // carries that factor (u = w (1 - q) is unchanged to FP32) and q / f_j
      // still gives the other factors' product.
      float2 q[kPairs];
#pragma unroll
      for (int p = 0; p < kPairs; ++p) q[p] = make_float2(1.f, 1.f);
      const float2 one = make_float2(1.f, 1.f), m1 = make_float2(-1.f, -1.f);
#pragma unroll 2
      for (int j = 0; j < nb; ++j) {
        const CoefA& k = T.coef[j];
#pragma unroll
        for (int p = 0; p < kPairs; ++p) {
          const float2 g = g_expanded2(k, ox[p], oy[p], oz[p], rr[p]);
          float2 f = __ffma2_rn(g, m1, one);
          f.x = f.x == 0.f ? 0x1p-100f : f.x;
          f.y = f.y == 0.f ? 0x1p-100f : f.y;
          q[p] = __fmul2_rn(q[p], f);
          const float2 e = make_float2(__fdividef(g.x, f.x), __fdividef(g.y, f.y));
          adj_add(k, e, ha[p], vx[p], vy[p], vz[p]);
        }
      }
#pragma unroll
      for (int p = 0; p < kPairs; ++p) {
        F[p] = make_float2(w[p].x * (1.f - q[p].x), w[p].y * (1.f - q[p].y));
        const float2 qw = __fmul2_rn(q[p], w[p]);  // h = 2 alpha e qw
        ha[p] = __fmul2_rn(ha[p], qw);
        vx[p] = __fmul2_rn(vx[p], qw);
        vy[p] = __fmul2_rn(vy[p], qw);
        vz[p] = __fmul2_rn(vz[p], qw);
      }
    }
    const float kLn2 = 0.6931471805599453f;
#pragma unroll
    for (int p = 0; p < kPairs; ++p) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!has[p][h]) continue;
        const float oxh = h ? ox[p].y : ox[p].x, oyh = h ? oy[p].y : oy[p].x, ozh = h ? oz[p].y : oz[p].x;
        const float hah = h ? ha[p].y : ha[p].x;
        const float ux = -kLn2 * fmaf(2.f * hah, oxh, h ? vx[p].y : vx[p].x);
        const float uy = -kLn2 * fmaf(2.f * hah, oyh, h ? vy[p].y : vy[p].x);
        const float uz = -kLn2 * fmaf(2.f * hah, ozh, h ? vz[p].y : vz[p].x);
        acc[0] += h ? F[p].y : F[p].x;
        acc[1] += ux; acc[2] += uy; acc[3] += uz;
        add_cross(acc, rs[p][h].x - t[0], rs[p][h].y - t[1], rs[p][h].z - t[2], ux, uy, uz);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 7; ++i) acc[i] = __shfl_sync(0xffffffffu, warp_sum(acc[i]), 0);
}

// dF/d(raw pose) from the force, the torque and the raw quaternion p
// (q = (w, v) = p / |p|): dF/dp = (-2 tau . v, 2 (w tau + tau x v)) / |p|.
__device__ void pose_gradient(const float pose[7], const float acc[7], float scale, float grad[7]) {
  const float inq = rsqrtf(pose[0] * pose[0] + pose[1] * pose[1] + pose[2] * pose[2] + pose[3] * pose[3]);
  const float w = pose[0] * inq, x = pose[1] * inq, y = pose[2] * inq, z = pose[3] * inq;
  const float tx = acc[4], ty = acc[5], tz = acc[6];
  const float k = 2.f * scale * inq;
  grad[0] = -k * (tx * x + ty * y + tz * z);
  grad[1] = k * (w * tx + ty * z - tz * y);
  grad[2] = k * (w * ty + tz * x - tx * z);
  grad[3] = k * (w * tz + tx * y - ty * x);
  grad[4] = scale * acc[1];
  grad[5] = scale * acc[2];
  grad[6] = scale * acc[3];
}

// Points 2s, 2s + 1 of the usual sample layout; antithetic: 2s + 1 is the
// reflection of 2s about its component centre (same pick, negated normals).
__global__ void crn_points_kernel(SetView Q, int32_t iq, Key key, uint64_t stream, uint32_t n, bool anti,
                                  float4* out) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;  // sample pair
  if (2u * s >= n) return;
  const int32_t a0 = Q.off[iq], na = Q.off[iq + 1] - a0;
  const uint32_t slo = (uint32_t)stream, shi = (uint32_t)(stream >> 32);
  const uint4 w0 = philox10(make_uint4(2u * s, slo, shi, SHP_TAG_CRN), key);
  const uint4 w1 = philox10(make_uint4(2u * s + 1u, slo, shi, SHP_TAG_CRN), key);
  float z[6];
  box_muller(w0.z, w0.w, z[0], z[1]);
  box_muller(w1.x, w1.y, z[2], z[3]);
  box_muller(w1.z, w1.w, z[4], z[5]);
  const uint32_t words[2] = {w0.x, anti ? w0.x : w0.y};
  const float zz[2][3] = {{z[0], z[1], z[4]}, {anti ? -z[0] : z[2], anti ? -z[1] : z[3], anti ? -z[4] : z[5]}};
  const float kLog2e = 1.4426950408889634f;
  for (int t = 0; t < 2; ++t) {
    if (2u * s + t >= n) break;
    const unsigned long long prod = (unsigned long long)words[t] * (unsigned)na;
    const uint32_t j = (uint32_t)(prod >> 32), f = (uint32_t)prod;
    const int i = f < Q.thr[a0 + j] ? (int)j : (int)Q.alias[a0 + j];
    const float4 c = Q.atom[a0 + i];
    const float sg = Q.aux[a0 + i].x;
    const float rx = fmaf(sg, zz[t][0], c.x), ry = fmaf(sg, zz[t][1], c.y), rz = fmaf(sg, zz[t][2], c.z);
    float m = 0.f, q = 1.f;
    for (int l = 0; l < na; ++l) {
      const float4 a = Q.atom[a0 + l];
      const float dx = rx - a.x, dy = ry - a.y, dz = rz - a.z;
      const float g = ex2_approx(fmaf(-a.w * kLog2e, fmaf(dx, dx, fmaf(dy, dy, dz * dz)), Q.aux[a0 + l].y));
      m += g;
      q = fmaf(-g, q, q);
    }
    out[2u * s + t] = make_float4(rx, ry, rz, __fdividef(1.f - q, m));
  }
}

struct GradArgs {
  SetView B;
  const int32_t* ib;
  const float* pose;
  const float4* pts;
  int n_pts;
  int objective;
  uint32_t scale_n;  // n of the CRN objectives (scale Z_Q / n, Z_Q read on the device), 0 for the closed form (1)
  SetView Q;
  int32_t iq;
  int64_t n_items;
  double* value;
  float* grad;
};

__global__ void __launch_bounds__(kAlignThreads) pose_grad_kernel(const GradArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  AlignTables& T = reinterpret_cast<AlignTables*>(smem_raw)[warp];
  const int64_t item = (int64_t)blockIdx.x * kAlignWarps + warp;
  if (item >= a.n_items) return;
  const int32_t xb = a.ib[item];
  if (xb < 0 || xb >= a.B.n_mol) {
    if (lane == 0) {
      a.value[item] = __longlong_as_double(0x7ff8000000000000ll);
      for (int d = 0; d < 7; ++d) a.grad[7 * item + d] = __int_as_float(0x7fc00000);
    }
    return;
  }
  const int32_t b0 = a.B.off[xb], nb = a.B.off[xb + 1] - b0;
  float pose[7];
  for (int d = 0; d < 7; ++d) pose[d] = a.pose[7 * item + d];
  const bool closed = a.objective == SHP_OBJ_FO_CLOSED;
  stage_body(T, a.B, b0, nb, closed, lane);
  if (closed) stage_query(T, a.Q, a.iq, lane);
  stage_origin(T, a.Q, a.iq, lane);
  stage_posed(T, nb, pose, closed, lane);
  float acc[7];
  value_grad(T, nb, a.Q.off[a.iq + 1] - a.Q.off[a.iq], a.pts, a.n_pts, a.objective, pose + 4, lane, acc);
  if (lane == 0) {
    const double scale = a.scale_n ? a.Q.Z[a.iq] / (double)a.scale_n : 1.0;
    float g[7];
    pose_gradient(pose, acc, (float)scale, g);
    a.value[item] = scale * (double)acc[0];
    for (int d = 0; d < 7; ++d) a.grad[7 * item + d] = g[d];
  }
}

struct AdamArgs {
  SetView Q, B;
  int32_t iq;
  const int32_t* ib;
  int64_t n_pairs;
  int starts, steps, objective;
  const float4* pts;
  int n_pts;
  uint32_t scale_n;  // as in GradArgs
  float lr, lr_t, beta1, beta2, eps;
  Key key;
  uint64_t stream;
  float* pose_out;   // [n_pairs * starts][7]
  float* value_out;  // [n_pairs * starts]
  unsigned long long* queue;
};

// Start s of pair (Q, B): s < 4 maps B's principal frame onto Q's with one
// of the four proper axis sign patterns; s >= 4 uses a uniform random
// rotation (Shoemake, from Philox words, tag SHP_TAG_START) between the two
// frames. The translation matches the frame centroids.
__device__ void start_pose(const AdamArgs& a, int32_t xb, int64_t pair, int s, float pose[7]) {
  const float* FA = a.Q.frame + 12 * (int64_t)a.iq;
  const float* FB = a.B.frame + 12 * (int64_t)xb;
  float M[9];  // middle rotation in principal coordinates
  if (s < 4) {
    const float sx = (s == 2 || s == 3) ? -1.f : 1.f, sy = (s == 1 || s == 3) ? -1.f : 1.f;
    const float sz = sx * sy;
    M[0] = sx; M[1] = 0.f; M[2] = 0.f; M[3] = 0.f; M[4] = sy; M[5] = 0.f; M[6] = 0.f; M[7] = 0.f; M[8] = sz;
  } else {
    const uint4 w = philox10(make_uint4((uint32_t)s, (uint32_t)pair, (uint32_t)((uint64_t)pair >> 32), SHP_TAG_START),
                             a.key);
    const float u1 = (float)(w.x >> 8) * 5.9604644775390625e-08f;
    const float u2 = (float)(w.y >> 8) * 5.9604644775390625e-08f;
    const float u3 = (float)(w.z >> 8) * 5.9604644775390625e-08f;
    const float r1 = sqrtf(1.f - u1), r2 = sqrtf(u1);
    float s2, c2, s3, c3;
    sincospif(2.f * u2, &s2, &c2);
    sincospif(2.f * u3, &s3, &c3);
    const float q[4] = {r2 * c3, r1 * s2, r1 * c2, r2 * s3};
    quat_to_rot(q, M);
  }
  // R = E_A M E_B^T
  float T1[9], R[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      float t = 0.f;
      for (int k = 0; k < 3; ++k) t = fmaf(FA[3 + 3 * i + k], M[3 * k + j], t);
      T1[3 * i + j] = t;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      float t = 0.f;
      for (int k = 0; k < 3; ++k) t = fmaf(T1[3 * i + k], FB[3 + 3 * j + k], t);
      R[3 * i + j] = t;
    }
  float q[4];
  rot_to_quat(R, q);
  for (int k = 0; k < 4; ++k) pose[k] = q[k];
  for (int i = 0; i < 3; ++i)
    pose[4 + i] = FA[i] - (R[3 * i] * FB[0] + R[3 * i + 1] * FB[1] + R[3 * i + 2] * FB[2]);
}

__global__ void __launch_bounds__(kAlignThreads) align_adam_kernel(const AdamArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  AlignTables& T = reinterpret_cast<AlignTables*>(smem_raw)[warp];
  const int64_t n_items = a.n_pairs * a.starts;
  const float scale = a.scale_n ? (float)(a.Q.Z[a.iq] / (double)a.scale_n) : 1.f;
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(a.queue, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= (unsigned long long)n_items) break;
    const int64_t pair = (int64_t)item / a.starts;
    const int s = (int)((int64_t)item - pair * a.starts);
    const int32_t xb = a.ib[pair];
    if (xb < 0 || xb >= a.B.n_mol) {
      if (lane == 0) {
        for (int d = 0; d < 7; ++d) a.pose_out[7 * item + d] = __int_as_float(0x7fc00000);
        a.value_out[item] = __int_as_float(0x7fc00000);
      }
      continue;
    }
    const int32_t b0 = a.B.off[xb], nb = a.B.off[xb + 1] - b0;
    float pose[7], m1[7], m2[7];
    start_pose(a, xb, pair, s, pose);
    for (int d = 0; d < 7; ++d) { m1[d] = 0.f; m2[d] = 0.f; }
    const bool closed = a.objective == SHP_OBJ_FO_CLOSED;
    stage_body(T, a.B, b0, nb, closed, lane);
    if (closed) stage_query(T, a.Q, a.iq, lane);
    stage_origin(T, a.Q, a.iq, lane);
    const int na = a.Q.off[a.iq + 1] - a.Q.off[a.iq];
    float b1t = 1.f, b2t = 1.f, value = 0.f;
    for (int step = 0; step < a.steps; ++step) {
      stage_posed(T, nb, pose, closed, lane);
      float acc[7];
      value_grad(T, nb, na, a.pts, a.n_pts, a.objective, pose + 4, lane, acc);
      float g[7];
      pose_gradient(pose, acc, scale, g);
      value = scale * acc[0];
      b1t *= a.beta1;
      b2t *= a.beta2;
      // cosine step-size decay: constant-step Adam keeps moving by about the
      // step size around the optimum, the decay lets it settle
      const float decay = 0.5f * (1.f + cospif((float)step / (float)a.steps));
      const float c1 = 1.f / (1.f - b1t), c2 = 1.f / (1.f - b2t);  // bias corrections
      for (int d = 0; d < 7; ++d) {  // Adam ascent (maximise the overlap)
        m1[d] = fmaf(a.beta1, m1[d], (1.f - a.beta1) * g[d]);
        m2[d] = fmaf(a.beta2, m2[d], (1.f - a.beta2) * g[d] * g[d]);
        const float mh = m1[d] * c1, vh = m2[d] * c2;
        pose[d] += __fdividef(decay * (d < 4 ? a.lr : a.lr_t) * mh, sqrtf(vh) + a.eps);
      }
      // keep the raw quaternion near unit length (the objective ignores its scale)
      const float inv = rsqrtf(pose[0] * pose[0] + pose[1] * pose[1] + pose[2] * pose[2] + pose[3] * pose[3]);
      for (int d = 0; d < 4; ++d) pose[d] *= inv;
    }
    if (lane == 0) {
      for (int d = 0; d < 7; ++d) a.pose_out[7 * item + d] = pose[d];
      a.value_out[item] = value;
    }
    __syncwarp();
  }
}

// Best start per pair by the union Tanimoto of the scored poses.
__global__ void select_best_kernel(int64_t n_pairs, int starts, const double* est, const double* self_q,
                                   int32_t iq, const double* self_db, int32_t n_db, const int32_t* ib,
                                   const float* poses, float* pose_out, float* T_out, float* T_starts) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pairs) return;
  const int32_t xb = ib[p];
  if (xb < 0 || xb >= n_db) {
    const float nan = __int_as_float(0x7fc00000);
    T_out[p] = nan;
    for (int d = 0; d < 7; ++d) pose_out[7 * p + d] = nan;
    if (T_starts)
      for (int s = 0; s < starts; ++s) T_starts[p * starts + s] = nan;
    return;
  }
  float best = -1.f;
  int bs = 0;
  for (int s = 0; s < starts; ++s) {
    const int64_t it = p * starts + s;
    const double O = est[2 * it + 1];
    const double S = self_q[2 * (int64_t)iq + 1] + self_db[2 * (int64_t)xb + 1];
    const float T = (float)(O / (S - O));
    if (T_starts) T_starts[it] = T;
    if (T > best) { best = T; bs = s; }
  }
  T_out[p] = best;
  for (int d = 0; d < 7; ++d) pose_out[7 * p + d] = poses[7 * (p * starts + bs) + d];
}

__global__ void pair_index_kernel(int64_t n_pairs, int starts, int32_t iq, const int32_t* ib, int32_t* ia_out,
                                  int32_t* ib_out) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= n_pairs * starts) return;
  ia_out[it] = iq;
  ib_out[it] = ib[it / starts];
}

int check_points_args(shp_set Q, int32_t iq, const char* who) {
  if (!Q) { set_error("%s: NULL set", who); return SHP_EINVAL; }
  if (iq < 0 || iq >= Q->n_mol) { set_error("%s: query index %d out of range", who, iq); return SHP_ERANGE; }
  return SHP_OK;
}

}  // namespace
}  // namespace shp

using namespace shp;

extern "C" int align_crn_points(shp_set Q, int32_t iq, const shp_mc* mc, float* points, void* stream) {
  clear_error();
  int rc = check_points_args(Q, iq, "align_crn_points");
  if (rc) return rc;
  if (!mc || mc->n_samples < 1 || !points || (mc->flags & ~SHP_ANTITHETIC)) {
    set_error("align_crn_points: bad arguments (flags: SHP_ANTITHETIC only)");
    return SHP_EINVAL;
  }
  const uint32_t pairs = (mc->n_samples + 1u) / 2u;
  crn_points_kernel<<<(pairs + 127u) / 128u, 128, 0, (cudaStream_t)stream>>>(
      view(Q), iq, Key{(uint32_t)mc->seed, (uint32_t)(mc->seed >> 32)}, mc->stream_base, mc->n_samples,
      (mc->flags & SHP_ANTITHETIC) != 0, reinterpret_cast<float4*>(points));
  SHP_CUDA(cudaGetLastError());
  return SHP_OK;
}

extern "C" int overlap_pose_grad(shp_set Q, int32_t iq, const float* points, uint32_t n_points, shp_set B,
                                 const int32_t* ib, int64_t n_items, const float* pose, uint32_t objective,
                                 double* value, float* grad, void* stream) {
  clear_error();
  int rc = check_points_args(Q, iq, "overlap_pose_grad");
  if (rc) return rc;
  const bool closed = objective == SHP_OBJ_FO_CLOSED;
  if (!B || objective > SHP_OBJ_FO_CLOSED || n_items < 0 || (!closed && n_points < 1)) {
    set_error("overlap_pose_grad: bad arguments");
    return SHP_EINVAL;
  }
  if (n_items == 0) return SHP_OK;
  if ((!closed && !points) || !ib || !pose || !value || !grad) {
    set_error("overlap_pose_grad: NULL array");
    return SHP_EINVAL;
  }
  GradArgs a{};
  a.B = view(B);
  a.Q = view(Q);
  a.iq = iq;
  a.ib = ib;
  a.pose = pose;
  a.pts = reinterpret_cast<const float4*>(points);
  a.n_pts = closed ? 0 : (int)n_points;
  a.objective = (int)objective;
  a.scale_n = closed ? 0u : n_points;
  a.n_items = n_items;
  a.value = value;
  a.grad = grad;
  SHP_CUDA(cudaFuncSetAttribute(pose_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAlignSmem));
  const int64_t blocks = (n_items + kAlignWarps - 1) / kAlignWarps;
  pose_grad_kernel<<<(unsigned)blocks, kAlignThreads, kAlignSmem, (cudaStream_t)stream>>>(a);
  SHP_CUDA(cudaGetLastError());
  return SHP_OK;
}

extern "C" int align_rigid(shp_set Q, int32_t iq, shp_set B, const int32_t* ib, int64_t n_pairs,
                           const shp_align* cfg, const double* self_q, const double* self_db, float* pose_out,
                           float* T_out, float* T_starts, float* pose_starts, void* stream) {
  clear_error();
  int rc = check_points_args(Q, iq, "align_rigid");
  if (rc) return rc;
  if (!B || !cfg || n_pairs < 0) { set_error("align_rigid: bad arguments"); return SHP_EINVAL; }
  if (cfg->starts < 1 || cfg->starts > 64 || cfg->n_crn < 2 || cfg->n_score < 2 || cfg->objective > SHP_OBJ_FO_CLOSED ||
      (cfg->crn_flags & ~SHP_ANTITHETIC) ||
      !(cfg->lr > 0.f) || !(cfg->lr_t > 0.f) || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) ||
      !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) || !(cfg->eps > 0.f)) {
    set_error("align_rigid: invalid configuration");
    return SHP_EINVAL;
  }
  if (n_pairs == 0) return SHP_OK;
  if (!ib || !self_q || !self_db || !pose_out || !T_out) { set_error("align_rigid: NULL array"); return SHP_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  rc = ensure_frames(Q, st);  // the principal-frame starts
  if (!rc) rc = ensure_frames(B, st);
  if (rc) return rc;
  const int64_t n_items = n_pairs * cfg->starts;
  float4* pts = nullptr;
  float* poses = nullptr;
  float* values = nullptr;
  int32_t* ia2 = nullptr;
  int32_t* ib2 = nullptr;
  double* est = nullptr;
  double* se = nullptr;
  unsigned long long* queue = nullptr;
  auto release = [&]() {
    for (void* p : {(void*)pts, (void*)poses, (void*)values, (void*)ia2, (void*)ib2, (void*)est, (void*)se,
                    (void*)queue})
      if (p) cudaFreeAsync(p, st);
  };
  cudaError_t e = dev_alloc((void**)&pts, sizeof(float4) * cfg->n_crn, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&poses, sizeof(float) * 7 * n_items, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&values, sizeof(float) * n_items, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&ia2, sizeof(int32_t) * n_items, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&ib2, sizeof(int32_t) * n_items, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&est, sizeof(double) * 2 * n_items, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&se, sizeof(double) * 2 * n_items, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&queue, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) { release(); return cuda_fail(e, "align_rigid: scratch"); }
  shp_mc mc{cfg->seed, cfg->stream, cfg->n_crn, cfg->crn_flags & SHP_ANTITHETIC};
  rc = align_crn_points(Q, iq, &mc, reinterpret_cast<float*>(pts), stream);
  if (rc) { release(); return rc; }
  AdamArgs a{};
  a.Q = view(Q);
  a.B = view(B);
  a.iq = iq;
  a.ib = ib;
  a.n_pairs = n_pairs;
  a.starts = (int)cfg->starts;
  a.steps = (int)cfg->steps;
  a.objective = (int)cfg->objective;
  a.pts = pts;
  a.n_pts = cfg->objective == SHP_OBJ_FO_CLOSED ? 0 : (int)cfg->n_crn;
  a.scale_n = cfg->objective == SHP_OBJ_FO_CLOSED ? 0u : cfg->n_crn;
  a.lr = cfg->lr;
  a.lr_t = cfg->lr_t;
  a.beta1 = cfg->beta1;
  a.beta2 = cfg->beta2;
  a.eps = cfg->eps;
  a.key = Key{(uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32)};
  a.stream = cfg->stream;
  a.pose_out = poses;
  a.value_out = values;
  a.queue = queue;
  e = cudaFuncSetAttribute(align_adam_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAlignSmem);
  int sms = 0, dev = 0, per_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, align_adam_kernel, kAlignThreads, kAlignSmem);
  if (e != cudaSuccess) { release(); return cuda_fail(e, "align_rigid: launch set-up"); }
  int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  const int64_t need = (n_items + kAlignWarps - 1) / kAlignWarps;
  if (need < grid) grid = need;
  align_adam_kernel<<<(unsigned)grid, kAlignThreads, kAlignSmem, st>>>(a);
  e = cudaGetLastError();
  if (e == cudaSuccess && pose_starts)
    e = cudaMemcpyAsync(pose_starts, poses, sizeof(float) * 7 * n_items, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) { release(); return cuda_fail(e, "align_rigid: optimiser launch"); }
  pair_index_kernel<<<(unsigned)((n_items + 255) / 256), 256, 0, st>>>(n_pairs, (int)cfg->starts, iq, ib, ia2, ib2);
  shp_mc score{cfg->seed ^ 0x5DEECE66Dull, cfg->stream, cfg->n_score, SHP_SYMMETRIC};
  // every start of a pair is scored on the same random numbers (stream base
  // + pair), so that the choice between starts is not decided by
  // independent sampling noise
  rc = overlap_estimate_grouped(Q, ia2, B, ib2, n_items, poses, &score, est, se, cfg->starts, st);
  if (rc) { release(); return rc; }
  select_best_kernel<<<(unsigned)((n_pairs + 255) / 256), 256, 0, st>>>(n_pairs, (int)cfg->starts, est, self_q, iq,
                                                                         self_db, B->n_mol, ib, poses, pose_out,
                                                                         T_out, T_starts);
  e = cudaGetLastError();
  release();
  if (e != cudaSuccess) return cuda_fail(e, "align_rigid: selection launch");
  return SHP_OK;
}
