/*
 * FP64 CPU oracle for importance-sampling estimation of Gaussian molecular
 * shape overlap (Tuzharov, Bochenkova, Maximov, arXiv 2607.20766).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it. It shares no code, header, table or constant
 * generator with the CUDA library; both sides were written independently
 * from the paper and from the stream/sampler conventions stated below.
 *
 * What it computes, each in plain double precision, in the paper's order:
 *   - atomic Gaussians g_i(r) = p_i exp(-alpha_i |r - c_i|^2)      (Eq. occ)
 *   - union occupancy u(r) = 1 - prod_i (1 - g_i(r))              (Eq. union)
 *   - first-order sum m(r) = sum_i g_i(r)                      (Sec. FO, Eq. fo)
 *   - the mixture proposal q = m/Z, Z = sum_i p_i (pi/alpha_i)^{3/2}, drawn
 *     exactly: component i with probability v_i/Z, then a normal offset of
 *     variance 1/(2 alpha_i) per axis                    (Eq. expectation)
 *   - IS estimators Z * mean(f) with f = m_B (first order) or
 *     f = (u_A/m_A) u_B (union), sample-variance standard errors (Eq. var,
 *     Eq. union-is), the symmetrised average over both proposals, the
 *     Tanimoto and its delta-method SE (Sec. confidence-bounded screening)
 *   - exact targets: the first-order closed form (Eq. fo), the full
 *     inclusion-exclusion series (Eq. incexc) for union volumes and union
 *     overlaps, and midpoint-rule grid quadrature of Eq. union-overlap.
 *
 * Conventions the paper leaves open (shared with the CUDA path as a written
 * specification, implemented separately on each side):
 *   - alpha_i = c_alpha / R_i^2 (default c_alpha = 2.41798793), height p_i
 *     (default 2 sqrt 2); v_i = p_i * t * sqrt(t) with t = pi / alpha_i;
 *     Z = sum of v_i in atom order.
 *   - Component choice: integer Vose alias table. Masses
 *     M_i = floor((v_i / Z) * N 2^32), remainder added to the last atom;
 *     FIFO small/large worklists in atom order; the front large atom stays
 *     at the front until it turns small. A 32-bit word x picks column
 *     j = hi32(x N), then atom j if lo32(x N) < thr_j else alias_j.
 *   - Random words: Philox4x32-10 (Salmon et al., SC'11), key =
 *     (seed lo, seed hi), counter = (block, stream lo, stream hi, tag).
 *     Sample pair s uses blocks 2s and 2s+1 (words w0..w7): sample 2s takes
 *     w0 for the component and normals (n0, n1, n4); sample 2s+1 takes w1
 *     and (n2, n3, n5), where (n0,n1) = BM(w2,w3), (n2,n3) = BM(w4,w5),
 *     (n4,n5) = BM(w6,w7). BM(a,b): u1 = ((a>>8)+1) 2^-24, t = 2((b>>8)
 *     2^-24) - 1, rho = sqrt(-2 ln u1), (rho cos(pi t), rho sin(pi t)).
 *     Antithetic mode: sample 2s+1 is the reflection c_i - sigma_i z of
 *     sample 2s, and the pair mean is the statistical unit.
 *   - Tags: 0 = samples from A (A->B), 1 = samples from B (B->A), 2 = a
 *     molecule's own volume / self-overlap.
 *   - SE uses the n-1 sample variance; the symmetrised SE is
 *     0.5 sqrt(SE_AB^2 + SE_BA^2) (independent streams per direction).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_MAXN 64

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ERANGE = -4 };
enum { ORC_SYMMETRIC = 1u, ORC_ANTITHETIC = 2u };
enum { ORC_TAG_AB = 0u, ORC_TAG_BA = 1u, ORC_TAG_SELF = 2u, ORC_TAG_FIT = 6u };

/* A set of molecules as flat arrays (host). p may be NULL (2 sqrt 2). */
typedef struct {
  const float* xyz;       /* [n_atoms][3] */
  const float* radius;    /* [n_atoms] */
  const float* height;    /* [n_atoms] or NULL */
  const int32_t* offsets; /* [n_mol + 1] */
  int32_t n_mol;
  double c_alpha;         /* <= 0 means 2.41798793 */
} orc_set;

/* One molecule, expanded to double precision. */
typedef struct {
  int n;
  double c[ORC_MAXN][3];
  double alpha[ORC_MAXN];
  double p[ORC_MAXN];
  double sigma[ORC_MAXN];
  double v[ORC_MAXN];
  double Z;
  uint32_t thr[ORC_MAXN];
  uint8_t alias[ORC_MAXN];
} orc_mol;

/* ------------------------------------------------------------------ */
/* Philox4x32-10                                                       */
/* ------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)prod1;
    uint32_t y2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)prod0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Box-Muller on two 32-bit words, as specified in the header comment. */
void orc_normal_pair(uint32_t a, uint32_t b, double out[2]) {
  double u1 = (double)((a >> 8) + 1u) * (1.0 / 16777216.0);
  double t = 2.0 * ((double)(b >> 8) * (1.0 / 16777216.0)) - 1.0;
  double rho = sqrt(-2.0 * log(u1));
  out[0] = rho * cos(ORC_PI * t);
  out[1] = rho * sin(ORC_PI * t);
}

/* ------------------------------------------------------------------ */
/* Mixture weights and alias tables                                    */
/* ------------------------------------------------------------------ */

/* Integer Vose alias table from positive weights v[0..n-1]. */
int orc_alias_build(int n, const double* v, uint32_t* thr, uint8_t* alias, uint64_t* mass_out) {
  if (n < 1 || n > ORC_MAXN) return ORC_ERANGE;
  const uint64_t ONE = (uint64_t)1 << 32;
  uint64_t M[ORC_MAXN];
  double Z = 0.0;
  for (int i = 0; i < n; ++i) {
    if (!(v[i] > 0.0)) return ORC_EINVAL;
    Z += v[i];
  }
  const double scale = (double)n * 4294967296.0;
  uint64_t total = 0;
  for (int i = 0; i < n; ++i) {
    M[i] = (uint64_t)floor((v[i] / Z) * scale);
    total += M[i];
  }
  M[n - 1] += (uint64_t)n * ONE - total;
  if (mass_out) memcpy(mass_out, M, sizeof(uint64_t) * (size_t)n);
  int small[ORC_MAXN], large[ORC_MAXN];
  int s_head = 0, s_tail = 0, l_head = 0, l_tail = 0;
  for (int i = 0; i < n; ++i) {
    if (M[i] < ONE) small[s_tail++] = i;
    else large[l_tail++] = i;
  }
  while (s_head < s_tail && l_head < l_tail) {
    int s = small[s_head++];
    int l = large[l_head];
    thr[s] = (uint32_t)M[s];
    alias[s] = (uint8_t)l;
    M[l] -= ONE - M[s];
    if (M[l] < ONE) {
      ++l_head;
      small[s_tail++] = l;
    }
  }
  while (s_head < s_tail) { int s = small[s_head++]; thr[s] = 0xFFFFFFFFu; alias[s] = (uint8_t)s; }
  while (l_head < l_tail) { int l = large[l_head++]; thr[l] = 0xFFFFFFFFu; alias[l] = (uint8_t)l; }
  return ORC_OK;
}

static int load_mol(const orc_set* S, int32_t idx, const float* pose, orc_mol* m) {
  if (idx < 0 || idx >= S->n_mol) return ORC_EINVAL;
  int32_t a0 = S->offsets[idx], a1 = S->offsets[idx + 1];
  int n = a1 - a0;
  if (n < 1 || n > ORC_MAXN) return ORC_ERANGE;
  double ca = S->c_alpha > 0 ? S->c_alpha : 2.41798793;
  double R[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, t[3] = {0, 0, 0};
  if (pose) {
    double w = pose[0], x = pose[1], y = pose[2], z = pose[3];
    double nq = sqrt(w * w + x * x + y * y + z * z);
    if (!(nq > 0)) return ORC_EINVAL;
    w /= nq; x /= nq; y /= nq; z /= nq;
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
    t[0] = pose[4]; t[1] = pose[5]; t[2] = pose[6];
  }
  m->n = n;
  m->Z = 0.0;
  for (int i = 0; i < n; ++i) {
    const float* c = S->xyz + 3 * (size_t)(a0 + i);
    double c0 = c[0], c1 = c[1], c2 = c[2];
    for (int k = 0; k < 3; ++k) m->c[i][k] = R[k][0] * c0 + R[k][1] * c1 + R[k][2] * c2 + t[k];
    double r = S->radius[a0 + i];
    if (!(r > 0)) return ORC_EINVAL;
    m->alpha[i] = ca / (r * r);
    m->p[i] = S->height ? (double)S->height[a0 + i] : 2.0 * sqrt(2.0);
    m->sigma[i] = 1.0 / sqrt(2.0 * m->alpha[i]);
    double tt = ORC_PI / m->alpha[i];
    m->v[i] = m->p[i] * tt * sqrt(tt);
    m->Z += m->v[i];
  }
  return orc_alias_build(n, m->v, m->thr, m->alias, NULL);
}

/* Per-molecule tables (for cross-checking the library's own tables). */
int orc_mol_tables(const orc_set* S, int32_t idx, double* alpha, double* v, double* Z,
                   uint32_t* thr, uint8_t* alias) {
  orc_mol m;
  int rc = load_mol(S, idx, NULL, &m);
  if (rc) return rc;
  for (int i = 0; i < m.n; ++i) {
    if (alpha) alpha[i] = m.alpha[i];
    if (v) v[i] = m.v[i];
    if (thr) thr[i] = m.thr[i];
    if (alias) alias[i] = m.alias[i];
  }
  if (Z) *Z = m.Z;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Sampling from the mixture q = m / Z (Eq. expectation)               */
/* ------------------------------------------------------------------ */

static int pick_component(const orc_mol* m, uint32_t x) {
  uint64_t prod = (uint64_t)x * (uint64_t)m->n;
  uint32_t j = (uint32_t)(prod >> 32), f = (uint32_t)prod;
  return f < m->thr[j] ? (int)j : (int)m->alias[j];
}

/* Samples 2s and 2s+1 of stream (seed, stream, tag) drawn from molecule m. */
static void draw_pair(const orc_mol* m, uint64_t seed, uint64_t stream, uint32_t tag, uint32_t s,
                      int antithetic, double r0[3], double r1[3], int* i0, int* i1) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t c[4] = {2u * s, (uint32_t)stream, (uint32_t)(stream >> 32), tag};
  uint32_t w[8];
  orc_philox4x32_10(c, key, w);
  c[0] = 2u * s + 1u;
  orc_philox4x32_10(c, key, w + 4);
  double n01[2], n23[2], n45[2];
  orc_normal_pair(w[2], w[3], n01);
  orc_normal_pair(w[4], w[5], n23);
  orc_normal_pair(w[6], w[7], n45);
  int a = pick_component(m, w[0]);
  double z0[3] = {n01[0], n01[1], n45[0]};
  for (int k = 0; k < 3; ++k) r0[k] = m->c[a][k] + m->sigma[a] * z0[k];
  *i0 = a;
  if (antithetic) {
    for (int k = 0; k < 3; ++k) r1[k] = m->c[a][k] - m->sigma[a] * z0[k];
    *i1 = a;
  } else {
    int b = pick_component(m, w[1]);
    double z1[3] = {n23[0], n23[1], n45[1]};
    for (int k = 0; k < 3; ++k) r1[k] = m->c[b][k] + m->sigma[b] * z1[k];
    *i1 = b;
  }
}

/* Draw n samples of one stream (for sampler tests): r[n][3], comp[n]. */
int orc_draw(const orc_set* S, int32_t idx, uint64_t seed, uint64_t stream, uint32_t tag,
             int64_t n, int antithetic, double* r, int32_t* comp) {
  orc_mol m;
  int rc = load_mol(S, idx, NULL, &m);
  if (rc) return rc;
  for (int64_t k = 0; k < n; k += 2) {
    double a[3], b[3];
    int ia, ib;
    draw_pair(&m, seed, stream, tag, (uint32_t)(k / 2), antithetic, a, b, &ia, &ib);
    memcpy(r + 3 * k, a, sizeof a);
    if (comp) comp[k] = ia;
    if (k + 1 < n) {
      memcpy(r + 3 * (k + 1), b, sizeof b);
      if (comp) comp[k + 1] = ib;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Occupancies (Eq. occ, Eq. union, first-order sum)                   */
/* ------------------------------------------------------------------ */

static void occupancy(const orc_mol* m, const double r[3], double* msum, double* u) {
  double s = 0.0, prod = 1.0;
  for (int i = 0; i < m->n; ++i) {
    double dx = r[0] - m->c[i][0], dy = r[1] - m->c[i][1], dz = r[2] - m->c[i][2];
    double g = m->p[i] * exp(-m->alpha[i] * (dx * dx + dy * dy + dz * dz));
    s += g;
    prod *= 1.0 - g;
  }
  *msum = s;
  *u = 1.0 - prod;
}

/* Evaluate m and u of a set member at points r[n][3] (test helper). */
int orc_occupancy(const orc_set* S, int32_t idx, const float* pose, int64_t n, const double* r,
                  double* msum, double* u) {
  orc_mol m;
  int rc = load_mol(S, idx, pose, &m);
  if (rc) return rc;
  for (int64_t k = 0; k < n; ++k) occupancy(&m, r + 3 * k, msum + k, u + k);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* IS sums for one direction: samples from X, other molecule Y         */
/* sums = {sum f_FO, sum f_FO^2, sum f_U, sum f_U^2}, unit count n_eff   */
/* ------------------------------------------------------------------ */

/* u~(r) = sum_i w_i g_i(r), the weighted-Gaussian control variate of u. */
static double weighted_sum(const orc_mol* m, const double* w, const double r[3]) {
  double s = 0.0;
  for (int i = 0; i < m->n; ++i) {
    double dx = r[0] - m->c[i][0], dy = r[1] - m->c[i][1], dz = r[2] - m->c[i][2];
    s += w[i] * m->p[i] * exp(-m->alpha[i] * (dx * dx + dy * dy + dz * dz));
  }
  return s;
}

/*
 * wx, wy: per-atom control-variate weights of X and Y, or NULL. With them
 * the union value is the residual (u_X u_Y - u~_X u~_Y) / m_X, whose
 * expectation is the union overlap minus the closed form of
 * integral u~_X u~_Y.
 */
static void sums_cross(const orc_mol* X, const orc_mol* Y, uint64_t seed, uint64_t stream,
                       uint32_t tag, uint32_t n, int antithetic, const double* wx, const double* wy,
                       double sums[4], double* n_eff) {
  double s[4] = {0, 0, 0, 0};
  for (uint32_t k = 0; k < n; k += 2) {
    double r[2][3];
    int ia, ib;
    draw_pair(X, seed, stream, tag, k / 2, antithetic, r[0], r[1], &ia, &ib);
    double ffo[2], fu[2];
    int cnt = (k + 1 < n) ? 2 : 1;
    for (int j = 0; j < cnt; ++j) {
      double mx, ux, my, uy;
      occupancy(X, r[j], &mx, &ux);
      occupancy(Y, r[j], &my, &uy);
      ffo[j] = my;                 /* first order: f = m_Y        */
      if (wx && wy)                /* union residual (control variate) */
        fu[j] = (ux * uy - weighted_sum(X, wx, r[j]) * weighted_sum(Y, wy, r[j])) / mx;
      else
        fu[j] = (ux / mx) * uy;    /* union: f = w_X u_Y, w = u/m */
    }
    if (antithetic) {
      double g0 = 0.5 * (ffo[0] + ffo[1]), g1 = 0.5 * (fu[0] + fu[1]);
      s[0] += g0; s[1] += g0 * g0; s[2] += g1; s[3] += g1 * g1;
    } else {
      for (int j = 0; j < cnt; ++j) {
        s[0] += ffo[j]; s[1] += ffo[j] * ffo[j]; s[2] += fu[j]; s[3] += fu[j] * fu[j];
      }
    }
  }
  memcpy(sums, s, sizeof s);
  *n_eff = antithetic ? (double)(n / 2) : (double)n;
}

/* Own volume and union self-overlap of X: f_V = u/m, f_S = u^2/m. */
static void sums_self(const orc_mol* X, uint64_t seed, uint64_t stream, uint32_t n, int antithetic,
                      double sums[4], double* n_eff) {
  double s[4] = {0, 0, 0, 0};
  for (uint32_t k = 0; k < n; k += 2) {
    double r[2][3];
    int ia, ib;
    draw_pair(X, seed, stream, ORC_TAG_SELF, k / 2, antithetic, r[0], r[1], &ia, &ib);
    double fv[2], fs[2];
    int cnt = (k + 1 < n) ? 2 : 1;
    for (int j = 0; j < cnt; ++j) {
      double mx, ux;
      occupancy(X, r[j], &mx, &ux);
      fv[j] = ux / mx;
      fs[j] = ux * ux / mx;
    }
    if (antithetic) {
      double g0 = 0.5 * (fv[0] + fv[1]), g1 = 0.5 * (fs[0] + fs[1]);
      s[0] += g0; s[1] += g0 * g0; s[2] += g1; s[3] += g1 * g1;
    } else {
      for (int j = 0; j < cnt; ++j) {
        s[0] += fv[j]; s[1] += fv[j] * fv[j]; s[2] += fs[j]; s[3] += fs[j] * fs[j];
      }
    }
  }
  memcpy(sums, s, sizeof s);
  *n_eff = antithetic ? (double)(n / 2) : (double)n;
}

/* Z * mean and Z * sqrt(s^2 / n) with the n-1 sample variance (Eq. var). */
static void finish(double Z, double sum, double sum2, double n, double* est, double* se) {
  double mean = sum / n;
  double var = n > 1 ? (sum2 - sum * mean) / (n - 1.0) : 0.0;
  if (var < 0) var = 0;
  *est = Z * mean;
  *se = Z * sqrt(var / n);
}

/* Raw one-direction sums (test helper): samples from A[ia] (tag 0) or from
 * posed B[ib] (tag 1). */
int orc_direction_sums(const orc_set* A, int32_t ia, const orc_set* B, int32_t ib,
                       const float* poseB, uint64_t seed, uint64_t stream, uint32_t tag, uint32_t n,
                       uint32_t flags, double sums[4], double* n_eff) {
  orc_mol ma, mb;
  int rc = load_mol(A, ia, NULL, &ma);
  if (!rc) rc = load_mol(B, ib, poseB, &mb);
  if (rc) return rc;
  if (tag == ORC_TAG_BA)
    sums_cross(&mb, &ma, seed, stream, tag, n, (flags & ORC_ANTITHETIC) != 0, NULL, NULL, sums, n_eff);
  else
    sums_cross(&ma, &mb, seed, stream, tag, n, (flags & ORC_ANTITHETIC) != 0, NULL, NULL, sums, n_eff);
  return ORC_OK;
}

static int nthreads_set(int n_threads) {
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
  return omp_get_max_threads();
#else
  (void)n_threads;
  return 1;
#endif
}

/*
 * Pair overlaps: est[n_pairs][2], se[n_pairs][2] with slot 0 = first order,
 * slot 1 = union. Pair k uses stream stream_base + k. With ORC_SYMMETRIC
 * both directions are estimated and averaged; otherwise only A->B.
 */
int orc_overlap_estimate(const orc_set* A, const int32_t* ia, const orc_set* B, const int32_t* ib,
                         int64_t n_pairs, const float* poses, uint64_t seed, uint64_t stream_base,
                         uint32_t n, uint32_t flags, double* est, double* se, int n_threads) {
  if (n < 2 || n_pairs < 0) return ORC_EINVAL;
  if ((flags & ORC_ANTITHETIC) && (n & 1u)) return ORC_EINVAL;
  nthreads_set(n_threads);
  int err = 0;
  const int anti = (flags & ORC_ANTITHETIC) != 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int64_t k = 0; k < n_pairs; ++k) {
    orc_mol ma, mb;
    if (load_mol(A, ia[k], NULL, &ma) || load_mol(B, ib[k], poses ? poses + 7 * k : NULL, &mb)) {
      err |= 1;
      continue;
    }
    uint64_t stream = stream_base + (uint64_t)k;
    double s[4], ne, e_fo, s_fo, e_u, s_u;
    sums_cross(&ma, &mb, seed, stream, ORC_TAG_AB, n, anti, NULL, NULL, s, &ne);
    finish(ma.Z, s[0], s[1], ne, &e_fo, &s_fo);
    finish(ma.Z, s[2], s[3], ne, &e_u, &s_u);
    if (flags & ORC_SYMMETRIC) {
      double e2_fo, s2_fo, e2_u, s2_u;
      sums_cross(&mb, &ma, seed, stream, ORC_TAG_BA, n, anti, NULL, NULL, s, &ne);
      finish(mb.Z, s[0], s[1], ne, &e2_fo, &s2_fo);
      finish(mb.Z, s[2], s[3], ne, &e2_u, &s2_u);
      e_fo = 0.5 * (e_fo + e2_fo);
      s_fo = 0.5 * sqrt(s_fo * s_fo + s2_fo * s2_fo);
      e_u = 0.5 * (e_u + e2_u);
      s_u = 0.5 * sqrt(s_u * s_u + s2_u * s2_u);
    }
    est[2 * k] = e_fo; se[2 * k] = s_fo;
    est[2 * k + 1] = e_u; se[2 * k + 1] = s_u;
  }
  return err ? ORC_EINVAL : ORC_OK;
}

/*
 * Union volume V = Z E_q[u/m] (Eq. expectation with f = u/m) and union
 * self-overlap O_XX = Z E_q[u^2/m] (Eq. union-is with B = A) of molecules
 * idx[0..n-1]; molecule k uses stream stream_base + k, tag 2.
 */
int orc_union_volume_estimate(const orc_set* S, const int32_t* idx, int64_t n_mol, uint64_t seed,
                              uint64_t stream_base, uint32_t n, uint32_t flags, double* vol,
                              double* vol_se, double* self_ov, double* self_se, int n_threads) {
  if (n < 2 || n_mol < 0) return ORC_EINVAL;
  if ((flags & ORC_ANTITHETIC) && (n & 1u)) return ORC_EINVAL;
  nthreads_set(n_threads);
  int err = 0;
  const int anti = (flags & ORC_ANTITHETIC) != 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int64_t k = 0; k < n_mol; ++k) {
    orc_mol m;
    if (load_mol(S, idx ? idx[k] : (int32_t)k, NULL, &m)) { err |= 1; continue; }
    double s[4], ne, e, sd;
    sums_self(&m, seed, stream_base + (uint64_t)k, n, anti, s, &ne);
    finish(m.Z, s[0], s[1], ne, &e, &sd);
    vol[k] = e;
    if (vol_se) vol_se[k] = sd;
    finish(m.Z, s[2], s[3], ne, &e, &sd);
    if (self_ov) self_ov[k] = e;
    if (self_se) self_se[k] = sd;
  }
  return err ? ORC_EINVAL : ORC_OK;
}

/* ------------------------------------------------------------------ */
/* First-order closed form (Eq. fo, with heights p_i p_j)              */
/* ------------------------------------------------------------------ */

/* sum_ij wa_i wb_j integral g_i g_j (Eq. fo); wa, wb NULL = unit weights. */
static double fo_closed_w(const orc_mol* a, const double* wa, const orc_mol* b, const double* wb) {
  double s = 0.0;
  for (int i = 0; i < a->n; ++i)
    for (int j = 0; j < b->n; ++j) {
      double ai = a->alpha[i], bj = b->alpha[j], sum = ai + bj;
      double dx = a->c[i][0] - b->c[j][0], dy = a->c[i][1] - b->c[j][1], dz = a->c[i][2] - b->c[j][2];
      double t = ORC_PI / sum;
      double w = (wa ? wa[i] : 1.0) * (wb ? wb[j] : 1.0);
      s += w * a->p[i] * b->p[j] * t * sqrt(t) * exp(-ai * bj / sum * (dx * dx + dy * dy + dz * dz));
    }
  return s;
}

static double fo_closed(const orc_mol* a, const orc_mol* b) { return fo_closed_w(a, NULL, b, NULL); }

int orc_fo_overlap(const orc_set* A, const int32_t* ia, const orc_set* B, const int32_t* ib,
                   int64_t n_pairs, const float* poses, double* out, int n_threads) {
  nthreads_set(n_threads);
  int err = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : err)
  for (int64_t k = 0; k < n_pairs; ++k) {
    orc_mol ma, mb;
    if (load_mol(A, ia[k], NULL, &ma) || load_mol(B, ib[k], poses ? poses + 7 * k : NULL, &mb)) {
      err |= 1;
      continue;
    }
    out[k] = fo_closed(&ma, &mb);
  }
  return err ? ORC_EINVAL : ORC_OK;
}

/* Z of each molecule (= its first-order volume, the integral of m). */
int orc_mixture_mass(const orc_set* S, const int32_t* idx, int64_t n_mol, double* Z) {
  for (int64_t k = 0; k < n_mol; ++k) {
    orc_mol m;
    int rc = load_mol(S, idx ? idx[k] : (int32_t)k, NULL, &m);
    if (rc) return rc;
    Z[k] = m.Z;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Inclusion-exclusion (Eq. incexc) -- exact union volume / overlap    */
/* ------------------------------------------------------------------ */

/* Product of the Gaussians of one subset: p = prod p_i, a = sum alpha_i,
 * b = sum alpha_i c_i, c = sum alpha_i |c_i|^2; its integral is
 * p (pi/a)^{3/2} exp(-(c - |b|^2 / a)). */
typedef struct { double p, a, b[3], c; int sign; } orc_subset;

static orc_subset* subsets_of(const orc_mol* m) {
  size_t ns = (size_t)1 << m->n;
  orc_subset* T = (orc_subset*)malloc(ns * sizeof(orc_subset));
  if (!T) return NULL;
  T[0].p = 1.0; T[0].a = 0.0; T[0].b[0] = T[0].b[1] = T[0].b[2] = 0.0; T[0].c = 0.0; T[0].sign = 1;
  for (size_t s = 1; s < ns; ++s) {
    int i = __builtin_ctzll((unsigned long long)s);
    const orc_subset* pr = &T[s & (s - 1)];
    orc_subset* q = &T[s];
    double al = m->alpha[i];
    q->p = pr->p * m->p[i];
    q->a = pr->a + al;
    for (int k = 0; k < 3; ++k) q->b[k] = pr->b[k] + al * m->c[i][k];
    q->c = pr->c + al * (m->c[i][0] * m->c[i][0] + m->c[i][1] * m->c[i][1] + m->c[i][2] * m->c[i][2]);
    q->sign = -pr->sign;
  }
  return T;
}

static double subset_integral(double p, double a, const double b[3], double c) {
  double t = ORC_PI / a;
  double e = c - (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]) / a;
  return p * t * sqrt(t) * exp(-e);
}

/* Neumaier compensated summation. */
typedef struct { double s, c; } orc_acc;
static void acc_add(orc_acc* A, double x) {
  double t = A->s + x;
  if (fabs(A->s) >= fabs(x)) A->c += (A->s - t) + x;
  else A->c += (x - t) + A->s;
  A->s = t;
}

/* V = sum over non-empty subsets S of (-1)^{|S|+1} I(S). */
int orc_union_volume_ie(const orc_set* S, int32_t idx, double* V) {
  orc_mol m;
  int rc = load_mol(S, idx, NULL, &m);
  if (rc) return rc;
  if (m.n > 26) return ORC_ERANGE;
  orc_subset* T = subsets_of(&m);
  if (!T) return ORC_EINVAL;
  size_t ns = (size_t)1 << m.n;
  orc_acc acc = {0, 0};
  for (size_t s = 1; s < ns; ++s) acc_add(&acc, -(double)T[s].sign * subset_integral(T[s].p, T[s].a, T[s].b, T[s].c));
  free(T);
  *V = acc.s + acc.c;
  return ORC_OK;
}

/* O_AB = integral of u_A u_B = sum over non-empty S in A, T in B of
 * (-1)^{|S|+|T|} I(S + T), S and T taken as disjoint atom multisets. */
int orc_union_overlap_ie(const orc_set* A, int32_t ia, const orc_set* B, int32_t ib,
                         const float* poseB, double* O, int n_threads) {
  orc_mol ma, mb;
  int rc = load_mol(A, ia, NULL, &ma);
  if (!rc) rc = load_mol(B, ib, poseB, &mb);
  if (rc) return rc;
  if (ma.n > 20 || mb.n > 20) return ORC_ERANGE;
  orc_subset* TA = subsets_of(&ma);
  orc_subset* TB = subsets_of(&mb);
  if (!TA || !TB) { free(TA); free(TB); return ORC_EINVAL; }
  nthreads_set(n_threads);
  int64_t na = (int64_t)1 << ma.n, nb = (int64_t)1 << mb.n;
  double total_s = 0.0, total_c = 0.0;
#pragma omp parallel
  {
    orc_acc acc = {0, 0};
#pragma omp for schedule(dynamic, 16)
    for (int64_t s = 1; s < na; ++s) {
      const orc_subset* x = &TA[s];
      for (int64_t t = 1; t < nb; ++t) {
        const orc_subset* y = &TB[t];
        double b[3] = {x->b[0] + y->b[0], x->b[1] + y->b[1], x->b[2] + y->b[2]};
        double v = subset_integral(x->p * y->p, x->a + y->a, b, x->c + y->c);
        acc_add(&acc, (double)(x->sign * y->sign) * v);
      }
    }
#pragma omp critical
    { total_s += acc.s; total_c += acc.c; }
  }
  free(TA);
  free(TB);
  *O = total_s + total_c;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Grid quadrature of Eq. union-overlap (independent ground truth)     */
/* ------------------------------------------------------------------ */

/*
 * Midpoint rule with spacing h over the joint bounding box of the centres
 * padded by pad. out = {V_A, V_B, O_AB (union), O_AB (first order),
 * integral of m_A, integral of u_A^2}. With nB == 0 only A's entries are
 * meaningful. The Gaussians are separable, so each atom keeps three 1-D
 * tables of exp(-alpha (x - c)^2).
 */
int orc_grid(const orc_set* A, int32_t ia, const orc_set* B, int32_t ib, const float* poseB,
             double h, double pad, double out[6], int n_threads) {
  orc_mol ma, mb;
  int rc = load_mol(A, ia, NULL, &ma);
  if (rc) return rc;
  int have_b = B != NULL;
  if (have_b && (rc = load_mol(B, ib, poseB, &mb))) return rc;
  if (!have_b) mb.n = 0;
  if (!(h > 0) || !(pad >= 0)) return ORC_EINVAL;
  double lo[3], hi[3];
  for (int k = 0; k < 3; ++k) { lo[k] = 1e300; hi[k] = -1e300; }
  for (int i = 0; i < ma.n; ++i)
    for (int k = 0; k < 3; ++k) { lo[k] = fmin(lo[k], ma.c[i][k]); hi[k] = fmax(hi[k], ma.c[i][k]); }
  for (int i = 0; i < mb.n; ++i)
    for (int k = 0; k < 3; ++k) { lo[k] = fmin(lo[k], mb.c[i][k]); hi[k] = fmax(hi[k], mb.c[i][k]); }
  int np[3];
  for (int k = 0; k < 3; ++k) {
    lo[k] -= pad; hi[k] += pad;
    np[k] = (int)ceil((hi[k] - lo[k]) / h);
  }
  int nat = ma.n + mb.n;
  double* tab[3];
  for (int k = 0; k < 3; ++k) {
    tab[k] = (double*)malloc(sizeof(double) * (size_t)nat * (size_t)np[k]);
    if (!tab[k]) return ORC_EINVAL;
    for (int a = 0; a < nat; ++a) {
      const double* c = a < ma.n ? ma.c[a] : mb.c[a - ma.n];
      double al = a < ma.n ? ma.alpha[a] : mb.alpha[a - ma.n];
      for (int i = 0; i < np[k]; ++i) {
        double x = lo[k] + (i + 0.5) * h - c[k];
        tab[k][(size_t)a * np[k] + i] = exp(-al * x * x);
      }
    }
  }
  nthreads_set(n_threads);
  double sums[6] = {0, 0, 0, 0, 0, 0};
#pragma omp parallel
  {
    double loc[6] = {0, 0, 0, 0, 0, 0};
    double pxy[2 * ORC_MAXN];
#pragma omp for schedule(dynamic, 1)
    for (int ix = 0; ix < np[0]; ++ix) {
      for (int iy = 0; iy < np[1]; ++iy) {
        for (int a = 0; a < nat; ++a) {
          double p = a < ma.n ? ma.p[a] : mb.p[a - ma.n];
          pxy[a] = p * tab[0][(size_t)a * np[0] + ix] * tab[1][(size_t)a * np[1] + iy];
        }
        double row[6] = {0, 0, 0, 0, 0, 0};
        for (int iz = 0; iz < np[2]; ++iz) {
          double mA = 0, qA = 1, mB = 0, qB = 1;
          for (int a = 0; a < ma.n; ++a) {
            double g = pxy[a] * tab[2][(size_t)a * np[2] + iz];
            mA += g; qA *= 1.0 - g;
          }
          for (int a = ma.n; a < nat; ++a) {
            double g = pxy[a] * tab[2][(size_t)a * np[2] + iz];
            mB += g; qB *= 1.0 - g;
          }
          double uA = 1.0 - qA, uB = 1.0 - qB;
          row[0] += uA; row[1] += uB; row[2] += uA * uB; row[3] += mA * mB; row[4] += mA;
          row[5] += uA * uA;
        }
        for (int t = 0; t < 6; ++t) loc[t] += row[t];
      }
    }
#pragma omp critical
    for (int t = 0; t < 6; ++t) sums[t] += loc[t];
  }
  double dv = h * h * h;
  for (int t = 0; t < 6; ++t) out[t] = sums[t] * dv;
  for (int k = 0; k < 3; ++k) free(tab[k]);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Fixed-budget Tanimoto screen (Sec. confidence-bounded screening)    */
/* ------------------------------------------------------------------ */

/*
 * Pairs (Q[iq[k]], D[id[k]]), both directions, n samples each, streams
 * stream_ids[k]. selfQ / selfD hold each molecule's self-overlaps as
 * [slot 0 = first order, slot 1 = union] (indexed by iq[k] / id[k]).
 * Outputs (slot 0 first order, slot 1 union), each [n_pairs][2]:
 * O, seO, T = O / (S - O) with S = O_QQ + O_DD, seT = S / (S - O)^2 seO.
 *
 * selfQ_se / selfD_se (same layout as selfQ / selfD, or both NULL): the
 * standard errors of estimated self-overlaps. The self-overlaps then carry
 * their own sampling error into T, and seT is the full first-order (delta
 * method) propagation of all three independent estimates through
 * T(O, O_QQ, O_DD) = O / (O_QQ + O_DD - O):
 *   dT/dO = S / (S - O)^2,   dT/dO_QQ = dT/dO_DD = -O / (S - O)^2,
 *   seT^2 = (dT/dO)^2 seO^2 + (O / (S - O)^2)^2 (seQQ^2 + seDD^2).
 * The paper's formula (Sec. confidence-bounded screening) keeps only the
 * first term, i.e. treats the self-overlaps as exact.
 */
/*
 * omega_q, omega_d: per-atom control-variate weights of each set (set atom
 * order), or both NULL. With them the union slot is estimated as
 *   O_U = C + (Z_A mean_AB + Z_B mean_BA) / 2,
 *   C = sum_ij w_i w_j integral g_i g_j (closed form),
 * from the residual values of sums_cross: unbiased for any weights, since
 * E_q[u~_A u~_B / m_A] Z_A = C (a weighted first-order overlap). Not in the
 * paper: it applies the learned crowding weights of the volume control
 * variate to both molecules of a pair.
 */
int orc_tanimoto_pairs(const orc_set* Q, const int32_t* iq, const orc_set* D, const int32_t* id,
                       const uint64_t* stream_ids, int64_t n_pairs, const double* selfQ,
                       const double* selfD, const double* selfQ_se, const double* selfD_se, uint64_t seed,
                       uint32_t n, uint32_t flags,
                       const double* omega_q, const double* omega_d, double* O, double* seO, double* T,
                       double* seT, int n_threads) {
  if (n < 2) return ORC_EINVAL;
  if ((omega_q == NULL) != (omega_d == NULL)) return ORC_EINVAL;
  if ((selfQ_se == NULL) != (selfD_se == NULL)) return ORC_EINVAL;
  nthreads_set(n_threads);
  int err = 0;
  const int anti = (flags & ORC_ANTITHETIC) != 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int64_t k = 0; k < n_pairs; ++k) {
    orc_mol mq, md;
    if (load_mol(Q, iq[k], NULL, &mq) || load_mol(D, id[k], NULL, &md)) { err |= 1; continue; }
    const double* wq = omega_q ? omega_q + Q->offsets[iq[k]] : NULL;
    const double* wd = omega_d ? omega_d + D->offsets[id[k]] : NULL;
    double s[4], ne, e1[2], s1[2], e2[2], s2[2];
    sums_cross(&mq, &md, seed, stream_ids[k], ORC_TAG_AB, n, anti, wq, wd, s, &ne);
    finish(mq.Z, s[0], s[1], ne, &e1[0], &s1[0]);
    finish(mq.Z, s[2], s[3], ne, &e1[1], &s1[1]);
    sums_cross(&md, &mq, seed, stream_ids[k], ORC_TAG_BA, n, anti, wd, wq, s, &ne);
    finish(md.Z, s[0], s[1], ne, &e2[0], &s2[0]);
    finish(md.Z, s[2], s[3], ne, &e2[1], &s2[1]);
    const double C = wq ? fo_closed_w(&mq, wq, &md, wd) : 0.0;
    for (int slot = 0; slot < 2; ++slot) {
      double o = 0.5 * (e1[slot] + e2[slot]) + (slot == 1 ? C : 0.0);
      double so = 0.5 * sqrt(s1[slot] * s1[slot] + s2[slot] * s2[slot]);
      double S = selfQ[2 * (size_t)iq[k] + slot] + selfD[2 * (size_t)id[k] + slot];
      double den = S - o;
      O[2 * k + slot] = o;
      seO[2 * k + slot] = so;
      T[2 * k + slot] = o / den;
      double var_t = (S / (den * den)) * (S / (den * den)) * so * so;
      if (selfQ_se) {
        double sq = selfQ_se[2 * (size_t)iq[k] + slot], sd = selfD_se[2 * (size_t)id[k] + slot];
        double d_self = o / (den * den);
        var_t += d_self * d_self * (sq * sq + sd * sd);
      }
      seT[2 * k + slot] = sqrt(var_t);
    }
  }
  return err ? ORC_EINVAL : ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Rigid alignment (Sec. differentiable alignment, Eq. pose, Eq. grad) */
/* ------------------------------------------------------------------ */

/*
 * Common random numbers: n points drawn once from the query's mixture
 * (tag 3, the usual sample layout; antithetic: each odd point the reflection
 * of the even one about its component centre) with their union weights
 * w = u/m. points[n][4] = (x, y, z, w).
 */
int orc_crn_points(const orc_set* S, int32_t idx, uint64_t seed, uint64_t stream, uint32_t n, int antithetic,
                   double* points) {
  orc_mol m;
  int rc = load_mol(S, idx, NULL, &m);
  if (rc) return rc;
  for (uint32_t k = 0; k < n; k += 2) {
    double r[2][3];
    int i0, i1;
    draw_pair(&m, seed, stream, 3u, k / 2, antithetic, r[0], r[1], &i0, &i1);
    for (int j = 0; j < 2 && k + j < n; ++j) {
      double ms, u;
      occupancy(&m, r[j], &ms, &u);
      double* p = points + 4 * (size_t)(k + j);
      p[0] = r[j][0]; p[1] = r[j][1]; p[2] = r[j][2]; p[3] = u / ms;
    }
  }
  return ORC_OK;
}

/*
 * CRN objective of molecule B[ib] moved by pose (raw quaternion w,x,y,z,
 * normalised inside, then translation): objective 0 = first order,
 * F = (Z_Q / n) sum_k m_B(r_k); objective 1 = union (Eq. grad),
 * F = (Z_Q / n) sum_k w_k u_B(r_k).
 */
static double crn_objective(const orc_mol* mb, const double* points, uint32_t n, double ZQ, int objective) {
  double s = 0.0;
  for (uint32_t k = 0; k < n; ++k) {
    const double* p = points + 4 * (size_t)k;
    double m, u;
    occupancy(mb, p, &m, &u);
    s += objective == 0 ? m : p[3] * u;
  }
  return ZQ * s / (double)n;
}

int orc_pose_objective(double ZQ, const double* points, uint32_t n, const orc_set* B, int32_t ib,
                       const float* pose, int objective, double* F) {
  orc_mol mb;
  int rc = load_mol(B, ib, pose, &mb);
  if (rc) return rc;
  *F = crn_objective(&mb, points, n, ZQ, objective);
  return ORC_OK;
}

/* Pose from doubles (the float pose of load_mol would round the FD step). */
static int load_mol_posed_d(const orc_set* S, int32_t idx, const double pose[7], orc_mol* m) {
  int rc = load_mol(S, idx, NULL, m);
  if (rc) return rc;
  double w = pose[0], x = pose[1], y = pose[2], z = pose[3];
  double nq = sqrt(w * w + x * x + y * y + z * z);
  if (!(nq > 0)) return ORC_EINVAL;
  w /= nq; x /= nq; y /= nq; z /= nq;
  double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                    {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                    {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
  for (int i = 0; i < m->n; ++i) {
    double c[3] = {m->c[i][0], m->c[i][1], m->c[i][2]};
    for (int k = 0; k < 3; ++k) m->c[i][k] = R[k][0] * c[0] + R[k][1] * c[1] + R[k][2] * c[2] + pose[4 + k];
  }
  return ORC_OK;
}

/* Central finite differences of the CRN objective in the 7 raw pose
 * parameters, step h. */
int orc_pose_grad_fd(double ZQ, const double* points, uint32_t n, const orc_set* B, int32_t ib,
                     const double pose[7], int objective, double h, double* F, double grad[7]) {
  orc_mol mb;
  int rc = load_mol_posed_d(B, ib, pose, &mb);
  if (rc) return rc;
  *F = crn_objective(&mb, points, n, ZQ, objective);
  for (int d = 0; d < 7; ++d) {
    double pp[7], pm[7];
    memcpy(pp, pose, sizeof pp);
    memcpy(pm, pose, sizeof pm);
    pp[d] += h;
    pm[d] -= h;
    orc_mol a, b;
    if ((rc = load_mol_posed_d(B, ib, pp, &a)) || (rc = load_mol_posed_d(B, ib, pm, &b))) return rc;
    grad[d] = (crn_objective(&a, points, n, ZQ, objective) - crn_objective(&b, points, n, ZQ, objective)) /
              (2.0 * h);
  }
  return ORC_OK;
}

/*
 * Analytic gradient of the closed-form first-order overlap (Eq. fo) with
 * respect to the 7 raw pose parameters of B: with c'_j = R(q) c_j + t,
 *   dO/dc'_j = sum_i K_ij 2 a_ij (c_i - c'_j),  a_ij = alpha_i alpha_j /
 *   (alpha_i + alpha_j), K_ij the (i, j) term of Eq. fo;
 *   dO/dt = sum_j dO/dc'_j,  dO/dR = sum_j dO/dc'_j c_j^T,
 * then through R(q) and q = p / |p|.
 */
int orc_fo_pose_grad(const orc_set* A, int32_t ia, const orc_set* B, int32_t ib, const double pose[7],
                     double* F, double grad[7]) {
  orc_mol ma, mb, mb0;
  int rc = load_mol(A, ia, NULL, &ma);
  if (!rc) rc = load_mol(B, ib, NULL, &mb0);
  if (!rc) rc = load_mol_posed_d(B, ib, pose, &mb);
  if (rc) return rc;
  double gt[3] = {0, 0, 0}, gR[3][3] = {{0}}, total = 0.0;
  for (int j = 0; j < mb.n; ++j) {
    double gc[3] = {0, 0, 0};
    for (int i = 0; i < ma.n; ++i) {
      double ai = ma.alpha[i], bj = mb.alpha[j], s = ai + bj, a = ai * bj / s;
      double d[3] = {ma.c[i][0] - mb.c[j][0], ma.c[i][1] - mb.c[j][1], ma.c[i][2] - mb.c[j][2]};
      double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      double t = ORC_PI / s;
      double K = ma.p[i] * mb.p[j] * t * sqrt(t) * exp(-a * d2);
      total += K;
      for (int k = 0; k < 3; ++k) gc[k] += K * 2.0 * a * d[k];
    }
    for (int k = 0; k < 3; ++k) {
      gt[k] += gc[k];
      for (int l = 0; l < 3; ++l) gR[k][l] += gc[k] * mb0.c[j][l];
    }
  }
  /* dR/dq for the unit quaternion q = (w, x, y, z) */
  double p0 = pose[0], p1 = pose[1], p2 = pose[2], p3 = pose[3];
  double nq = sqrt(p0 * p0 + p1 * p1 + p2 * p2 + p3 * p3);
  double q[4] = {p0 / nq, p1 / nq, p2 / nq, p3 / nq};
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double dR[4][3][3] = {
      {{0, -2 * z, 2 * y}, {2 * z, 0, -2 * x}, {-2 * y, 2 * x, 0}},
      {{0, 2 * y, 2 * z}, {2 * y, -4 * x, -2 * w}, {2 * z, 2 * w, -4 * x}},
      {{-4 * y, 2 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, 2 * z, -4 * y}},
      {{-4 * z, -2 * w, 2 * x}, {2 * w, -4 * z, 2 * y}, {2 * x, 2 * y, 0}}};
  double gq[4];
  for (int a = 0; a < 4; ++a) {
    gq[a] = 0.0;
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) gq[a] += gR[k][l] * dR[a][k][l];
  }
  /* q = p / |p|: dF/dp = (gq - (gq . q) q) / |p| */
  double dot = gq[0] * q[0] + gq[1] * q[1] + gq[2] * q[2] + gq[3] * q[3];
  for (int a = 0; a < 4; ++a) grad[a] = (gq[a] - dot * q[a]) / nq;
  for (int k = 0; k < 3; ++k) grad[4 + k] = gt[k];
  *F = total;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Learned control variate for the union volume                        */
/* ------------------------------------------------------------------ */

/*
 * Union attributions omega*_i = E_{r ~ N(c_i, I/(2 alpha_i))}[u(r)/m(r)]:
 * since q = sum_i (v_i / Z) N(c_i, .), V = Z E_q[u/m] = sum_i v_i omega*_i.
 * M samples per atom (M even) from stream stream_base + k (k = position in
 * idx), tag 5; atom i uses sample pairs i M/2 .. (i+1) M/2 - 1 of the usual
 * layout (normals only, the component words are unused).
 * omega [sum of the atom counts of idx] in idx order.
 */
static void attributions_one(const orc_mol* m, uint64_t seed, uint64_t stream, uint32_t M, double* omega) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int i = 0; i < m->n; ++i) {
    double s = 0.0;
    for (uint32_t p = 0; p < M / 2; ++p) {
      uint32_t blk = 2u * ((uint32_t)i * (M / 2) + p);
      uint32_t c[4] = {blk, (uint32_t)stream, (uint32_t)(stream >> 32), 5u};
      uint32_t w[8];
      orc_philox4x32_10(c, key, w);
      c[0] = blk + 1u;
      orc_philox4x32_10(c, key, w + 4);
      double n01[2], n23[2], n45[2];
      orc_normal_pair(w[2], w[3], n01);
      orc_normal_pair(w[4], w[5], n23);
      orc_normal_pair(w[6], w[7], n45);
      double z[2][3] = {{n01[0], n01[1], n45[0]}, {n23[0], n23[1], n45[1]}};
      for (int t = 0; t < 2; ++t) {
        double r[3], ms, u;
        for (int k = 0; k < 3; ++k) r[k] = m->c[i][k] + m->sigma[i] * z[t][k];
        occupancy(m, r, &ms, &u);
        s += u / ms;
      }
    }
    omega[i] = s / (double)M;
  }
}

int orc_attributions(const orc_set* S, const int32_t* idx, int64_t n_mol, uint64_t seed, uint64_t stream_base,
                     uint32_t M, double* omega, int n_threads) {
  if (M < 2 || (M & 1u)) return ORC_EINVAL;
  nthreads_set(n_threads);
  int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_mol + 1));
  if (!start) return ORC_EINVAL;
  start[0] = 0;
  for (int64_t k = 0; k < n_mol; ++k) {
    int32_t mi = idx ? idx[k] : (int32_t)k;
    if (mi < 0 || mi >= S->n_mol) { free(start); return ORC_EINVAL; }
    start[k + 1] = start[k] + (S->offsets[mi + 1] - S->offsets[mi]);
  }
  int err = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : err)
  for (int64_t k = 0; k < n_mol; ++k) {
    orc_mol m;
    if (load_mol(S, idx ? idx[k] : (int32_t)k, NULL, &m)) { err |= 1; continue; }
    attributions_one(&m, seed, stream_base + (uint64_t)k, M, omega + start[k]);
  }
  free(start);
  return err ? ORC_EINVAL : ORC_OK;
}

/*
 * Union volume with the weighted-Gaussian control variate
 * u~(r) = sum_i omega_i g_i(r):
 *   V = sum_i omega_i v_i + Z E_q[(u - u~) / m]
 * unbiased for any omega; same samples as orc_union_volume_estimate (tag 2,
 * stream stream_base + k). omega is per atom of the set (set atom order).
 */
int orc_union_volume_cv(const orc_set* S, const int32_t* idx, int64_t n_mol, const double* omega, uint64_t seed,
                        uint64_t stream_base, uint32_t n, double* vol, double* vol_se, int n_threads) {
  if (n < 2) return ORC_EINVAL;
  nthreads_set(n_threads);
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int64_t k = 0; k < n_mol; ++k) {
    int32_t mi = idx ? idx[k] : (int32_t)k;
    orc_mol m;
    if (load_mol(S, mi, NULL, &m)) { err |= 1; continue; }
    const double* om = omega + S->offsets[mi];
    double closed = 0.0;
    for (int i = 0; i < m.n; ++i) closed += om[i] * m.v[i];
    double s = 0.0, s2 = 0.0;
    for (uint32_t t = 0; t < n; t += 2) {
      double r[2][3];
      int i0, i1;
      draw_pair(&m, seed, stream_base + (uint64_t)k, ORC_TAG_SELF, t / 2, 0, r[0], r[1], &i0, &i1);
      for (int j = 0; j < 2 && t + j < n; ++j) {
        double ms = 0.0, prod = 1.0, ut = 0.0;
        for (int i = 0; i < m.n; ++i) {
          double dx = r[j][0] - m.c[i][0], dy = r[j][1] - m.c[i][1], dz = r[j][2] - m.c[i][2];
          double g = m.p[i] * exp(-m.alpha[i] * (dx * dx + dy * dy + dz * dz));
          ms += g;
          prod *= 1.0 - g;
          ut += om[i] * g;
        }
        double f = ((1.0 - prod) - ut) / ms;
        s += f;
        s2 += f * f;
      }
    }
    double mean = s / n, var = (s2 - s * mean) / (n - 1.0);
    if (var < 0) var = 0;
    vol[k] = closed + m.Z * mean;
    if (vol_se) vol_se[k] = m.Z * sqrt(var / n);
  }
  return err ? ORC_EINVAL : ORC_OK;
}

/*
 * Union volume and union self-overlap with the weighted-Gaussian control
 * variate u~(r) = sum_i omega_i g_i(r) (omega NULL: the plain estimators of
 * orc_union_volume_estimate, same numbers):
 *   V    = sum_i omega_i v_i                   + Z E_q[(u - u~) / m]
 *   O_XX = sum_ij omega_i omega_j int g_i g_j  + Z E_q[(u^2 - u~^2) / m]
 * Both residual identities hold for any omega because E_q[h / m] Z is the
 * integral of h (Eq. expectation), and the integrals of u~ and u~^2 are the
 * closed forms of Eq. fo with weights. Same samples as
 * orc_union_volume_estimate (tag 2, stream stream_base + k); n samples per
 * molecule. Not in the paper: the self-overlap counterpart of the screen's
 * union control variate.
 */
int orc_union_self_cv(const orc_set* S, const int32_t* idx, int64_t n_mol, const double* omega, uint64_t seed,
                      uint64_t stream_base, uint32_t n, double* vol, double* vol_se, double* self_ov,
                      double* self_se, int n_threads) {
  if (n < 2) return ORC_EINVAL;
  nthreads_set(n_threads);
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int64_t k = 0; k < n_mol; ++k) {
    int32_t mi = idx ? idx[k] : (int32_t)k;
    orc_mol m;
    if (load_mol(S, mi, NULL, &m)) { err |= 1; continue; }
    const double* om = omega ? omega + S->offsets[mi] : NULL;
    double closed_v = 0.0, closed_s = 0.0;
    if (om) {
      for (int i = 0; i < m.n; ++i) closed_v += om[i] * m.v[i];
      closed_s = fo_closed_w(&m, om, &m, om);
    }
    double s[4] = {0, 0, 0, 0};
    for (uint32_t t = 0; t < n; t += 2) {
      double r[2][3];
      int i0, i1;
      draw_pair(&m, seed, stream_base + (uint64_t)k, ORC_TAG_SELF, t / 2, 0, r[0], r[1], &i0, &i1);
      for (int j = 0; j < 2 && t + j < n; ++j) {
        double ms, u;
        occupancy(&m, r[j], &ms, &u);
        double ut = om ? weighted_sum(&m, om, r[j]) : 0.0;
        double fv = (u - ut) / ms, fs = (u * u - ut * ut) / ms;
        s[0] += fv; s[1] += fv * fv; s[2] += fs; s[3] += fs * fs;
      }
    }
    double e, sd;
    finish(m.Z, s[0], s[1], (double)n, &e, &sd);
    if (vol) vol[k] = closed_v + e;
    if (vol_se) vol_se[k] = sd;
    finish(m.Z, s[2], s[3], (double)n, &e, &sd);
    if (self_ov) self_ov[k] = closed_s + e;
    if (self_se) self_se[k] = sd;
  }
  return err ? ORC_EINVAL : ORC_OK;
}

/*
 * Least-squares control-variate weights (not in the paper): per molecule the
 * w minimising the integral of (u - sum_i w_i g_i)^2, the L2 projection of
 * the union occupancy onto the span of the molecule's own Gaussians:
 *   (G + lambda I) w = b,
 *   G_ij = integral g_i g_j        (closed form, the terms of Eq. fo),
 *   b_i  = integral u g_i = Z E_q[(u / m) g_i]
 *          (n samples of the molecule's own mixture, tag 6, stream
 *          stream_base + k, the usual sample layout),
 *   lambda = ridge * trace(G) / N.
 * Cholesky in FP64. omega [n_atoms] is written for the listed molecules.
 */
int orc_cv_fit_weights(const orc_set* S, const int32_t* idx, int64_t n_mol, uint64_t seed, uint64_t stream_base,
                       uint32_t n, double ridge, double* omega, int n_threads) {
  if (n < 2 || !(ridge >= 0.0)) return ORC_EINVAL;
  nthreads_set(n_threads);
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int64_t k = 0; k < n_mol; ++k) {
    int32_t mi = idx ? idx[k] : (int32_t)k;
    orc_mol m;
    if (load_mol(S, mi, NULL, &m)) { err |= 1; continue; }
    const int N = m.n;
    double b[ORC_MAXN] = {0}, A[ORC_MAXN][ORC_MAXN], L[ORC_MAXN][ORC_MAXN], y[ORC_MAXN];
    for (uint32_t t = 0; t < n; t += 2) {
      double r[2][3];
      int i0, i1;
      draw_pair(&m, seed, stream_base + (uint64_t)k, ORC_TAG_FIT, t / 2, 0, r[0], r[1], &i0, &i1);
      for (int j = 0; j < 2 && t + j < n; ++j) {
        double g[ORC_MAXN], ms = 0.0, prod = 1.0;
        for (int i = 0; i < N; ++i) {
          double dx = r[j][0] - m.c[i][0], dy = r[j][1] - m.c[i][1], dz = r[j][2] - m.c[i][2];
          g[i] = m.p[i] * exp(-m.alpha[i] * (dx * dx + dy * dy + dz * dz));
          ms += g[i];
          prod *= 1.0 - g[i];
        }
        const double w = (1.0 - prod) / ms;
        for (int i = 0; i < N; ++i) b[i] += w * g[i];
      }
    }
    double tr = 0.0;
    for (int i = 0; i < N; ++i) {
      b[i] *= m.Z / n;
      for (int j = 0; j < N; ++j) {
        double s2 = m.alpha[i] + m.alpha[j], t2 = ORC_PI / s2;
        double dx = m.c[i][0] - m.c[j][0], dy = m.c[i][1] - m.c[j][1], dz = m.c[i][2] - m.c[j][2];
        A[i][j] = m.p[i] * m.p[j] * t2 * sqrt(t2) * exp(-m.alpha[i] * m.alpha[j] / s2 * (dx * dx + dy * dy + dz * dz));
      }
      tr += A[i][i];
    }
    for (int i = 0; i < N; ++i) A[i][i] += ridge * tr / N;
    int ok = 1;
    for (int j = 0; j < N && ok; ++j) {  /* A = L L^T */
      double d = A[j][j];
      for (int l = 0; l < j; ++l) d -= L[j][l] * L[j][l];
      if (!(d > 0.0)) { ok = 0; break; }
      L[j][j] = sqrt(d);
      for (int i = j + 1; i < N; ++i) {
        double v = A[i][j];
        for (int l = 0; l < j; ++l) v -= L[i][l] * L[j][l];
        L[i][j] = v / L[j][j];
      }
    }
    if (!ok) { err |= 1; continue; }
    for (int i = 0; i < N; ++i) {  /* L y = b */
      double v = b[i];
      for (int l = 0; l < i; ++l) v -= L[i][l] * y[l];
      y[i] = v / L[i][i];
    }
    double* om = omega + S->offsets[mi];
    for (int i = N - 1; i >= 0; --i) {  /* L^T w = y */
      double v = y[i];
      for (int l = i + 1; l < N; ++l) v -= L[l][i] * om[l];
      om[i] = v / L[i][i];
    }
  }
  return err ? ORC_EINVAL : ORC_OK;
}

/*
 * Per-atom geometric features: the K = 16 nearest other atoms of the same
 * molecule by distance (ties by index), as (d / 4 A, R / 1.7 A) pairs, then
 * the atom's own R / 1.7 A; missing neighbours are (2.5, 0).
 * feat [n_atoms][33] for every atom of the set.
 */
int orc_cv_features(const orc_set* S, double* feat) {
  for (int32_t mi = 0; mi < S->n_mol; ++mi) {
    int32_t a0 = S->offsets[mi], n = S->offsets[mi + 1] - a0;
    for (int i = 0; i < n; ++i) {
      double d[ORC_MAXN];
      int id[ORC_MAXN], cnt = 0;
      for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        double dx = (double)S->xyz[3 * (a0 + i)] - S->xyz[3 * (a0 + j)];
        double dy = (double)S->xyz[3 * (a0 + i) + 1] - S->xyz[3 * (a0 + j) + 1];
        double dz = (double)S->xyz[3 * (a0 + i) + 2] - S->xyz[3 * (a0 + j) + 2];
        d[cnt] = sqrt(dx * dx + dy * dy + dz * dz);
        id[cnt++] = j;
      }
      /* insertion sort by (distance, index) */
      for (int a = 1; a < cnt; ++a) {
        double dv = d[a];
        int iv = id[a], b = a - 1;
        while (b >= 0 && (d[b] > dv || (d[b] == dv && id[b] > iv))) { d[b + 1] = d[b]; id[b + 1] = id[b]; --b; }
        d[b + 1] = dv;
        id[b + 1] = iv;
      }
      double* f = feat + 33 * (size_t)(a0 + i);
      for (int k = 0; k < 16; ++k) {
        if (k < cnt) { f[2 * k] = d[k] / 4.0; f[2 * k + 1] = (double)S->radius[a0 + id[k]] / 1.7; }
        else { f[2 * k] = 2.5; f[2 * k + 1] = 0.0; }
      }
      f[32] = (double)S->radius[a0 + i] / 1.7;
    }
  }
  return ORC_OK;
}
