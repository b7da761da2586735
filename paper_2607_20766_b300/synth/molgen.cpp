// Seeded synthetic drug-like molecules: heavy-atom random tree walks.
//
// This is an input generator only. It places atom centres and assigns
// elements and van der Waals radii; it holds none of the shape-overlap
// arithmetic (no Gaussians, no sampling of the estimator). Both the CUDA path
// and the CPU oracle are fed from it.
//
// Recipe (one molecule, own RNG stream seeded from (seed, molecule id)):
//   * atom 0 at the origin;
//   * each new atom attaches to a uniformly chosen existing atom P with fewer
//     than 3 neighbours; bond length U(1.40, 1.55) A;
//   * if P already has a neighbour G, the angle X-P-G is 109.5 or 120 degrees
//     (50/50) plus U(-5, 5) degrees and the dihedral about P-G is uniform;
//     otherwise the bond direction is uniform on the sphere;
//   * the new atom must be >= 2.5 A from every atom it is not bonded to,
//     except the other neighbours of P (atoms one bond angle away), which
//     must be >= 2.2 A;  up to 100 geometry retries per parent, then a new
//     parent is drawn;
//   * element C/N/O/S with probabilities 0.70/0.12/0.15/0.03, radius
//     C 1.70, N 1.55, O 1.52, S 1.80 A.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  // uniform in [0, 1) with 53 bits
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
  double uniform(double lo, double hi) { return lo + (hi - lo) * uniform(); }
  uint32_t below(uint32_t n) { return (uint32_t)(((next() >> 32) * (uint64_t)n) >> 32); }
  double normal() {
    double u1 = 1.0 - uniform();  // (0, 1]
    double u2 = uniform();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
};

uint64_t mol_seed(uint64_t seed, int64_t mol_id) {
  SplitMix64 g{seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(mol_id + 1))};
  g.next();
  return g.next();
}

const float kRadius[4] = {1.70f, 1.55f, 1.52f, 1.80f};  // C N O S

uint8_t draw_element(SplitMix64& g) {
  double u = g.uniform();
  if (u < 0.70) return 0;
  if (u < 0.82) return 1;
  if (u < 0.97) return 2;
  return 3;
}

// Build one molecule of n atoms into pos (n*3 doubles) and elem.
// Returns 0 on success, -1 if placement failed everywhere.
int build_one(SplitMix64& g, int n, double* pos, uint8_t* elem) {
  std::vector<int> deg(n, 0);
  std::vector<int> nbr(n * 3, -1);
  pos[0] = pos[1] = pos[2] = 0.0;
  elem[0] = draw_element(g);
  const double deg2rad = 3.14159265358979323846 / 180.0;
  for (int k = 1; k < n; ++k) {
    bool placed = false;
    for (int parent_try = 0; parent_try < 2000 && !placed; ++parent_try) {
      // uniform among atoms with < 3 neighbours
      int n_open = 0;
      for (int i = 0; i < k; ++i) n_open += deg[i] < 3;
      if (n_open == 0) return -1;
      int pick = (int)g.below((uint32_t)n_open), P = -1;
      for (int i = 0; i < k; ++i)
        if (deg[i] < 3 && pick-- == 0) { P = i; break; }
      const double* cp = pos + 3 * P;
      for (int attempt = 0; attempt < 100 && !placed; ++attempt) {
        double b = g.uniform(1.40, 1.55);
        double d[3];
        if (deg[P] == 0) {
          double z = g.uniform(-1.0, 1.0), ph = g.uniform(0.0, 6.283185307179586);
          double s = std::sqrt(1.0 - z * z);
          d[0] = s * std::cos(ph); d[1] = s * std::sin(ph); d[2] = z;
        } else {
          const double* cg = pos + 3 * nbr[3 * P];
          double u[3] = {cg[0] - cp[0], cg[1] - cp[1], cg[2] - cp[2]};
          double un = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
          for (double& x : u) x /= un;
          // any vector not parallel to u, then Gram-Schmidt
          double a[3] = {1, 0, 0};
          if (std::fabs(u[0]) > 0.9) { a[0] = 0; a[1] = 1; }
          double dot = a[0] * u[0] + a[1] * u[1] + a[2] * u[2];
          double v[3] = {a[0] - dot * u[0], a[1] - dot * u[1], a[2] - dot * u[2]};
          double vn = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
          for (double& x : v) x /= vn;
          double w[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2],
                         u[0] * v[1] - u[1] * v[0]};
          double theta = ((g.uniform() < 0.5) ? 109.5 : 120.0) + g.uniform(-5.0, 5.0);
          theta *= deg2rad;
          double phi = g.uniform(0.0, 6.283185307179586);
          double ct = std::cos(theta), st = std::sin(theta);
          double cph = std::cos(phi), sph = std::sin(phi);
          for (int c = 0; c < 3; ++c) d[c] = ct * u[c] + st * (cph * v[c] + sph * w[c]);
        }
        double x[3] = {cp[0] + b * d[0], cp[1] + b * d[1], cp[2] + b * d[2]};
        bool ok = true;
        for (int i = 0; i < k && ok; ++i) {
          if (i == P) continue;
          bool one_three = false;
          for (int t = 0; t < deg[P]; ++t) one_three |= (nbr[3 * P + t] == i);
          double lim = one_three ? 2.2 : 2.5;
          double dx = x[0] - pos[3 * i], dy = x[1] - pos[3 * i + 1], dz = x[2] - pos[3 * i + 2];
          ok = dx * dx + dy * dy + dz * dz >= lim * lim;
        }
        if (!ok) continue;
        pos[3 * k] = x[0]; pos[3 * k + 1] = x[1]; pos[3 * k + 2] = x[2];
        nbr[3 * P + deg[P]++] = k;
        nbr[3 * k + deg[k]++] = P;
        elem[k] = draw_element(g);
        placed = true;
      }
    }
    if (!placed) return -1;
  }
  return 0;
}

}  // namespace

extern "C" {

// Atom counts: kind 0 = uniform integer in [lo, hi]; kind 1 = heavy-tailed
// toward 40, round(40 + 6 t_3) clipped to [lo, hi] with t_3 a Student-t
// variate with 3 degrees of freedom.
int molgen_counts(uint64_t seed, int64_t n_mol, int kind, int lo, int hi, int32_t* out) {
  if (n_mol < 0 || lo < 1 || hi < lo) return -1;
  for (int64_t m = 0; m < n_mol; ++m) {
    SplitMix64 g{mol_seed(seed ^ 0x5bd1e9955bd1e995ull, m)};
    if (kind == 0) {
      out[m] = lo + (int32_t)g.below((uint32_t)(hi - lo + 1));
    } else {
      double z = g.normal();
      double c = 0;
      for (int i = 0; i < 3; ++i) { double t = g.normal(); c += t * t; }
      double t3 = z / std::sqrt(c / 3.0);
      double v = std::nearbyint(40.0 + 6.0 * t3);
      if (v < lo) v = lo;
      if (v > hi) v = hi;
      out[m] = (int32_t)v;
    }
  }
  return 0;
}

// Generate molecules mol_first .. mol_first+n_mol-1 of stream `seed`.
// offsets[n_mol+1] (host, int64) gives each molecule's atom range in the
// outputs; xyz is [n_atoms][3] float32 (A), radius [n_atoms] float32,
// elem [n_atoms] uint8 (0 C, 1 N, 2 O, 3 S). Returns 0, or -1 on a failed
// placement or a bad argument.
int molgen_generate(uint64_t seed, int64_t mol_first, int64_t n_mol, const int64_t* offsets,
                    float* xyz, float* radius, uint8_t* elem) {
  int err = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : err)
  for (int64_t m = 0; m < n_mol; ++m) {
    int n = (int)(offsets[m + 1] - offsets[m]);
    if (n < 1 || n > 4096) { err |= 1; continue; }
    SplitMix64 g{mol_seed(seed, mol_first + m)};
    std::vector<double> pos(3 * (size_t)n);
    std::vector<uint8_t> el(n);
    if (build_one(g, n, pos.data(), el.data()) != 0) { err |= 1; continue; }
    int64_t o = offsets[m];
    for (int i = 0; i < n; ++i) {
      for (int c = 0; c < 3; ++c) xyz[3 * (o + i) + c] = (float)pos[3 * i + c];
      elem[o + i] = el[i];
      radius[o + i] = kRadius[el[i]];
    }
  }
  return err ? -1 : 0;
}

}  // extern "C"
