// Molecule sets: host validation, packing and upload; per-atom parameters,
// mixture masses and alias tables on the device (Eq. occ, Eq. expectation).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace shp {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}

void clear_error() { g_err.clear(); }

int cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? SHP_ENOMEM : SHP_ECUDA;
}

// Per-molecule preparation on the device (molecules taken in size order, so
// the molecules a warp handles together have similar sizes). Per atom, from
// the radius R and height p (FP64, IEEE-rounded operations throughout, so the
// values do not depend on the compiler's contraction choices):
//   alpha = c_alpha / R^2,  t = pi / alpha,  v = p t sqrt(t)   (Gaussian volume)
//   sigma = 1 / sqrt(2 alpha) (sampling width),  log2 p,  Z = sum_i v_i in
//   atom order.
// Integer alias table of the v_i: column masses in units of 2^-32 of one
// column, M_i = floor((v_i / Z) * n 2^32), the rounding remainder to the last
// atom; small (M < 2^32) and large worklists are FIFO in atom order, and a
// large atom stays at the head of its list until its residual mass turns
// small. Full columns get threshold 2^32 - 1 and alias themselves. The list
// building is sequential (lane 0) on the warp's shared-memory copy.
constexpr int kRadiusClasses = 16;

struct PrepArgs {
  float4* atom;          // in: x, y, z; out: w = alpha
  float2* aux;           // out: sigma, log2 p (the volumes, as doubles, between phases)
  const float* radius;   // [n_atoms]
  const float* height;   // [n_atoms] heights staged in the threshold slots, or NULL: p_default
  uint32_t* thr;         // out: alias thresholds (after the heights are read)
  uint8_t* alias;        // out: alias targets
  double* Z;             // out: [n_mol]
  const int32_t* off;
  const int32_t* order;
  int32_t n_mol;
  double c_alpha, p_default;
  float log2p_default;
  // radius classes: radii come from a few element types, so the host
  // evaluates the terms that depend on R alone once per class (up to
  // kRadiusClasses radii, bits ascending), with the same IEEE operations as
  // the kernel; an atom whose radius has no class evaluates them itself.
  int32_t n_cls;
  uint32_t cls_bits[kRadiusClasses];
  float cls_alpha[kRadiusClasses], cls_sigma[kRadiusClasses];
  double cls_t[kRadiusClasses], cls_sqrt_t[kRadiusClasses];
};

constexpr int kPrepWarps = 8;
constexpr int kPrepGroup = 16;  // molecules a warp takes at a time (<= 32)

struct PrepWarp {
  unsigned long long mass[SHP_MAX_ATOMS];
  uint8_t small[SHP_MAX_ATOMS], large[SHP_MAX_ATOMS];
};

// The terms of atom radius Rf that depend on R alone: from its class when
// the radius has one, else evaluated (FP64, IEEE-rounded).
__device__ __forceinline__ void radius_terms(const PrepArgs& a, const uint32_t* cls_bits, float Rf, double& t,
                                             double& sqrt_t, float& alpha_f, float& sigma_f) {
  const uint32_t bits = __float_as_uint(Rf);
  int c = 0;
  for (int step = kRadiusClasses / 2; step; step >>= 1)
    if (c + step < a.n_cls && cls_bits[c + step] <= bits) c += step;
  if (a.n_cls && cls_bits[c] == bits) {
    t = a.cls_t[c];
    sqrt_t = a.cls_sqrt_t[c];
    alpha_f = a.cls_alpha[c];
    sigma_f = a.cls_sigma[c];
  } else {
    const double kPi = 3.14159265358979323846;
    const double R = Rf;
    const double alpha = __ddiv_rn(a.c_alpha, __dmul_rn(R, R));
    t = __ddiv_rn(kPi, alpha);
    sqrt_t = __dsqrt_rn(t);
    alpha_f = (float)alpha;
    sigma_f = (float)__ddiv_rn(1.0, __dsqrt_rn(__dmul_rn(2.0, alpha)));
  }
}

// A warp takes kPrepGroup molecules at a time (consecutive in size order).
// Phase 1, per molecule with lanes over atoms: the volumes v_i, parked in the
// atoms' aux slots (8 B, a double), and alpha. Phase 2, lane j: Z of molecule
// j in atom order (a sequential FP64 sum, one per lane: on one lane per
// molecule each addition would still take a whole warp instruction of the
// slow FP64 pipe). Phase 3, per molecule: the masses, then sigma and log2 p
// over the parked volumes, then the alias table (lane 0).
__global__ void __launch_bounds__(32 * kPrepWarps) set_prep_kernel(const PrepArgs a) {
  __shared__ PrepWarp W[kPrepWarps];
  __shared__ uint32_t cls_bits[kRadiusClasses];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  PrepWarp& w = W[warp];
  const unsigned long long kOne = 1ull << 32;
  const unsigned kAll = 0xffffffffu;
  double* vol = reinterpret_cast<double*>(a.aux);
  if (threadIdx.x < kRadiusClasses) cls_bits[threadIdx.x] = a.cls_bits[threadIdx.x];
  __syncthreads();
  const int64_t n_groups = ((int64_t)a.n_mol + kPrepGroup - 1) / kPrepGroup;
  for (int64_t g = (int64_t)blockIdx.x * kPrepWarps + warp; g < n_groups; g += (int64_t)gridDim.x * kPrepWarps) {
    const int64_t k0 = (int64_t)kPrepGroup * g;
    const int nm = (int)min((int64_t)kPrepGroup, (int64_t)a.n_mol - k0);
    int32_t my_m = 0, my_a0 = 0, my_n = 0;
    if (lane < nm) {
      my_m = a.order[k0 + lane];
      my_a0 = a.off[my_m];
      my_n = a.off[my_m + 1] - my_a0;
    }
    for (int j = 0; j < nm; ++j) {
      const int32_t a0 = __shfl_sync(kAll, my_a0, j), n = __shfl_sync(kAll, my_n, j);
      for (int i = lane; i < n; i += 32) {
        const double p = a.height ? (double)a.height[a0 + i] : a.p_default;
        double t, sqrt_t;
        float alpha_f, sigma_f;
        radius_terms(a, cls_bits, a.radius[a0 + i], t, sqrt_t, alpha_f, sigma_f);
        vol[a0 + i] = __dmul_rn(__dmul_rn(p, t), sqrt_t);
        reinterpret_cast<float*>(a.atom + a0 + i)[3] = alpha_f;
      }
    }
    __syncwarp();
    double my_Z = 0.0;
    for (int i = 0; i < my_n; ++i) my_Z = __dadd_rn(my_Z, vol[my_a0 + i]);
    if (lane < nm) a.Z[my_m] = my_Z;
    __syncwarp();
    for (int j = 0; j < nm; ++j) {
      const int32_t a0 = __shfl_sync(kAll, my_a0, j), n = __shfl_sync(kAll, my_n, j);
      const double Z = __shfl_sync(kAll, my_Z, j);
      const double scale = __dmul_rn((double)n, 4294967296.0);
      unsigned long long sum = 0;
      for (int i = lane; i < n; i += 32) {
        // truncation = floor: 0 <= (v_i / Z) n 2^32 < 2^38
        const unsigned long long M = (unsigned long long)(long long)__dmul_rn(__ddiv_rn(vol[a0 + i], Z), scale);
        w.mass[i] = M;
        sum += M;
        double t, sqrt_t;
        float alpha_f, sigma_f;
        radius_terms(a, cls_bits, a.radius[a0 + i], t, sqrt_t, alpha_f, sigma_f);
        a.aux[a0 + i] = make_float2(sigma_f, a.height ? (float)log2((double)a.height[a0 + i]) : a.log2p_default);
      }
      for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(kAll, sum, o);
      __syncwarp();
      if (lane == 0) {
        unsigned long long* mass = w.mass;
        mass[n - 1] += (unsigned long long)n * kOne - sum;
        uint32_t* thr = a.thr + a0;  // overwrites this molecule's heights, all read above
        uint8_t* alias = a.alias + a0;
        int sh = 0, st = 0, lh = 0, lt = 0;
        for (int i = 0; i < n; ++i) (mass[i] < kOne ? w.small[st++] : w.large[lt++]) = (uint8_t)i;
        while (sh < st && lh < lt) {
          const int sm = w.small[sh++];
          const int lg = w.large[lh];
          thr[sm] = (uint32_t)mass[sm];
          alias[sm] = (uint8_t)lg;
          mass[lg] -= kOne - mass[sm];
          if (mass[lg] < kOne) {
            ++lh;
            w.small[st++] = (uint8_t)lg;
          }
        }
        for (; sh < st; ++sh) { thr[w.small[sh]] = 0xFFFFFFFFu; alias[w.small[sh]] = w.small[sh]; }
        for (; lh < lt; ++lh) { thr[w.large[lh]] = 0xFFFFFFFFu; alias[w.large[lh]] = w.large[lh]; }
      }
      __syncwarp();
    }
  }
}

// Gaussian volume v_i = p_i (pi/alpha_i)^{3/2} and centre of atom i, from
// the stored alpha and log2 p (FP64).
__device__ __forceinline__ double atom_volume(const float4* atom, const float2* aux, int i, double c[3]) {
  const float4 a = atom[i];
  c[0] = a.x; c[1] = a.y; c[2] = a.z;
  const double t = 3.14159265358979323846 / (double)a.w;
  return exp2((double)aux[i].y) * t * sqrt(t);
}

// Principal frame of one molecule: centroid weighted by the Gaussian
// volumes v_i, and the eigenvectors of the weighted second-moment matrix
// (cyclic Jacobi rotations, FP64) sorted by decreasing eigenvalue; the first
// two axes point so the weighted third moment of the projection is >= 0, the
// third completes a proper rotation. out = centroid (3), E row-major (9)
// with the axes as columns. Computed on the device at first use.
__device__ void principal_frame(int n, const float4* atom, const float2* aux, float* out) {
  double W = 0.0, cen[3] = {0, 0, 0}, c[3];
  for (int i = 0; i < n; ++i) {
    const double v = atom_volume(atom, aux, i, c);
    W += v;
    for (int k = 0; k < 3; ++k) cen[k] += v * c[k];
  }
  for (int k = 0; k < 3; ++k) cen[k] /= W;
  double A[3][3] = {{0}};
  for (int i = 0; i < n; ++i) {
    const double v = atom_volume(atom, aux, i, c);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) A[a][b] += v * (c[a] - cen[a]) * (c[b] - cen[b]);
  }
  double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int sweep = 0; sweep < 50; ++sweep) {
    const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const double diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-30 * (diag + 1e-300)) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < 3; ++k) {  // A <- A J
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = cs * akp - sn * akq;
          A[k][q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < 3; ++k) {  // A <- J^T A
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = cs * apk - sn * aqk;
          A[q][k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < 3; ++k) {  // V <- V J
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = cs * vkp - sn * vkq;
          V[k][q] = sn * vkp + cs * vkq;
        }
      }
  }
  int ord[3] = {0, 1, 2};  // axes by decreasing second moment (stable)
  for (int i = 1; i < 3; ++i)
    for (int j = i; j > 0 && A[ord[j]][ord[j]] > A[ord[j - 1]][ord[j - 1]]; --j) {
      const int t = ord[j]; ord[j] = ord[j - 1]; ord[j - 1] = t;
    }
  double E[3][3];
  for (int a = 0; a < 2; ++a) {
    double skew = 0.0;
    for (int i = 0; i < n; ++i) {
      const double v = atom_volume(atom, aux, i, c);
      double pr = 0.0;
      for (int k = 0; k < 3; ++k) pr += (c[k] - cen[k]) * V[k][ord[a]];
      skew += v * pr * pr * pr;
    }
    const double sg = skew < 0 ? -1.0 : 1.0;
    for (int k = 0; k < 3; ++k) E[k][a] = sg * V[k][ord[a]];
  }
  E[0][2] = E[1][0] * E[2][1] - E[2][0] * E[1][1];
  E[1][2] = E[2][0] * E[0][1] - E[0][0] * E[2][1];
  E[2][2] = E[0][0] * E[1][1] - E[1][0] * E[0][1];
  for (int k = 0; k < 3; ++k) out[k] = (float)cen[k];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) out[3 + 3 * a + b] = (float)E[a][b];
}

// One thread per molecule.
__global__ void frames_kernel(const float4* __restrict__ atom, const float2* __restrict__ aux,
                              const int32_t* __restrict__ off, int32_t n_mol, float* __restrict__ frame) {
  const int32_t m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_mol) return;
  const int32_t a0 = off[m];
  principal_frame(off[m + 1] - a0, atom + a0, aux + a0, frame + 12 * (size_t)m);
}

// All device arrays of a set live in one stream-ordered allocation: one copy
// of the inputs (20 B per atom, 24 with heights) from one of two pinned
// staging buffers that the library keeps (and grows) across loads, then
// set_prep_kernel writes the rest; each buffer's event marks the end of its
// last use, so a load waits only for the upload two loads back, never for
// the caller's kernels.
struct SetLayout {
  size_t atom, aux, radius, thr, alias, off, Z, order, frame, total;
};

static size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

static SetLayout set_layout(int64_t n_atoms, int32_t n_mol) {
  SetLayout L{};
  size_t o = 0;
  // uploaded from the host: atoms (x, y, z), radii, offsets, size order,
  // then the thresholds' slots (which carry the heights when given)
  L.atom = o;   o = align16(o + sizeof(float4) * n_atoms);
  L.radius = o; o = align16(o + sizeof(float) * n_atoms);
  L.off = o;    o = align16(o + sizeof(int32_t) * (n_mol + 1));
  L.order = o;  o = align16(o + sizeof(int32_t) * n_mol);
  L.thr = o;    o = align16(o + sizeof(uint32_t) * n_atoms);
  // written on the device
  L.aux = o;    o = align16(o + sizeof(float2) * n_atoms);
  L.alias = o;  o = align16(o + n_atoms);
  L.Z = o;      o = align16(o + sizeof(double) * n_mol);
  L.frame = o;  o = align16(o + sizeof(float) * 12 * n_mol);
  L.total = o;
  return L;
}

struct StageBuf {
  void* ptr = nullptr;
  size_t cap = 0;
  cudaEvent_t done = nullptr;  // recorded after the buffer's last upload
};
static std::mutex g_stage_mu;
static StageBuf g_stage[2];
static int g_stage_next = 0;
static cudaStream_t g_copy_stream[64];  // per device: uploads overlap the caller's kernels

// The library's upload stream of device `dev` (non-blocking, created once).
// Caller holds g_stage_mu.
static int copy_stream(int dev, cudaStream_t* out) {
  if (dev < 0 || dev >= 64) { *out = nullptr; return SHP_OK; }
  if (!g_copy_stream[dev]) SHP_CUDA(cudaStreamCreateWithFlags(&g_copy_stream[dev], cudaStreamNonBlocking));
  *out = g_copy_stream[dev];
  return SHP_OK;
}

// A staging buffer of at least `bytes`, its previous upload finished.
// Caller holds g_stage_mu.
static int stage_buffer(size_t bytes, StageBuf** out) {
  StageBuf& b = g_stage[g_stage_next];
  g_stage_next ^= 1;
  if (!b.done) SHP_CUDA(cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming));
  SHP_CUDA(cudaEventSynchronize(b.done));
  if (bytes > b.cap) {
    if (b.ptr) cudaFreeHost(b.ptr);
    b.ptr = nullptr;
    b.cap = 0;
    const size_t cap = bytes + bytes / 4;
    SHP_CUDA(cudaMallocHost(&b.ptr, cap));
    b.cap = cap;
  }
  *out = &b;
  return SHP_OK;
}

// Stable order of molecule ids by atom count, descending (counting sort).
static void order_by_size(const int32_t* offsets, int32_t n_mol, int32_t* order) {
  int64_t start[SHP_MAX_ATOMS + 2] = {0};
  for (int32_t m = 0; m < n_mol; ++m) ++start[SHP_MAX_ATOMS - (offsets[m + 1] - offsets[m]) + 1];
  for (int k = 1; k <= SHP_MAX_ATOMS + 1; ++k) start[k] += start[k - 1];
  for (int32_t m = 0; m < n_mol; ++m) order[start[SHP_MAX_ATOMS - (offsets[m + 1] - offsets[m])]++] = m;
}

// Stream-ordered free (the set's memory comes from cudaMallocAsync); callers
// that free synchronously have synchronised the device first.
static void free_set_memory(shp_set_s* s, cudaStream_t stream = nullptr) {
  if (s->dbase) cudaFreeAsync(s->dbase, stream);
  if (s->frames_done) cudaEventDestroy(s->frames_done);
  s->frames_done = nullptr;
  s->dbase = nullptr;
  s->atom = nullptr; s->aux = nullptr; s->thr = nullptr; s->alias = nullptr;
  s->off = nullptr; s->Z = nullptr; s->order = nullptr; s->frame = nullptr; s->radius = nullptr;
}

static std::atomic<int32_t> g_fail_allocs{0};

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t stream) {
  int32_t pending = g_fail_allocs.load();
  while (pending > 0) {
    if (g_fail_allocs.compare_exchange_weak(pending, pending - 1)) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
  }
  return cudaMallocAsync(p, bytes, stream);
}

int ensure_frames(shp_set_s* s, cudaStream_t stream) {
  std::lock_guard<std::mutex> lk(s->frames_mu);
  if (!s->frames_ready) {
    if (s->n_mol > 0) {
      if (!s->frames_done) SHP_CUDA(cudaEventCreateWithFlags(&s->frames_done, cudaEventDisableTiming));
      const int threads = 128;
      frames_kernel<<<(s->n_mol + threads - 1) / threads, threads, 0, stream>>>(s->atom, s->aux, s->off, s->n_mol,
                                                                               s->frame);
      SHP_CUDA(cudaGetLastError());
      SHP_CUDA(cudaEventRecord(s->frames_done, stream));
    }
    s->frames_ready = true;
    return SHP_OK;
  }
  if (s->frames_done) SHP_CUDA(cudaStreamWaitEvent(stream, s->frames_done, 0));
  return SHP_OK;
}

}  // namespace shp

using namespace shp;

extern "C" const char* shp_last_error(void) { return g_err.c_str(); }

extern "C" int shp_version(void) { return 6; }

extern "C" int shp_fail_next_allocations(int32_t count) {
  clear_error();
  if (count < 0) { set_error("shp_fail_next_allocations: negative count"); return SHP_EINVAL; }
  g_fail_allocs.store(count);
  return SHP_OK;
}

extern "C" int shape_set_load(const float* xyz, const float* radius, const float* height,
                              double c_alpha, const int32_t* offsets, int32_t n_mol, void* stream,
                              shp_set* out) {
  clear_error();
  if (!out || !offsets || n_mol < 0) {
    set_error("shape_set_load: NULL output/offsets or negative n_mol");
    return SHP_EINVAL;
  }
  *out = nullptr;
  if (offsets[0] != 0) { set_error("shape_set_load: offsets[0] must be 0"); return SHP_EINVAL; }
  int32_t max_atoms = 0;
  for (int32_t m = 0; m < n_mol; ++m) {
    const int32_t c = offsets[m + 1] - offsets[m];
    if (c < 1 || c > SHP_MAX_ATOMS) {
      set_error("shape_set_load: molecule %d has %d atoms (allowed 1..%d)", m, c, SHP_MAX_ATOMS);
      return SHP_ERANGE;
    }
    max_atoms = std::max(max_atoms, c);
  }
  const int64_t n_atoms = offsets[n_mol];
  if (n_atoms > 0 && (!xyz || !radius)) { set_error("shape_set_load: NULL xyz/radius"); return SHP_EINVAL; }
  const double ca = c_alpha > 0 ? c_alpha : 2.41798793;
  const double kPi = 3.14159265358979323846;

  auto* s = new (std::nothrow) shp_set_s;
  if (!s) { set_error("shape_set_load: host allocation failed"); return SHP_ENOMEM; }
  SHP_CUDA(cudaGetDevice(&s->device));
  s->n_mol = n_mol;
  s->n_atoms = n_atoms;
  s->max_atoms = max_atoms;
  s->h_count.resize(n_mol);
  for (int32_t m = 0; m < n_mol; ++m) s->h_count[m] = (uint8_t)(offsets[m + 1] - offsets[m]);
  const SetLayout L = set_layout(n_atoms, n_mol);
  std::lock_guard<std::mutex> stage_lock(g_stage_mu);
  StageBuf* sb = nullptr;
  int rc = stage_buffer(L.total, &sb);
  if (rc) { delete s; return rc; }
  unsigned char* hb = static_cast<unsigned char*>(sb->ptr);
  float4* atom = reinterpret_cast<float4*>(hb + L.atom);
  float* rad = reinterpret_cast<float*>(hb + L.radius);
  float* hgt = reinterpret_cast<float*>(hb + L.thr);
  // host side: validate and pack (x, y, z, -) and R (and p) into the staging
  // buffer, molecules in parallel; the arithmetic runs in set_prep_kernel
  int32_t bad_mol = -1;
#pragma omp parallel for schedule(dynamic, 256)
  for (int32_t m = 0; m < n_mol; ++m) {
    const int64_t a0 = offsets[m], a1 = offsets[m + 1];
    bool ok = true;
    for (int64_t a = a0; a < a1; ++a) {
      const float x = xyz[3 * a], y = xyz[3 * a + 1], z = xyz[3 * a + 2], R = radius[a];
      const float p = height ? height[a] : 1.f;
      ok &= std::isfinite(x) && std::isfinite(y) && std::isfinite(z) && R > 0 && std::isfinite(R) && p > 0 &&
            std::isfinite(p);
      atom[a] = make_float4(x, y, z, 0.f);
      rad[a] = R;
      if (height) hgt[a] = p;
    }
    if (!ok) {
#pragma omp critical
      { if (bad_mol < 0 || m < bad_mol) bad_mol = m; }
    }
  }
  if (bad_mol >= 0) {
    set_error("shape_set_load: molecule %d has a non-finite or non-positive coordinate, radius or height", bad_mol);
    delete s;
    return SHP_EINVAL;
  }
  order_by_size(offsets, n_mol, reinterpret_cast<int32_t*>(hb + L.order));
  std::memcpy(hb + L.off, offsets, sizeof(int32_t) * (n_mol + 1));
  // allocate and upload on the library's copy stream, prepare on the device
  // there, then order the caller's stream after both: the copy overlaps
  // kernels already queued on the caller's stream
  cudaStream_t st = (cudaStream_t)stream, cs = nullptr;
  rc = copy_stream(s->device, &cs);
  if (rc) { delete s; return rc; }
  if (!cs) cs = st;
  unsigned char* db = nullptr;
  cudaError_t e = dev_alloc((void**)&db, L.total, cs);
  if (e != cudaSuccess) { delete s; return cuda_fail(e, "shape_set_load: device allocation"); }
  s->dbase = db;
  s->atom = reinterpret_cast<float4*>(db + L.atom);
  s->aux = reinterpret_cast<float2*>(db + L.aux);
  s->radius = reinterpret_cast<float*>(db + L.radius);
  s->thr = reinterpret_cast<uint32_t*>(db + L.thr);
  s->alias = db + L.alias;
  s->off = reinterpret_cast<int32_t*>(db + L.off);
  s->Z = reinterpret_cast<double*>(db + L.Z);
  s->order = reinterpret_cast<int32_t*>(db + L.order);
  s->frame = reinterpret_cast<float*>(db + L.frame);
  // the heights travel in the threshold slots, read before the thresholds
  // are written
  e = cudaMemcpyAsync(db, hb, height ? L.aux : L.thr, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess && n_mol > 0) {
    PrepArgs pa{};
    pa.atom = s->atom;
    pa.aux = s->aux;
    pa.radius = s->radius;
    pa.height = height ? reinterpret_cast<const float*>(s->thr) : nullptr;
    pa.thr = s->thr;
    pa.alias = s->alias;
    pa.Z = s->Z;
    pa.off = s->off;
    pa.order = s->order;
    pa.n_mol = n_mol;
    pa.c_alpha = ca;
    pa.p_default = 2.0 * std::sqrt(2.0);
    pa.log2p_default = (float)std::log2(pa.p_default);
    // radius classes from the distinct radii of a strided sample of 4096
    // atoms (the first kRadiusClasses found); a radius outside the table is
    // evaluated by the kernel, so the sample decides speed, not values
    uint32_t cls[kRadiusClasses];
    int n_cls = 0;
    const int64_t stride = std::max<int64_t>(1, n_atoms / 4096);
    for (int64_t at = 0; at < n_atoms && n_cls < kRadiusClasses; at += stride) {
      uint32_t bits;
      std::memcpy(&bits, &radius[at], sizeof bits);
      int k = 0;
      while (k < n_cls && cls[k] != bits) ++k;
      if (k == n_cls) cls[n_cls++] = bits;
    }
    std::sort(cls, cls + n_cls);
    pa.n_cls = n_cls;
    for (int k = 0; k < n_cls; ++k) {
      float Rf;
      std::memcpy(&Rf, &cls[k], sizeof Rf);
      const double R = Rf;
      const double alpha = ca / (R * R);
      pa.cls_bits[k] = cls[k];
      pa.cls_t[k] = kPi / alpha;
      pa.cls_sqrt_t[k] = std::sqrt(pa.cls_t[k]);
      pa.cls_alpha[k] = (float)alpha;
      pa.cls_sigma[k] = (float)(1.0 / std::sqrt(2.0 * alpha));
    }
    const int64_t groups = (n_mol + kPrepGroup - 1) / kPrepGroup;
    const int64_t blocks = std::min<int64_t>((groups + kPrepWarps - 1) / kPrepWarps, 148 * 16);
    set_prep_kernel<<<(unsigned)blocks, 32 * kPrepWarps, 0, cs>>>(pa);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(sb->done, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, sb->done, 0);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "shape_set_load: upload");
    cudaStreamSynchronize(cs);
    free_set_memory(s, cs);
    delete s;
    return rc;
  }
  *out = s;
  return SHP_OK;
}

extern "C" int shape_set_free(shp_set s) {
  clear_error();
  if (!s) return SHP_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != s->device) cudaSetDevice(s->device);
  cudaDeviceSynchronize();
  free_set_memory(s);
  if (prev != s->device) cudaSetDevice(prev);
  delete s;
  return SHP_OK;
}

extern "C" int shape_set_free_async(shp_set s, void* stream) {
  clear_error();
  if (!s) return SHP_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != s->device) cudaSetDevice(s->device);
  free_set_memory(s, (cudaStream_t)stream);
  if (prev != s->device) cudaSetDevice(prev);
  delete s;
  return SHP_OK;
}

extern "C" int shape_set_info(shp_set s, int32_t* n_mol, int64_t* n_atoms, int32_t* max_atoms) {
  clear_error();
  if (!s) { set_error("shape_set_info: NULL set"); return SHP_EINVAL; }
  if (n_mol) *n_mol = s->n_mol;
  if (n_atoms) *n_atoms = s->n_atoms;
  if (max_atoms) *max_atoms = s->max_atoms;
  return SHP_OK;
}

extern "C" int shape_set_tables(shp_set s, double* Z, uint32_t* thr, uint8_t* alias) {
  clear_error();
  if (!s) { set_error("shape_set_tables: NULL set"); return SHP_EINVAL; }
  if ((Z || thr || alias) && s->n_mol) {
    SHP_CUDA(cudaDeviceSynchronize());
    if (Z) SHP_CUDA(cudaMemcpy(Z, s->Z, sizeof(double) * s->n_mol, cudaMemcpyDeviceToHost));
    if (thr) SHP_CUDA(cudaMemcpy(thr, s->thr, sizeof(uint32_t) * s->n_atoms, cudaMemcpyDeviceToHost));
    if (alias) SHP_CUDA(cudaMemcpy(alias, s->alias, s->n_atoms, cudaMemcpyDeviceToHost));
  }
  return SHP_OK;
}

extern "C" int shape_set_frames(shp_set s, float* frames) {
  clear_error();
  if (!s || !frames) { set_error("shape_set_frames: NULL argument"); return SHP_EINVAL; }
  if (s->n_mol) {
    const int rc = ensure_frames(s, nullptr);
    if (rc) return rc;
    SHP_CUDA(cudaDeviceSynchronize());
    SHP_CUDA(cudaMemcpy(frames, s->frame, sizeof(float) * 12 * (size_t)s->n_mol, cudaMemcpyDeviceToHost));
  }
  return SHP_OK;
}
