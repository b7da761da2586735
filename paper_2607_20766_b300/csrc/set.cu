// Molecule sets: validation, per-atom parameters, mixture masses and alias
// tables (Eq. occ, Eq. expectation), device upload. Host code.
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

// Integer alias table for weights v[0..n-1] (n <= 64). Column masses are in
// units of 2^-32 of one column: M_i = floor((v_i / Z) * n 2^32), the
// rounding remainder goes to the last atom; small (M < 2^32) and large
// worklists are FIFO in atom order, and a large atom stays at the head of
// its list until its residual mass turns small. Full columns get threshold
// 2^32 - 1 and alias themselves.
static void build_alias(int n, const double* v, uint32_t* thr, uint8_t* alias) {
  const uint64_t kOne = 1ull << 32;
  double Z = 0.0;
  for (int i = 0; i < n; ++i) Z += v[i];
  const double scale = (double)n * 4294967296.0;
  uint64_t mass[SHP_MAX_ATOMS];
  uint64_t sum = 0;
  for (int i = 0; i < n; ++i) {
    mass[i] = (uint64_t)std::floor((v[i] / Z) * scale);
    sum += mass[i];
  }
  mass[n - 1] += (uint64_t)n * kOne - sum;
  int sq[SHP_MAX_ATOMS], lq[SHP_MAX_ATOMS];
  int sh = 0, st = 0, lh = 0, lt = 0;
  for (int i = 0; i < n; ++i) (mass[i] < kOne ? sq[st++] : lq[lt++]) = i;
  while (sh < st && lh < lt) {
    const int s = sq[sh++];
    const int l = lq[lh];
    thr[s] = (uint32_t)mass[s];
    alias[s] = (uint8_t)l;
    mass[l] -= kOne - mass[s];
    if (mass[l] < kOne) {
      ++lh;
      sq[st++] = l;
    }
  }
  for (; sh < st; ++sh) { thr[sq[sh]] = 0xFFFFFFFFu; alias[sq[sh]] = (uint8_t)sq[sh]; }
  for (; lh < lt; ++lh) { thr[lq[lh]] = 0xFFFFFFFFu; alias[lq[lh]] = (uint8_t)lq[lh]; }
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

// All device arrays of a set live in one stream-ordered allocation, filled
// by one copy from one of two pinned staging buffers that the library keeps
// (and grows) across loads; each buffer's event marks the end of its last
// upload, so a load waits only for the upload two loads back, never for the
// caller's kernels.
struct SetLayout {
  size_t atom, aux, radius, thr, alias, off, Z, order, frame, total;
};

static size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

static SetLayout set_layout(int64_t n_atoms, int32_t n_mol) {
  SetLayout L{};
  size_t o = 0;
  L.atom = o;   o = align16(o + sizeof(float4) * n_atoms);
  L.aux = o;    o = align16(o + sizeof(float2) * n_atoms);
  L.radius = o; o = align16(o + sizeof(float) * n_atoms);
  L.thr = o;    o = align16(o + sizeof(uint32_t) * n_atoms);
  L.alias = o;  o = align16(o + n_atoms);
  L.off = o;    o = align16(o + sizeof(int32_t) * (n_mol + 1));
  L.Z = o;      o = align16(o + sizeof(double) * n_mol);
  L.order = o;  o = align16(o + sizeof(int32_t) * n_mol);
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
  s->h_Z.assign(n_mol, 0.0);
  s->h_count.resize(n_mol);
  for (int32_t m = 0; m < n_mol; ++m) s->h_count[m] = (uint8_t)(offsets[m + 1] - offsets[m]);
  const SetLayout L = set_layout(n_atoms, n_mol);
  std::lock_guard<std::mutex> stage_lock(g_stage_mu);
  StageBuf* sb = nullptr;
  int rc = stage_buffer(L.total, &sb);
  if (rc) { delete s; return rc; }
  unsigned char* hb = static_cast<unsigned char*>(sb->ptr);
  float4* atom = reinterpret_cast<float4*>(hb + L.atom);
  float2* aux = reinterpret_cast<float2*>(hb + L.aux);
  float* rad = reinterpret_cast<float*>(hb + L.radius);
  uint32_t* thr = reinterpret_cast<uint32_t*>(hb + L.thr);
  uint8_t* alias = hb + L.alias;
  double* Zs = reinterpret_cast<double*>(hb + L.Z);
  // per-molecule preparation, molecules in parallel, written straight into
  // the staging buffer
  int32_t bad_mol = -1;
#pragma omp parallel for schedule(dynamic, 256)
  for (int32_t m = 0; m < n_mol; ++m) {
    const int32_t a0 = offsets[m], n = offsets[m + 1] - a0;
    double v[SHP_MAX_ATOMS];
    double Z = 0.0;
    bool ok = true;
    for (int i = 0; i < n; ++i) {
      const int64_t a = a0 + i;
      const double x = xyz[3 * a], y = xyz[3 * a + 1], z = xyz[3 * a + 2];
      const double R = radius[a];
      const double p = height ? (double)height[a] : 2.0 * std::sqrt(2.0);
      if (!std::isfinite(x) || !std::isfinite(y) || !std::isfinite(z) || !(R > 0) || !std::isfinite(R) ||
          !(p > 0) || !std::isfinite(p)) {
        ok = false;
        break;
      }
      const double alpha = ca / (R * R);
      const double t = kPi / alpha;
      v[i] = p * t * std::sqrt(t);
      Z += v[i];
      atom[a] = make_float4((float)x, (float)y, (float)z, (float)alpha);
      aux[a] = make_float2((float)(1.0 / std::sqrt(2.0 * alpha)), (float)std::log2(p));
      rad[a] = radius[a];
    }
    if (!ok) {
#pragma omp critical
      { if (bad_mol < 0 || m < bad_mol) bad_mol = m; }
      continue;
    }
    s->h_Z[m] = Z;
    Zs[m] = Z;
    build_alias(n, v, thr + a0, alias + a0);
  }
  if (bad_mol >= 0) {
    set_error("shape_set_load: molecule %d has a non-finite or non-positive coordinate, radius or height", bad_mol);
    delete s;
    return SHP_EINVAL;
  }
  order_by_size(offsets, n_mol, reinterpret_cast<int32_t*>(hb + L.order));
  std::memcpy(hb + L.off, offsets, sizeof(int32_t) * (n_mol + 1));
  // allocate and upload on the library's copy stream, then order the
  // caller's stream after the upload: the copy overlaps kernels already
  // queued on the caller's stream
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
  e = cudaMemcpyAsync(db, hb, L.frame, cudaMemcpyHostToDevice, cs);  // the frames (last) are computed on demand
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
  if (Z && s->n_mol) std::memcpy(Z, s->h_Z.data(), sizeof(double) * s->n_mol);
  if ((thr || alias) && s->n_atoms) {
    SHP_CUDA(cudaDeviceSynchronize());
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
