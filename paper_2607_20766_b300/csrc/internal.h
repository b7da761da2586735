// Host-side internals shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "shape.h"

struct shp_set_s {
  int device = 0;
  int32_t n_mol = 0;
  int64_t n_atoms = 0;
  int32_t max_atoms = 0;
  // device arrays (owned: one allocation, dbase)
  unsigned char* dbase = nullptr;
  float4* atom = nullptr;    // [n_atoms] x, y, z, alpha
  float2* aux = nullptr;     // [n_atoms] sigma = 1/sqrt(2 alpha), log2 p
  uint32_t* thr = nullptr;   // [n_atoms] alias thresholds
  uint8_t* alias = nullptr;  // [n_atoms] alias targets (local index)
  int32_t* off = nullptr;    // [n_mol + 1]
  double* Z = nullptr;       // [n_mol] mixture mass
  int32_t* order = nullptr;  // [n_mol] molecule ids, atom count descending
  float* radius = nullptr;   // [n_atoms] van der Waals radius (A)
  float* frame = nullptr;    // [n_mol][12] principal frame: centroid (3), axes E (3x3 row-major,
                             // columns = axes, det +1); computed on the device at first use
  bool frames_ready = false;
  cudaEvent_t frames_done = nullptr;
  std::mutex frames_mu;
  // host mirror of the atom counts
  std::vector<uint8_t> h_count;
  int32_t h_off_count(int32_t m) const { return h_count[m]; }
};

namespace shp {

// Read-only device view of a set, passed to kernels by value.
struct SetView {
  const float4* atom;
  const float2* aux;
  const uint32_t* thr;
  const uint8_t* alias;
  const int32_t* off;
  const double* Z;
  const float* frame;
  const float* radius;
  int32_t n_mol;
};

// Stream-ordered device allocation used by every library call; fails with
// cudaErrorMemoryAllocation, without calling CUDA, while the test hook of
// shp_fail_next_allocations has failures pending.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t stream);

// Makes the principal frames of s available to work enqueued on `stream`
// after this call (computes them on the device the first time).
int ensure_frames(shp_set_s* s, cudaStream_t stream);

inline SetView view(const shp_set_s* s) {
  return SetView{s->atom, s->aux, s->thr, s->alias, s->off, s->Z, s->frame, s->radius, s->n_mol};
}

// overlap_estimate with item k drawing from stream mc->stream_base + k / group
// (group consecutive items share their random numbers).
int overlap_estimate_grouped(shp_set A, const int32_t* ia, shp_set B, const int32_t* ib, int64_t n_pairs,
                             const float* poseB, const shp_mc* mc, double* est, double* se, int64_t group,
                             cudaStream_t stream);

int mlp_loss_grad_into(const float* params, const float* x, const float* target, const int32_t* rows, int64_t n,
                       float* part, float* grad, double* loss, cudaStream_t st);

void set_error(const char* fmt, ...);
void clear_error();
int cuda_fail(cudaError_t e, const char* what);

}  // namespace shp

#define SHP_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return shp::cuda_fail(e_, #call); \
  } while (0)
