// mlp_loss_grad without any device allocation.
//
// Some callers cannot allocate device memory while they run: a host
// framework that owns the device allocator and forbids allocation inside its
// training step, or a latency-bound loop that cannot take an allocation. For
// them the per-block partial gradients of the loss/gradient kernels go to a
// fixed array in this file instead of stream-ordered scratch.
#include <mutex>

#include "internal.h"

namespace shp {
namespace {

constexpr int64_t kRowsPerBlock = 64;
constexpr int64_t kStaticBlocks = 128;                        // at most 128 x 64 = 8192 rows per call
constexpr int64_t kStaticRows = kStaticBlocks * kRowsPerBlock;
constexpr int64_t kRowFloats = SHP_MLP_PARAMS + 1;            // gradient entries + squared-error sum

// 128 x 6402 floats = 3.3 MB, held by every device that loads the library
// until the process exits. The backward kernel writes every entry of each
// block's row before the reduction reads it, so nothing needs clearing
// between calls; calls that overlap on the GPU race on this array.
static __device__ __align__(256) float g_partials[kStaticBlocks * kRowFloats];

std::mutex g_mu;
float* g_ptr[64] = {nullptr};

// Device address of g_partials for the current device. Looked up once per
// device, with that device current, on its first call.
int partials_ptr(float** out) {
  int dev = 0;
  SHP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("mlp_loss_grad_noalloc: device index %d is not supported", dev);
    return SHP_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess) return cuda_fail(e, "mlp_loss_grad_noalloc: cudaGetSymbolAddress");
    g_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_ptr[dev];
  return SHP_OK;
}

}  // namespace
}  // namespace shp

using namespace shp;

extern "C" int mlp_loss_grad_noalloc(const float* params, const float* x, const float* target,
                                     const int32_t* rows, int64_t n, float* grad, double* loss, void* stream) {
  clear_error();
  if (n <= 0 || !params || !x || !target || !grad || !loss) {
    set_error("mlp_loss_grad_noalloc: bad arguments");
    return SHP_EINVAL;
  }
  if (n > kStaticRows) {
    set_error("mlp_loss_grad_noalloc: %lld rows exceed the fixed scratch of %lld rows per call",
              (long long)n, (long long)kStaticRows);
    return SHP_ERANGE;
  }
  float* part = nullptr;
  const int rc = partials_ptr(&part);
  if (rc) return rc;
  return mlp_loss_grad_into(params, x, target, rows, n, part, grad, loss, (cudaStream_t)stream);
}
