// Per-query top-k selection of a [n_q][n_db] score matrix: the selection step
// of the first-order prefilter (Sec. hybrid pipeline: the cheap first-order
// stage in front of the union screen).
//
// Exact and deterministic: each FP32 score becomes an order-preserving
// 32-bit key; a radix select in three passes (key bits 31..20, 19..8, 7..0:
// a 4096-bin shared-memory histogram per block, summed into a per-query
// global histogram, then one block per query finds the digit where the
// running count from the top reaches k) gives the k-th largest key v* and the
// number of keys above it. Every key above v* is kept, and of the keys equal
// to v* the first ones in database order until k are kept. The kept pairs are
// written in database order: per 2048-entry chunk a count pass, a per-query
// scan over chunks, and a block scan inside each chunk give every kept entry
// its output position.
#include <cstdint>

#include "device.cuh"
#include "internal.h"

namespace shp {
namespace {

constexpr int kDigitBits = 12;
constexpr int kBins = 1 << kDigitBits;  // 4096
constexpr int kSelThreads = 256;
constexpr int kPerThread = 8;
constexpr int kChunk = kSelThreads * kPerThread;  // 2048

struct SelState {
  uint32_t prefix;  // key bits fixed so far
  uint32_t mask;    // which bits of prefix are fixed
  uint32_t above;   // keys above the fixed prefix range
  uint32_t pad;
};

__device__ __forceinline__ uint32_t order_key(float t) {
  const uint32_t b = __float_as_uint(t);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Inclusive scan of one value over the block (kSelThreads threads); returns
// the inclusive prefix and the block total in *total.
__device__ uint32_t block_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_tot[kSelThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) warp_tot[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kSelThreads / 32 ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kSelThreads / 32) warp_tot[lane] = w;
  }
  __syncthreads();
  const uint32_t off = warp ? warp_tot[warp - 1] : 0u;
  *total = warp_tot[kSelThreads / 32 - 1];
  __syncthreads();
  return v + off;
}

// Histogram of the pass's digit over the keys that match the fixed prefix.
__global__ void __launch_bounds__(kSelThreads) hist_kernel(const float* __restrict__ T, int64_t n_db, int shift,
                                                           const SelState* st, uint32_t* hist) {
  __shared__ uint32_t h[kBins];
  const int q = blockIdx.y;
  for (int i = threadIdx.x; i < kBins; i += kSelThreads) h[i] = 0u;
  __syncthreads();
  const SelState s = st[q];
  const float* row = T + (int64_t)q * n_db;
  for (int64_t d = (int64_t)blockIdx.x * kSelThreads + threadIdx.x; d < n_db; d += (int64_t)gridDim.x * kSelThreads) {
    const uint32_t key = order_key(row[d]);
    if ((key & s.mask) == s.prefix) atomicAdd(&h[(key >> shift) & (kBins - 1)], 1u);
  }
  __syncthreads();
  uint32_t* g = hist + (int64_t)q * kBins;
  for (int i = threadIdx.x; i < kBins; i += kSelThreads)
    if (h[i]) atomicAdd(&g[i], h[i]);
}

// One block per query: the digit at which the count from the top reaches k.
__global__ void __launch_bounds__(kSelThreads) find_kernel(const uint32_t* hist, int shift, int64_t k, SelState* st) {
  const int q = blockIdx.x;
  const uint32_t* g = hist + (int64_t)q * kBins;
  constexpr int kPer = kBins / kSelThreads;  // 16 bins per thread, thread 0 holds the top ones
  const int top = kBins - 1 - threadIdx.x * kPer;
  uint32_t mine = 0;
  for (int j = 0; j < kPer; ++j) mine += g[top - j];
  uint32_t total;
  const uint32_t incl = block_scan(mine, &total);
  const uint32_t excl = incl - mine;
  const SelState s = st[q];
  // the thread whose range holds the crossing: above + excl < k <= above + incl
  if ((uint64_t)s.above + excl < (uint64_t)k && (uint64_t)k <= (uint64_t)s.above + incl) {
    uint32_t run = s.above + excl;
    for (int j = 0; j < kPer; ++j) {
      const uint32_t c = g[top - j];
      if ((uint64_t)run + c >= (uint64_t)k) {
        SelState n;
        n.prefix = s.prefix | ((uint32_t)(top - j) << shift);
        n.mask = s.mask | ((uint32_t)(kBins - 1) << shift);
        n.above = run;
        n.pad = 0u;
        st[q] = n;
        break;
      }
      run += c;
    }
  }
}

// Per chunk of 2048 entries: keys above the k-th key, and ties with it.
__global__ void __launch_bounds__(kSelThreads) count_kernel(const float* __restrict__ T, int64_t n_db,
                                                            const SelState* st, uint32_t* cnt, int64_t n_chunks) {
  const int q = blockIdx.y;
  const int64_t c = blockIdx.x;
  const uint32_t v = st[q].prefix;
  const float* row = T + (int64_t)q * n_db;
  uint32_t above = 0, ties = 0;
  const int64_t d0 = c * kChunk + (int64_t)threadIdx.x * kPerThread;
  for (int j = 0; j < kPerThread; ++j) {
    const int64_t d = d0 + j;
    if (d < n_db) {
      const uint32_t key = order_key(row[d]);
      above += key > v;
      ties += key == v;
    }
  }
  uint32_t ta, tt;
  block_scan(above, &ta);
  block_scan(ties, &tt);
  if (threadIdx.x == 0) {
    cnt[2 * ((int64_t)q * n_chunks + c)] = ta;
    cnt[2 * ((int64_t)q * n_chunks + c) + 1] = tt;
  }
}

// One block per query: exclusive prefix over chunks of both counts (in place).
__global__ void __launch_bounds__(kSelThreads) chunk_scan_kernel(uint32_t* cnt, int64_t n_chunks) {
  const int q = blockIdx.x;
  uint32_t* row = cnt + 2 * (int64_t)q * n_chunks;
  uint32_t carry_a = 0, carry_t = 0;
  for (int64_t base = 0; base < n_chunks; base += kSelThreads) {
    const int64_t c = base + threadIdx.x;
    const uint32_t a = c < n_chunks ? row[2 * c] : 0u, t = c < n_chunks ? row[2 * c + 1] : 0u;
    uint32_t ta, tt;
    const uint32_t ia = block_scan(a, &ta);
    const uint32_t it = block_scan(t, &tt);
    if (c < n_chunks) {
      row[2 * c] = carry_a + ia - a;
      row[2 * c + 1] = carry_t + it - t;
    }
    carry_a += ta;
    carry_t += tt;
    __syncthreads();
  }
}

// Writes the kept pairs of each chunk at their positions in database order.
__global__ void __launch_bounds__(kSelThreads) write_kernel(const float* __restrict__ T, int64_t n_db,
                                                            const SelState* st, const uint32_t* pre, int64_t n_chunks,
                                                            int64_t k, int32_t* pairs_q, int32_t* pairs_db) {
  const int q = blockIdx.y;
  const int64_t c = blockIdx.x;
  const SelState s = st[q];
  const uint32_t v = s.prefix;
  const uint64_t need = (uint64_t)k - s.above;
  const float* row = T + (int64_t)q * n_db;
  const int64_t d0 = c * kChunk + (int64_t)threadIdx.x * kPerThread;
  uint32_t keys[kPerThread];
  uint32_t above = 0, ties = 0;
  for (int j = 0; j < kPerThread; ++j) {
    const int64_t d = d0 + j;
    keys[j] = d < n_db ? order_key(row[d]) : 0u;
    if (d < n_db) {
      above += keys[j] > v;
      ties += keys[j] == v;
    }
  }
  uint32_t ta, tt;
  uint32_t ra = block_scan(above, &ta) - above;  // entries before this thread's, within the chunk
  uint32_t rt = block_scan(ties, &tt) - ties;
  ra += pre[2 * ((int64_t)q * n_chunks + c)];
  rt += pre[2 * ((int64_t)q * n_chunks + c) + 1];
  for (int j = 0; j < kPerThread; ++j) {
    const int64_t d = d0 + j;
    if (d >= n_db) break;
    const bool is_above = keys[j] > v, is_tie = keys[j] == v;
    if (is_above || (is_tie && rt < need)) {
      const uint64_t pos = (uint64_t)ra + ((uint64_t)rt < need ? (uint64_t)rt : need);
      const int64_t o = (int64_t)q * k + (int64_t)pos;
      pairs_q[o] = q;
      pairs_db[o] = (int32_t)d;
    }
    ra += is_above;
    rt += is_tie;
  }
}

}  // namespace
}  // namespace shp

using namespace shp;

extern "C" int fo_prefilter_select(shp_set Q, shp_set D, const float* T_fo, int64_t k, int32_t* pairs_q,
                                   int32_t* pairs_db, void* stream) {
  clear_error();
  if (!Q || !D) { set_error("fo_prefilter_select: NULL set"); return SHP_EINVAL; }
  const int64_t n_q = Q->n_mol, n_db = D->n_mol;
  if (n_q == 0) return SHP_OK;
  if (k < 1 || k > n_db) { set_error("fo_prefilter_select: k must be in 1 .. n_db"); return SHP_ERANGE; }
  if (!T_fo || !pairs_q || !pairs_db) { set_error("fo_prefilter_select: NULL array"); return SHP_EINVAL; }
  if (n_q > 65535) { set_error("fo_prefilter_select: at most 65535 queries per call"); return SHP_ERANGE; }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n_chunks = (n_db + kChunk - 1) / kChunk;
  if (n_chunks > 0x7fffffff) { set_error("fo_prefilter_select: database too large"); return SHP_ERANGE; }
  SelState* state = nullptr;
  uint32_t* hist = nullptr;
  uint32_t* cnt = nullptr;
  cudaError_t e = dev_alloc((void**)&state, sizeof(SelState) * n_q, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&hist, sizeof(uint32_t) * kBins * n_q, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&cnt, sizeof(uint32_t) * 2 * n_chunks * n_q, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(state, 0, sizeof(SelState) * n_q, st);
  const int grid_x = (int)((n_db + kSelThreads * 16 - 1) / (kSelThreads * 16));  // 16 entries per thread
  for (int pass = 0; pass < 3 && e == cudaSuccess; ++pass) {
    const int shift = pass == 0 ? 20 : (pass == 1 ? 8 : 0);
    e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kBins * n_q, st);
    if (e != cudaSuccess) break;
    hist_kernel<<<dim3((unsigned)grid_x, (unsigned)n_q), kSelThreads, 0, st>>>(T_fo, n_db, shift, state, hist);
    find_kernel<<<(unsigned)n_q, kSelThreads, 0, st>>>(hist, shift, k, state);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    count_kernel<<<dim3((unsigned)n_chunks, (unsigned)n_q), kSelThreads, 0, st>>>(T_fo, n_db, state, cnt, n_chunks);
    chunk_scan_kernel<<<(unsigned)n_q, kSelThreads, 0, st>>>(cnt, n_chunks);
    write_kernel<<<dim3((unsigned)n_chunks, (unsigned)n_q), kSelThreads, 0, st>>>(T_fo, n_db, state, cnt, n_chunks, k,
                                                                                   pairs_q, pairs_db);
    e = cudaGetLastError();
  }
  for (void* p : {(void*)state, (void*)hist, (void*)cnt})
    if (p) cudaFreeAsync(p, st);
  if (e != cudaSuccess) return cuda_fail(e, "fo_prefilter_select");
  return SHP_OK;
}

namespace shp {
namespace {

__global__ void fill_ids_kernel(int32_t* ids, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ids[i] = -1;
}

// Every listed database id d marks ids[d] = d (several pairs may mark the
// same entry with the same value); ids outside 0 .. n_db - 1 are ignored.
__global__ void mark_ids_kernel(const int32_t* pairs_db, int64_t n_pairs, int32_t n_db, int32_t* ids) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pairs) return;
  const int32_t d = pairs_db[i];
  if (d >= 0 && d < n_db) ids[d] = d;
}

}  // namespace
}  // namespace shp

extern "C" int prefilter_db_ids(shp_set D, const int32_t* pairs_db, int64_t n_pairs, int32_t* ids, void* stream) {
  clear_error();
  if (!D) { set_error("prefilter_db_ids: NULL set"); return SHP_EINVAL; }
  if (n_pairs < 0) { set_error("prefilter_db_ids: negative n_pairs"); return SHP_EINVAL; }
  const int64_t n_db = D->n_mol;
  if (n_db == 0) return SHP_OK;
  if (!ids || (n_pairs > 0 && !pairs_db)) { set_error("prefilter_db_ids: NULL array"); return SHP_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  fill_ids_kernel<<<(unsigned)((n_db + 255) / 256), 256, 0, st>>>(ids, n_db);
  if (n_pairs > 0)
    mark_ids_kernel<<<(unsigned)((n_pairs + 255) / 256), 256, 0, st>>>(pairs_db, n_pairs, (int32_t)n_db, ids);
  SHP_CUDA(cudaGetLastError());
  return SHP_OK;
}
