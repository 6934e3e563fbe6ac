// tsf_static.cu -- tsf_zero_pairs_static: the zero-persistence pairs of a
// field, computed without allocating any device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a framework
// which owns all device memory through its own pool, or a latency-critical
// loop where cudaMalloc's implicit device-wide synchronisation is not
// acceptable.  This entry point takes their input and output buffers and does
// all its intermediate work (vertex order, ranks, sort scratch, counters) in
// one file-scope device array of fixed size, which every GPU that loads this
// library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/tsf.h"
#include "tsf_kernels.cuh"

namespace {

constexpr int64_t kMaxV = TSF_STATIC_MAX_VERTICES;
// counter (2 words) + status (1) padding to 64 words, order, rank, sort scratch
constexpr int64_t kSortWords = 4 * kMaxV + 1024 + 64 + 4 * 256 * (kMaxV / 4096 + 1) + 64;
constexpr int64_t kWords = 64 + 2 * kMaxV + kSortWords;

static __device__ __align__(256) uint32_t g_scratch[kWords];

std::mutex g_mu;
uint32_t* g_addr[64] = {};  // device address of g_scratch, per device

// Host code may not use g_scratch's name as a device address: fetch the real
// address once per device, with that device current.
int scratch_address(uint32_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TSF_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return TSF_ECUDA;
    g_addr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_addr[dev];
  return TSF_OK;
}

}  // namespace

extern "C" int tsf_zero_pairs_static(int lx, int ly, int lz, const float* values, uint64_t* out, int64_t cap_pairs,
                                     int64_t* n_out, void* cuda_stream) {
  if (!values || !n_out || cap_pairs < 0 || (cap_pairs > 0 && !out) || lx < 2 || ly < 2 || lz < 2)
    return TSF_EINVAL;
  int64_t nv = (int64_t)lx * ly * lz;
  if (nv > kMaxV) return TSF_EINVAL;
  if (tsf::sort_scratch_words(nv) + 2 * nv + 64 > kWords) return TSF_EINTERNAL;
  uint32_t* base = nullptr;
  int r = scratch_address(&base);
  if (r != TSF_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(base);
  uint32_t* status = base + 2;
  uint32_t* order = base + 64;
  uint32_t* rank = order + nv;
  uint32_t* sort = rank + nv;
  // the array keeps the previous call's contents: clear what must start at zero
  if (cudaMemsetAsync(base, 0, 64 * sizeof(uint32_t), st) != cudaSuccess) return TSF_ECUDA;
  tsf::vertex_order(values, nv, order, rank, nullptr, sort, status, st);
  tsf::Dims d;
  d.lx = lx;
  d.ly = ly;
  d.lz = lz;
  d.nv = nv;
  tsf::launch_zero_pairs(d, rank, reinterpret_cast<unsigned long long*>(out), cap_pairs, counter, status, st);
  // launch errors are checked right after the launches, with a peek that
  // leaves the thread's error state as the caller had it
  if (cudaPeekAtLastError() != cudaSuccess) return TSF_ECUDA;
  unsigned long long n = 0;
  uint32_t s = 0;
  if (cudaMemcpyAsync(&n, counter, sizeof(n), cudaMemcpyDeviceToHost, st) != cudaSuccess) return TSF_ECUDA;
  if (cudaMemcpyAsync(&s, status, sizeof(s), cudaMemcpyDeviceToHost, st) != cudaSuccess) return TSF_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return TSF_ECUDA;
  *n_out = (int64_t)n;
  // the same mapping as every other entry point: NaN/Inf, then a device wait
  // that gave up (a sort look-back spin), then an internal inconsistency
  const int code = tsf::status_code(s);
  if (code != TSF_OK) return code;
  return (int64_t)n > cap_pairs ? TSF_ECAPACITY : TSF_OK;
}
