// k_order.cu -- incremental update of the vertex order (Section 2.1) after a
// gradient step that changed few values.  The vertices the step left alone
// keep their relative order, so the new order is the merge of the old order
// without the updated vertices and the updated vertices sorted by their new
// (value key, id):
//   a kept vertex at old position i lands at  i - #{updated u : rank(u) < i}
//                                               + #{updated u : key'(u) < key(i)}
//   the q-th updated vertex (by new key) at     q + #{kept vertices with key < key'(u)}.
// The old order's sorted keys (kept from the previous ordering) give the
// second count by a binary search, even though the updated vertices' old
// values are gone.
#include <algorithm>
#include <atomic>

#include "../../include/tsf.h"
#include "tsf_group.cuh"
#include "tsf_kernels.cuh"

namespace tsf {

constexpr int kOT = 1024;  // threads of the one-block kernels

// The old ranks of the updated vertices as a bitmap over positions.
__global__ void k_order_mark(const uint32_t* __restrict__ upd, int nu, const uint32_t* __restrict__ rank,
                             uint32_t* __restrict__ ubits) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nu) {
    uint32_t r = __ldg(rank + upd[q]);
    atomicOr(ubits + (r >> 5), 1u << (r & 31));
  }
}

constexpr int kCntT = 1024;  // words per counting block

// ucnt[w] = set bits in ubits[blk*1024 .. w) for w's block blk, btot[blk] =
// the block's total (coalesced, one word per thread).
__global__ void __launch_bounds__(kCntT) k_order_count(const uint32_t* __restrict__ ubits, int64_t nw,
                                                       uint32_t* __restrict__ ucnt, uint32_t* __restrict__ btot) {
  __shared__ uint32_t wsum[kCntT / 32];
  const int64_t w = (int64_t)blockIdx.x * kCntT + threadIdx.x;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  uint32_t c = w < nw ? (uint32_t)__popc(__ldg(ubits + w)) : 0u;
  uint32_t inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[wi] = inc;
  __syncthreads();
  if (wi == 0) {
    uint32_t x = wsum[lane], xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xFFFFFFFFu, xi, o);
      if (lane >= o) xi += t;
    }
    wsum[lane] = xi - x;
    if (lane == 31) btot[blockIdx.x] = xi;
  }
  __syncthreads();
  if (w < nw) ucnt[w] = wsum[wi] + inc - c;
}

// One block: boff[b] = set bits in the counting blocks before b, and B = the
// updated vertices' new keys value_key << 32 | id, ascending (bitonic sort
// in shared memory).
__global__ void __launch_bounds__(kOT) k_order_prep(const uint32_t* __restrict__ upd, int nu,
                                                    const float* __restrict__ f, const uint32_t* __restrict__ btot,
                                                    int nblk, uint32_t* __restrict__ boff,
                                                    unsigned long long* __restrict__ B, uint32_t* status) {
  extern __shared__ __align__(16) unsigned long long sb[];
  __shared__ uint32_t part[kOT];
  const int tid = threadIdx.x;
  const int per = (nblk + kOT - 1) / kOT;
  const int b0 = tid * per, b1 = b0 + per < nblk ? b0 + per : nblk;
  uint32_t mine = 0;
  for (int b = b0; b < b1; ++b) mine += btot[b];
  part[tid] = mine;
  __syncthreads();
  for (int o = 1; o < kOT; o <<= 1) {  // inclusive scan of the runs' totals
    uint32_t x = tid >= o ? part[tid - o] : 0u;
    __syncthreads();
    part[tid] += x;
    __syncthreads();
  }
  uint32_t run = part[tid] - mine;
  for (int b = b0; b < b1; ++b) {
    boff[b] = run;
    run += btot[b];
  }
  int n2 = 1;
  while (n2 < nu) n2 <<= 1;
  bool bad = false;
  for (int i = tid; i < n2; i += kOT) {
    unsigned long long k = 0ull;
    if (i < nu) {
      uint32_t u = upd[i];
      float x = __ldg(f + u);
      bad |= !isfinite(x);
      k = ((unsigned long long)value_key(x) << 32) | u;
    }
    sb[i] = k;
  }
  if (bad) atomicOr(status, kErrNaN);
  __syncthreads();
  group_sort_desc<kOT>(sb, n2);  // keys are > 0, the padding sorts last
  for (int i = tid; i < nu; i += kOT) B[i] = sb[nu - 1 - i];
}

__device__ __forceinline__ int count_below(const unsigned long long* __restrict__ s, int n, unsigned long long x) {
  int lo = 0, hi = n;  // #{k : s[k] < x}, s ascending
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (__ldg(s + mid) < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
// #{updated vertices with old rank < i}
__device__ __forceinline__ int updated_below(const uint32_t* __restrict__ ubits, const uint32_t* __restrict__ ucnt,
                                             const uint32_t* __restrict__ boff, int64_t i) {
  int64_t w = i >> 5;
  return (int)(__ldg(boff + (w >> 10)) + __ldg(ucnt + w) + __popc(__ldg(ubits + w) & ((1u << (i & 31)) - 1u)));
}

constexpr int kKeepT = 256, kKeepC = 16;  // threads, positions per lane
constexpr int kKeepTile = kKeepT * kKeepC;

// The kept vertices: each lane walks old positions i0, i0 + 32, ... and
// advances its count of smaller new keys (non-decreasing in i).
__global__ void __launch_bounds__(kKeepT) k_order_keep(int64_t n, const uint32_t* __restrict__ order,
                                                       const uint32_t* __restrict__ skey,
                                                       const uint32_t* __restrict__ ubits,
                                                       const uint32_t* __restrict__ ucnt,
                                                       const uint32_t* __restrict__ boff, int nu,
                                                       const unsigned long long* __restrict__ B,
                                                       uint32_t* __restrict__ order2, uint32_t* __restrict__ skey2,
                                                       uint32_t* __restrict__ rank) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * kKeepTile + (int64_t)w * (32 * kKeepC) + lane;
  if (i0 >= n) return;
  int b = count_below(B, nu, ((unsigned long long)__ldg(skey + i0) << 32) | __ldg(order + i0));
#pragma unroll 4
  for (int k = 0; k < kKeepC; ++k) {
    int64_t i = i0 + 32 * k;
    if (i >= n) break;
    uint32_t v = __ldg(order + i);
    uint32_t kk = __ldg(skey + i);
    if ((__ldg(ubits + (i >> 5)) >> (i & 31)) & 1u) continue;  // updated: placed by k_order_moved
    unsigned long long key = ((unsigned long long)kk << 32) | v;
    while (b < nu && __ldg(B + b) < key) ++b;
    uint32_t ni = (uint32_t)(i - updated_below(ubits, ucnt, boff, i) + b);
    order2[ni] = v;
    skey2[ni] = kk;
    rank[v] = ni;
  }
}

// The updated vertices, one thread each.
__global__ void k_order_moved(int64_t n, const uint32_t* __restrict__ order, const uint32_t* __restrict__ skey,
                              const uint32_t* __restrict__ ubits, const uint32_t* __restrict__ ucnt,
                              const uint32_t* __restrict__ boff, int nu, const unsigned long long* __restrict__ B,
                              uint32_t* __restrict__ order2,
                              uint32_t* __restrict__ skey2, uint32_t* __restrict__ rank) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nu) return;
  unsigned long long key = B[q];
  int64_t lo = 0, hi = n;  // old positions whose (old key, id) is below key
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    unsigned long long k = ((unsigned long long)__ldg(skey + mid) << 32) | __ldg(order + mid);
    if (k < key) lo = mid + 1;
    else hi = mid;
  }
  int la = lo < n ? updated_below(ubits, ucnt, boff, lo) : nu;
  uint32_t ni = (uint32_t)(q + lo - la);
  uint32_t u = (uint32_t)key;
  order2[ni] = u;
  skey2[ni] = (uint32_t)(key >> 32);
  rank[u] = ni;
}

void vertex_order_incremental(const float* f, int64_t n, const uint32_t* upd, int nu, const uint32_t* order,
                              const uint32_t* skey, uint32_t* order2, uint32_t* skey2, uint32_t* rank,
                              uint32_t* ubits, uint32_t* ucnt, unsigned long long* B, uint32_t* status,
                              cudaStream_t st) {
  if (nu <= 0 || nu > kIncOrderMax) return;
  const int64_t nw = (n + 31) / 32;
  const int nblk = (int)((nw + kCntT - 1) / kCntT);
  uint32_t* btot = ucnt + nw;  // ucnt holds nw + 2 * nblk words
  uint32_t* boff = btot + nblk;
  const size_t smem = sizeof(unsigned long long) * (size_t)kIncOrderMax;
  int dev = 0;
  cudaGetDevice(&dev);
  static std::atomic<bool> attr[64] = {};  // fields may be driven from several host threads
  if (dev >= 0 && dev < 64 && !attr[dev].load(std::memory_order_acquire)) {
    cudaFuncSetAttribute(k_order_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr[dev].store(true, std::memory_order_release);
  }
  cudaMemsetAsync(ubits, 0, sizeof(uint32_t) * (size_t)nw, st);
  k_order_mark<<<(nu + 255) / 256, 256, 0, st>>>(upd, nu, rank, ubits); note_launch();
  k_order_count<<<nblk, kCntT, 0, st>>>(ubits, nw, ucnt, btot); note_launch();
  k_order_prep<<<1, kOT, smem, st>>>(upd, nu, f, btot, nblk, boff, B, status); note_launch();
  k_order_keep<<<(unsigned)((n + kKeepTile - 1) / kKeepTile), kKeepT, 0, st>>>(n, order, skey, ubits, ucnt, boff, nu,
                                                                              B, order2, skey2, rank); note_launch();
  k_order_moved<<<(nu + 255) / 256, 256, 0, st>>>(n, order, skey, ubits, ucnt, boff, nu, B, order2, skey2, rank);
  note_launch();
}

int64_t order_count_words(int64_t n) {
  const int64_t nw = (n + 31) / 32;
  return nw + 2 * ((nw + kCntT - 1) / kCntT);
}

}  // namespace tsf
