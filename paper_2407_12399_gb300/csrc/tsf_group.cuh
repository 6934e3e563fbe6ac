// tsf_group.cuh -- cooperative helpers of a thread group (part of a warp,
// a warp or a block): barrier, exclusive scan, and a descending bitonic sort of keyed
// entries held in registers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace tsf {

// A keyed entry: 64-bit sort key and a 32-bit payload (the parity mask of
// a frontier entry of the saddle-saddle reduction).
struct __align__(16) FEnt {
  unsigned long long key;
  uint32_t mask;
  uint32_t pad;
};

// A group is GS threads: an aligned part of a warp (GS = 8 or 16, lanes
// [GS*k, GS*(k+1))), one warp (GS = 32) or the whole block (GS = blockDim.x
// > 32).  Helpers for the group of the calling thread.
template <int GS>
__device__ __forceinline__ int gtid() {
  return GS > 32 ? (int)threadIdx.x : (int)(threadIdx.x & (GS - 1));
}
template <int GS>
__device__ __forceinline__ unsigned gmask() {
  static_assert(GS > 32 || (GS >= 1 && (GS & (GS - 1)) == 0), "a part of a warp is a power of two");
  if (GS >= 32) return 0xFFFFFFFFu;
  // GS < 32 here; the guard keeps the shift in range when GS = 32 instantiates this line
  constexpr unsigned low = GS >= 32 ? 0xFFFFFFFFu : ((1u << (GS & 31)) - 1u);
  return low << ((threadIdx.x & 31u) & ~(unsigned)(GS - 1));
}
template <int GS>
__device__ __forceinline__ void gsync() {
  if (GS > 32) __syncthreads();
  else __syncwarp(gmask<GS>());
}

template <int GS>
__device__ __forceinline__ int gscan(int v, int& total, int* sm) {  // exclusive; sm: >= GS/32 + 1 ints (GS > 32)
  if (GS <= 32) {
    const unsigned m = gmask<GS>();
    const int lane = gtid<GS>();
    int inc = v;
#pragma unroll
    for (int o = 1; o < GS; o <<= 1) {
      int t = __shfl_up_sync(m, inc, o, GS);
      if (lane >= o) inc += t;
    }
    total = __shfl_sync(m, inc, GS - 1, GS);
    return inc - v;
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sm[w] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int k = 0; k < GS / 32; ++k) {
      int t = sm[k];
      sm[k] = run;
      run += t;
    }
    sm[GS / 32] = run;
  }
  __syncthreads();
  int res = sm[w] + inc - v;
  total = sm[GS / 32];
  __syncthreads();
  return res;
}

// Descending bitonic sort of a[0..n2) (n2 a power of two) by key, 64-bit
// values (shared or global memory of the group; its barrier orders both).
template <int GS>
__device__ void group_sort_desc(unsigned long long* a, int n2) {
  for (int size = 2; size <= n2; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = gtid<GS>(); i < n2; i += GS) {
        int jx = i ^ stride;
        if (jx > i) {
          bool desc = (i & size) == 0;
          unsigned long long x = a[i], y = a[jx];
          if ((x < y) == desc) {
            a[i] = y;
            a[jx] = x;
          }
        }
      }
      gsync<GS>();
    }
}
// Descending bitonic sort of keyed entries a[0..n) in shared memory (a[]
// holds the next power of two; compact code for the rare long stages).
template <int GS>
__device__ void group_sort_smem(FEnt* a, int n) {
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  for (int i = n + gtid<GS>(); i < n2; i += GS) {
    a[i].key = 0ull;
    a[i].mask = 0u;
  }
  gsync<GS>();
  for (int size = 2; size <= n2; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = gtid<GS>(); i < n2; i += GS) {
        int jx = i ^ stride;
        if (jx > i) {
          bool desc = (i & size) == 0;
          FEnt x = a[i], y = a[jx];
          if ((x.key < y.key) == desc) {
            a[i] = y;
            a[jx] = x;
          }
        }
      }
      gsync<GS>();
    }
}

// Descending bitonic sort of a[0..n) (n <= GS * E) by key, E entries per
// thread in registers (entry i = thread * E + e): strides below E swap
// registers, strides below min(GS, 32) E exchange with a lane by shuffles,
// longer strides (blocks of several warps only) go through a[] in shared
// memory.
// Equal keys may stay in either order.  All threads of the group call it.
template <int GS, int E>
__device__ void group_sort_reg(FEnt* a, int n) {
  constexpr int N = GS * E;
  constexpr int W = GS < 32 ? GS : 32;  // threads that exchange by shuffles
  const int tid = gtid<GS>(), lane = tid & 31;
  const unsigned gm = gmask<GS>();
  unsigned long long k[E];
  uint32_t m[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    int i = tid * E + e;
    k[e] = 0ull;
    m[e] = 0u;
    if (i < n) {
      k[e] = a[i].key;
      m[e] = a[i].mask;
    }
  }
#pragma unroll
  for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride < E) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          int p = e ^ stride;
          if (p > e) {
            bool desc = ((tid * E + e) & size) == 0;
            if ((k[e] < k[p]) == desc) {
              unsigned long long tk = k[e];
              k[e] = k[p];
              k[p] = tk;
              uint32_t tm = m[e];
              m[e] = m[p];
              m[p] = tm;
            }
          }
        }
      } else if (stride < W * E) {
        const int lx = stride / E;
        const bool lower = (lane & lx) == 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          unsigned long long ok = __shfl_xor_sync(gm, k[e], lx);
          uint32_t om = __shfl_xor_sync(gm, m[e], lx);
          bool desc = ((tid * E + e) & size) == 0;
          bool take = lower == desc ? ok > k[e] : ok < k[e];
          if (take) {
            k[e] = ok;
            m[e] = om;
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          a[tid * E + e].key = k[e];
          a[tid * E + e].mask = m[e];
        }
        __syncthreads();
        const bool lower = ((tid * E) & stride) == 0;
        unsigned long long ok[E];
        uint32_t om[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
          int jx = (tid * E + e) ^ stride;
          ok[e] = a[jx].key;
          om[e] = a[jx].mask;
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) {
          bool desc = ((tid * E + e) & size) == 0;
          bool take = lower == desc ? ok[e] > k[e] : ok[e] < k[e];
          if (take) {
            k[e] = ok[e];
            m[e] = om[e];
          }
        }
      }
    }
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    a[tid * E + e].key = k[e];
    a[tid * E + e].mask = m[e];
  }
  gsync<GS>();
}

}  // namespace tsf
