// k_sort.cu -- global vertex order (Section 2.1 / Section 2.2): a stable LSD
// radix sort of (value key, vertex id), 4 passes of 8 bits, then the rank
// scatter.  Stability of every pass keeps equal values in id order, which is
// the id tie-break of the vertex order.
#include <algorithm>

#include "tsf_kernels.cuh"

namespace tsf {

constexpr int kRT = 256;            // threads
constexpr int kRW = kRT / 32;       // warps
constexpr int kRI = 16;             // items per thread
constexpr int kRTile = kRT * kRI;   // 4096 items per tile
constexpr int kRWarpItems = kRTile / kRW;  // 512 items per warp, contiguous

__device__ __forceinline__ uint32_t rs_key(bool first, const float* __restrict__ f, const uint32_t* __restrict__ keys,
                                           int64_t i) {
  return first ? value_key(__ldg(f + i)) : __ldg(keys + i);
}

__global__ void k_rank_scatter(int64_t n, const uint32_t* __restrict__ order, uint32_t* __restrict__ rank) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rank[__ldg(order + i)] = (uint32_t)i;
}

// ---- exclusive scan of uint32 (block sums, one-block scan, apply) ---------
constexpr int kST = 1024, kSI = 4, kSTile = kST * kSI;

__device__ __forceinline__ uint32_t block_exscan_u32(uint32_t v, uint32_t& total) {
  static_assert(kST == 1024, "one warp scans the 32 warp sums");
  __shared__ uint32_t sw[kST / 32 + 1];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sw[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = sw[lane];
    uint32_t si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xFFFFFFFFu, si, o);
      if (lane >= o) si += t;
    }
    sw[lane] = si - s;
    if (lane == 31) sw[32] = si;
  }
  __syncthreads();
  uint32_t res = sw[wid] + inc - v;
  total = sw[32];
  __syncthreads();
  return res;
}

__global__ void k_scan_sums(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ sums) {
  uint32_t acc = 0;
  int64_t base = (int64_t)blockIdx.x * kSTile;
  for (int k = 0; k < kSI; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * kSI + k;
    if (i < n) acc += in[i];
  }
  uint32_t tot = 0;
  block_exscan_u32(acc, tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_top(uint32_t* __restrict__ sums, int nb) {
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b = 0; b < nb; b += kST) {
    int i = b + threadIdx.x;
    uint32_t v = i < nb ? sums[i] : 0;
    uint32_t tot = 0;
    uint32_t ex = block_exscan_u32(v, tot);
    uint32_t c = carry;
    if (i < nb) sums[i] = c + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry = c + tot;
    __syncthreads();
  }
}

__global__ void k_scan_apply(const uint32_t* __restrict__ in, int64_t n, const uint32_t* __restrict__ sums,
                             uint32_t* __restrict__ out) {
  int64_t base = (int64_t)blockIdx.x * kSTile;
  uint32_t loc[kSI];
  uint32_t acc = 0;
  for (int k = 0; k < kSI; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * kSI + k;
    loc[k] = i < n ? in[i] : 0;
    acc += loc[k];
  }
  uint32_t tot = 0;
  uint32_t ex = block_exscan_u32(acc, tot) + sums[blockIdx.x];
  for (int k = 0; k < kSI; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * kSI + k;
    if (i < n) out[i] = ex;
    ex += loc[k];
  }
}

void exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* sums, cudaStream_t st) {
  int nb = (int)((n + kSTile - 1) / kSTile);
  if (nb == 0) return;
  k_scan_sums<<<nb, kST, 0, st>>>(in, n, sums); note_launch();
  k_scan_top<<<1, kST, 0, st>>>(sums, nb); note_launch();
  k_scan_apply<<<nb, kST, 0, st>>>(in, n, sums, out); note_launch();
}

// ---------------------------------------------------------------------------
// Onesweep: one histogram pass for the four digits, then one kernel per digit
// that ranks a tile, publishes its digit counts and finds its global offsets
// by a decoupled look-back over the earlier tiles (tile ids come from an
// atomic counter, so a block only waits for tiles that started before it).
// ---------------------------------------------------------------------------
constexpr uint32_t kLbAgg = 1u << 30, kLbInc = 2u << 30, kLbVal = (1u << 30) - 1;
constexpr int kSpinLimit = 1 << 24;

__global__ void k_os_hist(int64_t n, const float* __restrict__ f, uint32_t* __restrict__ hist, uint32_t* status) {
  __shared__ uint32_t h[4][256];
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  bool bad = false;
  const int lane = threadIdx.x & 31;
  // whole warps iterate together so that equal digits are added once per warp
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    int64_t i = i0 + threadIdx.x;
    uint32_t k = 0;
    bool in = i < n;
    if (in) {
      float x = __ldg(f + i);
      bad |= !isfinite(x);
      k = value_key(x);
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      uint32_t dg = in ? (k >> (8 * d)) & 255u : 256u;
      unsigned peers = __match_any_sync(0xFFFFFFFFu, dg);
      if (dg < 256 && lane == __ffs(peers) - 1) atomicAdd(&h[d][dg], (uint32_t)__popc(peers));
    }
  }
  if (bad) atomicOr(status, kErrNaN);
  __syncthreads();
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
    uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(hist + i, c);
  }
}

// exclusive scan of each digit's 256 counts (one block of 256 threads)
__global__ void k_os_bases(uint32_t* __restrict__ hist) {
  __shared__ uint32_t t[256];
  for (int pass = 0; pass < 4; ++pass) {
    uint32_t v = hist[pass * 256 + threadIdx.x];
    t[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
      uint32_t a = threadIdx.x >= o ? t[threadIdx.x - o] : 0u;
      __syncthreads();
      t[threadIdx.x] += a;
      __syncthreads();
    }
    hist[pass * 256 + threadIdx.x] = t[threadIdx.x] - v;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kRT) k_os_pass(int64_t n, int shift, bool first, bool last,
                                                 const float* __restrict__ f, const uint32_t* __restrict__ keys_in,
                                                 const uint32_t* __restrict__ vals_in, uint32_t* __restrict__ keys_out,
                                                 uint32_t* __restrict__ vals_out, const uint32_t* __restrict__ bases,
                                                 uint32_t* lookback, uint32_t* tile_counter, uint32_t* status) {
  __shared__ uint32_t whist[kRW][256];
  __shared__ uint32_t s_off[256];
  __shared__ uint32_t s_tile;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
  for (int i = threadIdx.x; i < kRW * 256; i += kRT) (&whist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t tile = s_tile;
  const int64_t wbase = (int64_t)tile * kRTile + (int64_t)w * kRWarpItems;
  uint32_t key[kRI], val[kRI];
#pragma unroll
  for (int c = 0; c < kRI; ++c) {
    int64_t i = wbase + c * 32 + lane;
    key[c] = 0xFFFFFFFFu;
    val[c] = 0;
    if (i < n) {
      key[c] = first ? value_key(__ldg(f + i)) : __ldg(keys_in + i);
      val[c] = first ? (uint32_t)i : __ldg(vals_in + i);
    }
  }
  // per-warp digit counts (the warp's 512 items are contiguous and in order)
#pragma unroll
  for (int c = 0; c < kRI; ++c) {
    int64_t i = wbase + c * 32 + lane;
    uint32_t dg = i < n ? (key[c] >> shift) & 255u : 256u;
    unsigned peers = __match_any_sync(0xFFFFFFFFu, dg);
    if (dg < 256 && lane == __ffs(peers) - 1) whist[w][dg] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // tile count per digit; per-warp bases inside the tile
  const uint32_t d = threadIdx.x;
  uint32_t cnt = 0;
#pragma unroll
  for (int ww = 0; ww < kRW; ++ww) {
    uint32_t c = whist[ww][d];
    whist[ww][d] = cnt;
    cnt += c;
  }
  volatile uint32_t* lb = lookback;
  uint32_t excl = 0;
  if (tile == 0) {
    lb[d] = kLbInc | cnt;
  } else {
    lb[(int64_t)tile * 256 + d] = kLbAgg | cnt;
    int64_t t = (int64_t)tile - 1;
    int spins = 0;
    while (t >= 0) {
      uint32_t word = lb[t * 256 + d];
      uint32_t flag = word & ~kLbVal;
      if (flag == 0) {
        if (++spins > kSpinLimit) {
          atomicOr(status, kErrSpin);
          break;
        }
        continue;
      }
      excl += word & kLbVal;
      if (flag == kLbInc) break;
      --t;
    }
    lb[(int64_t)tile * 256 + d] = kLbInc | (excl + cnt);
  }
  s_off[d] = bases[d] + excl;
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int c = 0; c < kRI; ++c) {
    int64_t i = wbase + c * 32 + lane;
    uint32_t dg = i < n ? (key[c] >> shift) & 255u : 256u;
    unsigned peers = __match_any_sync(0xFFFFFFFFu, dg);
    uint32_t pos = 0;
    if (dg < 256) pos = s_off[dg] + whist[w][dg] + __popc(peers & lt);
    __syncwarp();
    if (dg < 256) {
      if (keys_out) keys_out[pos] = key[c];
      vals_out[pos] = val[c];
      if (lane == __ffs(peers) - 1) whist[w][dg] += __popc(peers);
    }
    __syncwarp();
  }
}

// Digit histograms of u32 keys (all four 8-bit digits at once).
__global__ void k_os_hist_u32(int64_t n, const uint32_t* __restrict__ keys, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[4][256];
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    const int64_t i = i0 + threadIdx.x;
    const bool in = i < n;
    const uint32_t k = in ? __ldg(keys + i) : 0u;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const uint32_t dg = in ? (k >> (8 * d)) & 255u : 256u;
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, dg);
      if (dg < 256 && lane == __ffs(peers) - 1) atomicAdd(&h[d][dg], (uint32_t)__popc(peers));
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(hist + i, c);
  }
}

// Stable sort of (key, value) pairs by the u32 key: histogram, then four
// onesweep passes.  keys_out may be null.  scratch: sort_scratch_words(n).
void sort_u32_pairs(const uint32_t* keys, const uint32_t* vals, int64_t n, uint32_t* keys_out, uint32_t* vals_out,
                    uint32_t* scratch, uint32_t* status, cudaStream_t st) {
  if (n <= 0) return;
  const int ntiles = (int)((n + kRTile - 1) / kRTile);
  uint32_t* kA = scratch;
  uint32_t* vA = kA + n;
  uint32_t* kB = vA + n;
  uint32_t* vB = kB + n;
  uint32_t* hist = vB + n;
  uint32_t* counters = hist + 1024;
  uint32_t* lookback = counters + 64;
  cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (1024 + 64 + 4 * 256 * (size_t)ntiles), st);
  k_os_hist_u32<<<std::min(ntiles, 1216), 256, 0, st>>>(n, keys, hist); note_launch();
  k_os_bases<<<1, 256, 0, st>>>(hist); note_launch();
  const uint32_t* kin = keys;
  const uint32_t* vin = vals;
  for (int pass = 0; pass < 4; ++pass) {
    const bool last = pass == 3;
    uint32_t* kout = last ? keys_out : ((pass & 1) ? kB : kA);
    uint32_t* vout = last ? vals_out : ((pass & 1) ? vB : vA);
    if (!last && !kout) kout = (pass & 1) ? kB : kA;
    k_os_pass<<<ntiles, kRT, 0, st>>>(n, 8 * pass, false, last, nullptr, kin, vin, kout, vout, hist + 256 * pass,
                                      lookback + (size_t)pass * 256 * ntiles, counters + pass, status); note_launch();
    kin = kout;
    vin = vout;
  }
}

int64_t sort_scratch_words(int64_t n) {
  int64_t ntiles = (n + kRTile - 1) / kRTile;
  // keys/ids ping-pong, 4 digit histograms, 4 tile counters, 4 look-back tables
  return 4 * n + 1024 + 64 + 4 * 256 * ntiles + 64;
}

// Vertex order: order[r] = id of the r-th vertex, rank[id] = r.
void vertex_order(const float* f, int64_t n, uint32_t* order, uint32_t* rank, uint32_t* skey, uint32_t* scratch,
                  uint32_t* status, cudaStream_t st) {
  int ntiles = (int)((n + kRTile - 1) / kRTile);
  uint32_t* kA = scratch;
  uint32_t* vA = kA + n;
  uint32_t* kB = vA + n;
  uint32_t* vB = kB + n;
  uint32_t* hist = vB + n;
  uint32_t* counters = hist + 1024;
  uint32_t* lookback = counters + 64;
  cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (1024 + 64 + 4 * 256 * (size_t)ntiles), st);
  k_os_hist<<<std::min(ntiles, 1216), 256, 0, st>>>(n, f, hist, status); note_launch();
  k_os_bases<<<1, 256, 0, st>>>(hist); note_launch();
  const uint32_t* kin = nullptr;
  const uint32_t* vin = nullptr;
  for (int pass = 0; pass < 4; ++pass) {
    bool first = pass == 0, last = pass == 3;
    uint32_t* kout = last ? skey : ((pass & 1) ? kB : kA);
    uint32_t* vout = last ? order : ((pass & 1) ? vB : vA);
    k_os_pass<<<ntiles, kRT, 0, st>>>(n, 8 * pass, first, last, f, kin, vin, kout, vout, hist + 256 * pass,
                                      lookback + (size_t)pass * 256 * ntiles, counters + pass, status); note_launch();
    kin = kout;
    vin = vout;
  }
  k_rank_scatter<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, order, rank); note_launch();
}

}  // namespace tsf
