// tsf_internal.cuh -- device-side building blocks shared by the kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "tsf_geo.cuh"

namespace tsf {

// Device status word bits (a kernel that hits a bound sets one and returns).
enum : uint32_t {
  kErrTrace = 1u << 0,     // an integral-line trace exceeded its step bound
  kErrRounds = 1u << 1,    // a union-find / reduction round loop exceeded its bound
  kErrPool = 1u << 2,      // the D1 column pool is exhausted (host retries larger)
  kErrInconsistent = 1u << 3,  // local pairing contradiction (must never happen)
  kErrEmptyColumn = 1u << 4,   // a saddle-saddle column reduced to zero
  kErrSpin = 1u << 5,      // a bounded spin-wait gave up
  kErrCapacity = 1u << 6,  // an output list is larger than its buffer
};

static __constant__ Geo c_geo = make_geo();
static __constant__ UpSteps c_up = make_up_steps();

// ---------------------------------------------------------------------------
// Per-vertex gradient record (32 bytes), bit layout:
//   [0,4)     vnext: neighbour index of the vertex's paired edge, 15 = minimum
//   [4,18)    critical lower-star edges v*a, by neighbour index a
//   [18,54)   critical lower-star triangles v*(a,b), by link edge index
//   [54]      the lower star holds a critical tetrahedron (a maximum)
//   [56,224)  24 x 7-bit codes, one per link triangle tau (tetrahedron v*tau):
//               0..23    tau is non-critical; the integral line continues in
//                        the same lower star, at link triangle `code`
//               24..95   it continues at link triangle (code-24)/3 of v's link,
//                        whose vertex number (code-24)%3 is higher than v: the
//                        next tetrahedron belongs to that vertex's lower star
//               124      it continues to the outside of the domain
//               125      tau is critical (a maximum)
//               127      tau is not in the lower star of v
// ---------------------------------------------------------------------------
struct __align__(16) Rec {
  uint32_t w[8];
};

enum : int { kCodeOut = 124, kCodeMax = 125, kCodeNone = 127, kVnextMin = 15 };

__host__ __device__ inline uint32_t rec_bits(const Rec& r, int off, int n) {
  int wi = off >> 5, bi = off & 31;
  uint64_t lo = r.w[wi];
  uint64_t hi = (wi + 1 < 8) ? r.w[wi + 1] : 0;
  uint64_t both = lo | (hi << 32);
  return (uint32_t)((both >> bi) & ((1ull << n) - 1));
}
__host__ __device__ inline void rec_set(Rec& r, int off, int n, uint32_t val) {
  for (int i = 0; i < n; ++i) {
    int b = off + i;
    uint32_t bit = (val >> i) & 1u;
    r.w[b >> 5] = (r.w[b >> 5] & ~(1u << (b & 31))) | (bit << (b & 31));
  }
}
__host__ __device__ inline int rec_vnext(const Rec& r) { return (int)(r.w[0] & 15u); }
__host__ __device__ inline uint32_t rec_crit_edges(const Rec& r) { return (r.w[0] >> 4) & 0x3FFFu; }
__host__ __device__ inline uint64_t rec_crit_tris(const Rec& r) {
  uint64_t lo = r.w[0] >> 18;                 // 14 bits
  uint64_t hi = (uint64_t)(r.w[1] & 0x3FFFFFu);  // 22 bits
  return lo | (hi << 14);
}
__host__ __device__ inline bool rec_has_max(const Rec& r) { return (r.w[1] >> 22) & 1u; }
__host__ __device__ inline int rec_tet_code(const Rec& r, int tau) { return (int)rec_bits(r, 56 + 7 * tau, 7); }

// Per-vertex expansion table for the saddle-saddle reduction (144 bytes).
// Eliminating the gradient-paired edges of one lower star is linear over
// Z/2, so the table holds the effect of each lower-star edge v*x eliminated
// alone, its *closure*: v*x paired with triangle v*(x, ..) is replaced by
// v*y + (link path x..y), v*y in turn by its own closure, until the chain
// reaches a critical edge (kept) or the lowest edge v*x0 (negative: not a
// row of the reduction).  Layout:
//   q[0..7]   bits 36x .. 36x+35: link edges (36-bit mask over v's link
//             edges) that the closure of v*x leaves in lower stars below v
//   q[8]      bits 4x .. 4x+3: the critical edge v*c the closure of v*x ends
//             at (c = x when v*x itself is critical), 15 = none
//   q[9]      bits 0..35: orientation of the link edges (a, b), a < b as
//             neighbour indices: 1 when a ranks above b (edge a*b then lies
//             in the lower star of v + off[a])
//   nkey[i]   value_key of neighbour i (0 outside the grid): with the vertex
//             id it orders lower stars exactly as their ranks do
struct __align__(16) D1Tab {
  unsigned long long q[10];
  uint32_t nkey[14];
  uint32_t pad[2];
};
static_assert(sizeof(D1Tab) == 144, "nine 16-byte loads per row");

template <int X>
__host__ __device__ __forceinline__ uint64_t tab_closure(const D1Tab& t) {
  constexpr int off = 36 * X, wi = off >> 6, bi = off & 63;
  uint64_t lo = t.q[wi] >> bi;
  if constexpr (bi > 28) lo |= t.q[wi + 1] << (64 - bi);
  return lo & ((1ull << 36) - 1);
}
__host__ __device__ inline void tab_set_closure(D1Tab& t, int x, uint64_t path) {
  int off = 36 * x, wi = off >> 6, bi = off & 63;
  t.q[wi] |= path << bi;
  if (bi > 28) t.q[wi + 1] |= path >> (64 - bi);
}
__host__ __device__ __forceinline__ int tab_end(const D1Tab& t, int x) { return (int)((t.q[8] >> (4 * x)) & 15ull); }

// Grid helpers -------------------------------------------------------------
struct Dims {
  int lx, ly, lz;
  int64_t nv;
};

__device__ __forceinline__ void vxyz(const Dims& d, uint32_t v, int& x, int& y, int& z) {
  x = (int)(v % (uint32_t)d.lx);
  uint32_t t = v / (uint32_t)d.lx;
  y = (int)(t % (uint32_t)d.ly);
  z = (int)(t / (uint32_t)d.ly);
}
__device__ __forceinline__ bool nbr_xyz(const Dims& d, int x, int y, int z, int i, int& nx, int& ny, int& nz) {
  nx = x + c_geo.off[i][0];
  ny = y + c_geo.off[i][1];
  nz = z + c_geo.off[i][2];
  return nx >= 0 && ny >= 0 && nz >= 0 && nx < d.lx && ny < d.ly && nz < d.lz;
}
__device__ __forceinline__ uint32_t vid(const Dims& d, int x, int y, int z) {
  return (uint32_t)x + (uint32_t)d.lx * ((uint32_t)y + (uint32_t)d.ly * (uint32_t)z);
}
__device__ __forceinline__ int nbr_index(int dx, int dy, int dz) {
  return c_geo.nbr_of[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)];
}
__device__ __forceinline__ int nbr_index(const Geo& G, int dx, int dy, int dz) {
  return G.nbr_of[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)];
}

// The geometry tables are read with lane-dependent indices in the lower-star
// kernels; constant memory serialises such reads, shared memory does not.
// Every thread of the block must call this (it ends with a barrier).
__device__ inline void geo_to_shared(Geo& sg) {
  const unsigned char* src = reinterpret_cast<const unsigned char*>(&c_geo);
  unsigned char* dst = reinterpret_cast<unsigned char*>(&sg);
  for (int i = threadIdx.x; i < (int)sizeof(Geo); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// Monotone float -> uint32 key for the vertex order (Section 2.1: ties are
// broken by vertex id; -0.0 and +0.0 are the same value).
__device__ __forceinline__ uint32_t value_key(float f) {
  uint32_t u = __float_as_uint(f);
  if (u == 0x80000000u) u = 0u;
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Canonical cell id: (dim << 60) | (base << 6) | type, base = the lowest
// corner of the chain, type = axis mask (edges) or 8*A + B (triangles,
// tetrahedra).  `xs` are vertex coordinates, any order.
__device__ inline uint64_t cell_id_of(const Dims& d, int n, int (*xs)[3]) {
  // chain order = increasing coordinate sum (the simplex is a chain)
  int idx[4] = {0, 1, 2, 3};
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0; --j) {
      int a = idx[j], b = idx[j - 1];
      if (xs[a][0] + xs[a][1] + xs[a][2] < xs[b][0] + xs[b][1] + xs[b][2]) {
        idx[j] = b;
        idx[j - 1] = a;
      }
    }
  auto mask = [&](int p, int q) {
    return (xs[q][0] - xs[p][0]) | ((xs[q][1] - xs[p][1]) << 1) | ((xs[q][2] - xs[p][2]) << 2);
  };
  int base_i = idx[0];
  uint64_t base = vid(d, xs[base_i][0], xs[base_i][1], xs[base_i][2]);
  int type = 0;
  if (n == 2) type = mask(idx[0], idx[1]);
  if (n >= 3) type = mask(idx[0], idx[1]) * 8 + mask(idx[1], idx[2]);
  return ((uint64_t)(n - 1) << 60) | (base << 6) | (uint64_t)type;
}

}  // namespace tsf
