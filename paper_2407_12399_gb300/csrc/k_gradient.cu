// k_gradient.cu -- lower-star discrete gradient (Section 4.2) and compaction
// of the critical cells in lexicographic order.
#include <algorithm>

#include "tsf_kernels.cuh"
#include "tsf_star.cuh"

namespace tsf {

// ---------------------------------------------------------------------------
// The lower star of v (Section 4.2) in registers and a per-thread slice of
// shared memory.  Lane-dependent array indices would otherwise put the star
// in local memory, whose traffic outgrows L1 at full occupancy and spills
// to DRAM.  Small tables are packed into 64-bit words:
//   P  nibble i = rank position of neighbour i among the lower ones (15: not lower)
//   B  nibble p = the neighbour at rank position p
//   L  nibble p = the root (smallest rank position) of p's lower-link component
//   D0, D1  5-bit fields: the root of each link triangle in the dual sweep
//           (triangles 0..11 in D0, 12..23 in D1; 24 = outside the lower star)
// Shared memory keeps, with the thread index innermost (a warp's accesses hit
// 32 different banks), the link adjacency by neighbour, the dual record
// codes, and per rank position the link edges of the forest path to its
// root.
// ---------------------------------------------------------------------------
constexpr int kGT = 128;  // threads per block of the gradient kernels

// The link tables the sweeps index with lane-dependent values, packed:
//   edge_desc[e]  the two link triangles t_k on link edge e, each with the slot
//                 j_k of its third vertex and that vertex c_k:
//                 t0 | c0 << 5 | j0 << 9 | t1 << 11 | c1 << 16 | j1 << 20
//   tri3[t]       the vertices of link triangle t: a | b << 4 | c << 8
//   edge_idx      link edge of a neighbour pair (as in the full table)
struct GradGeo {
  uint32_t edge_desc[36];
  uint32_t tri3[24];
  int8_t edge_idx[14][14];
  int8_t pad[4];
};
static_assert(sizeof(GradGeo) % 4 == 0, "copied as words");

constexpr GradGeo make_grad_geo() {
  GradGeo g{};
  for (int e = 0; e < 36; ++e) {
    uint32_t w = 0;
    for (int k = 0; k < 2; ++k) {
      const uint32_t t = (uint32_t)kGeo.edge_tri[e][k], j = (uint32_t)kGeo.edge_third[e][k];
      const uint32_t c = (uint32_t)kGeo.tri[t][j];
      w |= (t | (c << 5) | (j << 9)) << (11 * k);
    }
    g.edge_desc[e] = w;
  }
  for (int t = 0; t < 24; ++t)
    g.tri3[t] = (uint32_t)kGeo.tri[t][0] | ((uint32_t)kGeo.tri[t][1] << 4) | ((uint32_t)kGeo.tri[t][2] << 8);
  for (int a = 0; a < 14; ++a)
    for (int b = 0; b < 14; ++b) g.edge_idx[a][b] = kGeo.edge_idx[a][b];
  return g;
}
constexpr bool grad_geo_matches() {
  const GradGeo g = make_grad_geo();
  for (int e = 0; e < 36; ++e)
    for (int k = 0; k < 2; ++k) {
      const uint32_t dk = g.edge_desc[e] >> (11 * k);
      const int t = (int)(dk & 31u), c = (int)((dk >> 5) & 15u), j = (int)((dk >> 9) & 3u);
      if (t != kGeo.edge_tri[e][k] || j != kGeo.edge_third[e][k] || c != kGeo.tri[t][j]) return false;
    }
  for (int t = 0; t < 24; ++t)
    for (int i = 0; i < 3; ++i)
      if ((int)((g.tri3[t] >> (4 * i)) & 15u) != kGeo.tri[t][i]) return false;
  return true;
}
static_assert(grad_geo_matches(), "packed link tables decode to the full ones");
static __constant__ GradGeo c_grad_geo = make_grad_geo();

// Every thread of the block must call this (it ends with a barrier).
__device__ __forceinline__ void grad_geo_to_shared(GradGeo& sg) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&c_grad_geo);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&sg);
  for (int i = threadIdx.x; i < (int)(sizeof(GradGeo) / 4); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

struct GradSmem {
  unsigned long long rp[14][kGT];  // forest path (link-edge mask) to the tree root, by rank position
  uint32_t adj[7][kGT];            // rank-position adjacency of neighbour 2k (low half) and 2k+1 (high half)
  uint32_t code[6][kGT];           // record code of link triangle t in byte t & 3 of word t >> 2
};

__device__ __forceinline__ int nib(uint64_t w, int i) { return (int)((w >> (4 * i)) & 15u); }

// bit 4i set where nibble i of w equals v
__device__ __forceinline__ uint64_t nib_eq(uint64_t w, int v) {
  uint64_t x = w ^ (0x1111111111111111ull * (uint64_t)v);
  x |= x >> 1;
  x |= x >> 2;
  return ~x & 0x1111111111111111ull;
}

constexpr uint64_t kF5 = 0x0084210842108421ull;  // bit 5i for i < 12
__host__ __device__ constexpr uint64_t f5_iota(int base) {
  uint64_t w = 0;
  for (int i = 0; i < 12; ++i) w |= (uint64_t)(base + i) << (5 * i);
  return w;
}
static_assert(kF5 == [] {
  uint64_t m = 0;
  for (int i = 0; i < 12; ++i) m |= 1ull << (5 * i);
  return m;
}(), "field mask");

// bit 5i set where 5-bit field i of w equals v
__device__ __forceinline__ uint64_t f5_eq(uint64_t w, int v) {
  uint64_t x = w ^ (kF5 * (uint64_t)v);
  x |= (x >> 1) | (x >> 2) | (x >> 3) | (x >> 4);
  return ~x & kF5;
}
__device__ __forceinline__ int dual_root(uint64_t D0, uint64_t D1, int t) {
  if (t >= 24) return 24;
  return t < 12 ? (int)((D0 >> (5 * t)) & 31u) : (int)((D1 >> (5 * (t - 12))) & 31u);
}

template <int I>
__device__ __forceinline__ uint32_t adj_positions(uint32_t lower, uint64_t P) {
  uint32_t r = 0;
#pragma unroll
  for (int j = 0; j < 14; ++j)
    if ((geo_adj(I) >> j) & 1u)
      if ((lower >> j) & 1u) r |= 1u << nib(P, j);
  return r;
}
template <int... K>
__device__ __forceinline__ void store_adj(GradSmem& sm, uint32_t lower, uint64_t P, std::integer_sequence<int, K...>) {
  ((sm.adj[K][threadIdx.x] = adj_positions<2 * K>(lower, P) | (adj_positions<2 * K + 1>(lower, P) << 16)), ...);
}
__device__ __forceinline__ uint32_t adj_of(const GradSmem& sm, int a) {
  return (sm.adj[a >> 1][threadIdx.x] >> (16 * (a & 1))) & 0xFFFFu;
}

// Initial record code of link triangle T: a maximum while v*T lies in the
// lower star, else "not in the lower star".
template <int T>
__device__ __forceinline__ uint32_t initial_code(uint32_t lower) {
  constexpr uint32_t m = (1u << kGeo.tri[T][0]) | (1u << kGeo.tri[T][1]) | (1u << kGeo.tri[T][2]);
  return (lower & m) == m ? (uint32_t)kCodeMax : (uint32_t)kCodeNone;
}
template <int... K>
__device__ __forceinline__ void store_codes(GradSmem& sm, uint32_t lower, std::integer_sequence<int, K...>) {
  ((sm.code[K][threadIdx.x] = initial_code<4 * K>(lower) | (initial_code<4 * K + 1>(lower) << 8) |
                              (initial_code<4 * K + 2>(lower) << 16) | (initial_code<4 * K + 3>(lower) << 24)),
   ...);
}

// Neighbour pairs (i, j), i < j, numbered 0..90 for fully unrolled pair loops.
__host__ __device__ constexpr int pair_i(int k) {
  int i = 0;
  while (k >= 13 - i) k -= 13 - i++;
  return i;
}
__host__ __device__ constexpr int pair_j(int k) {
  int i = 0;
  while (k >= 13 - i) k -= 13 - i++;
  return i + 1 + k;
}
// One comparison per pair: the neighbour ranked below the other adds one to
// the other's count; for a link edge (i, j) the result is also kept.
template <int K>
__device__ __forceinline__ void rank_pair(const uint32_t* nr, int* cnt, unsigned long long& below36) {
  constexpr int i = pair_i(K), j = pair_j(K), le = kGeo.edge_idx[i][j];
  const bool jb = nr[j] < nr[i];
  cnt[i] += jb ? 1 : 0;
  cnt[j] += jb ? 0 : 1;
  if constexpr (le >= 0) below36 |= (unsigned long long)jb << le;
}
template <int... K>
__device__ __forceinline__ void rank_pairs(const uint32_t* nr, int* cnt, unsigned long long& below36,
                                           std::integer_sequence<int, K...>) {
  (rank_pair<K>(nr, cnt, below36), ...);
}
static_assert(pair_i(90) == 12 && pair_j(90) == 13 && pair_i(12) == 0 && pair_j(12) == 13 && pair_j(13) == 2,
              "pair numbering");

// Link edges (a, b), a < b, whose first vertex a is lower.
__host__ __device__ constexpr unsigned long long edges_from(int a) {
  unsigned long long m = 0;
  for (int le = 0; le < 36; ++le)
    if (kGeo.edge[le][0] == a) m |= 1ull << le;
  return m;
}
template <int... A>
__device__ __forceinline__ unsigned long long edges_from_lower(uint32_t lower, std::integer_sequence<int, A...>) {
  return (((lower >> A) & 1u ? edges_from(A) : 0ull) | ...);
}

// Key of link triangle t in the backward sweep (larger = later in the filtration).
__device__ __forceinline__ int tri_key(uint64_t P, int t, const GradGeo& G) {
  const uint32_t w = G.tri3[t];
  int p0 = nib(P, w & 15u), p1 = nib(P, (w >> 4) & 15u), p2 = nib(P, (w >> 8) & 15u);
  int hi = max(p0, max(p1, p2)), lo = min(p0, min(p1, p2));
  return hi * 196 + (p0 + p1 + p2 - hi - lo) * 14 + lo;
}

// The lower star of v: its gradient record, the byte naming the edge v is
// paired with, and (tab non-null) the saddle-saddle table row.
//
// Forward sweep (0-dimensional persistence of the lower link, elder rule):
// link vertices by rank position, each one's link edges to earlier ones by
// increasing position; an edge joining two components kills the younger root.
// Backward sweep: link edges in the reverse order over the dual graph (link
// triangles of the lower link, plus one node for everything outside); an
// edge joining two dual components kills the one whose root triangle comes
// first in the filtration.  The same sweeps as the plain formulation in
// tsf_star.cuh (which the zero-pair test kernel and the single-thread D1
// heap kernel use), with union-find replaced by always-compressed root labels.
//
// Closures: the chain of the table's closure of v*x (v*x -> v*y + path x..y
// -> ...) runs through the older representatives x's component merged into,
// and ends at the root of x's tree in the final link forest: the lowest edge
// v*x0 (root position 0) or a critical edge.  Its link-edge sum telescopes
// into the forest path from x to that root, which is kept per position while
// the forest grows: when the component of root `young` joins `old` through
// link edge e = (a, b), every member u of the young component extends its
// path by path(a) + e + path(b).
__device__ __forceinline__ void gradient_star(const Dims& d, const uint32_t* __restrict__ rank,
                                              const float* __restrict__ values, int64_t v, Rec* __restrict__ rec,
                                              uint8_t* __restrict__ vnext8, D1Tab* __restrict__ tab,
                                              uint32_t* status, const GradGeo& sg, GradSmem& sm) {
  const int tid = threadIdx.x;
  int vx, vy, vz;
  vxyz(d, (uint32_t)v, vx, vy, vz);
  const uint32_t rv = __ldg(rank + v);
  uint32_t nr[14];
  uint32_t valid = 0, lower = 0;
#pragma unroll
  for (int i = 0; i < 14; ++i) {
    int nx, ny, nz;
    nr[i] = 0xFFFFFFFFu;
    if (nbr_xyz(d, vx, vy, vz, i, nx, ny, nz)) {
      valid |= 1u << i;
      nr[i] = __ldg(rank + vid(d, nx, ny, nz));
      if (nr[i] < rv) lower |= 1u << i;
    }
  }
  const int nl = __popc(lower);
  // rank positions: a lower neighbour's position counts the neighbours ranked
  // below it (all of them lower, as v is above them; outside ranks stay above)
  int cnt[14];
#pragma unroll
  for (int i = 0; i < 14; ++i) cnt[i] = 0;
  unsigned long long below36 = 0;  // link edge (a, b), a < b: b ranks below a
  rank_pairs(nr, cnt, below36, std::make_integer_sequence<int, 91>{});
  uint64_t P = 0, B = 0;
#pragma unroll
  for (int i = 0; i < 14; ++i) {
    if ((lower >> i) & 1u) {
      P |= (uint64_t)cnt[i] << (4 * i);
      B |= (uint64_t)i << (4 * cnt[i]);
    } else {
      P |= 15ull << (4 * i);
    }
  }
  store_adj(sm, lower, P, std::make_integer_sequence<int, 7>{});
  if (tab) {
#pragma unroll
    for (int k = 0; k < 14; ++k) sm.rp[k][tid] = 0;
  }

  // forward sweep
  constexpr uint64_t kIota4 = 0xFEDCBA9876543210ull;
  uint64_t L = kIota4;
  uint64_t link_pos = 0;
  for (int p = 1; p < nl; ++p) {
    const int a = nib(B, p);
    for (uint32_t qm = adj_of(sm, a) & ((1u << p) - 1u); qm; qm &= qm - 1) {
      const int q = __ffs(qm) - 1;
      const int e = sg.edge_idx[a][nib(B, q)];
      const int ra = nib(L, p), rb = nib(L, q);
      if (ra == rb) {
        link_pos |= 1ull << e;
        continue;
      }
      const int young = max(ra, rb), old = min(ra, rb);
      uint64_t fl = nib_eq(L, young);
      L ^= fl * (uint64_t)(young ^ old);
      if (tab) {
        const unsigned long long c = sm.rp[p][tid] ^ sm.rp[q][tid] ^ (1ull << e);
        for (; fl; fl &= fl - 1) sm.rp[(__ffsll((long long)fl) - 1) >> 2][tid] ^= c;
      }
    }
  }
  uint32_t crit_edges = 0;
  {
    const uint64_t span = nl > 1 ? (((1ull << (4 * nl)) - 1ull) & ~15ull) : 0ull;
    for (uint64_t rm = nib_eq(L ^ kIota4, 0) & span; rm; rm &= rm - 1)
      crit_edges |= 1u << nib(B, (__ffsll((long long)rm) - 1) >> 2);
  }

  // backward (dual) sweep
  store_codes(sm, lower, std::make_integer_sequence<int, 6>{});
  constexpr uint64_t kIota5a = f5_iota(0), kIota5b = f5_iota(12);
  uint64_t D0 = kIota5a, D1 = kIota5b;
  uint64_t crit_tris = 0;
  bool inconsistent = false;
  uint8_t* code8 = reinterpret_cast<uint8_t*>(&sm.code[0][0]);
  for (int p = nl - 1; p >= 1; --p) {
    const int a = nib(B, p);
    for (uint32_t qm = adj_of(sm, a) & ((1u << p) - 1u); qm;) {
      const int q = 31 - __clz(qm);
      qm ^= 1u << q;
      const int e = sg.edge_idx[a][nib(B, q)];
      const uint32_t desc = sg.edge_desc[e];
      int node[2], tcode[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const uint32_t dk = desc >> (11 * k);
        const int t = (int)(dk & 31u), c = (int)((dk >> 5) & 15u), j = (int)((dk >> 9) & 3u);
        if (!((valid >> c) & 1u)) {
          node[k] = 24;
          tcode[k] = kCodeOut;
        } else if ((lower >> c) & 1u) {
          node[k] = t;
          tcode[k] = t;
        } else {
          node[k] = 24;
          tcode[k] = 24 + 3 * t + j;
        }
      }
      const int r0 = dual_root(D0, D1, node[0]), r1 = dual_root(D0, D1, node[1]);
      const bool lp = (link_pos >> e) & 1ull;
      if (r0 == r1) {
        if (lp) crit_tris |= 1ull << e;
        continue;
      }
      const int k0 = r0 == 24 ? 0x7FFFFFFF : tri_key(P, r0, sg);
      const int k1 = r1 == 24 ? 0x7FFFFFFF : tri_key(P, r1, sg);
      const int dside = k0 < k1 ? 0 : 1;
      const int rd = dside == 0 ? r0 : r1, ro = dside == 0 ? r1 : r0;
      code8[((rd >> 2) * kGT + tid) * 4 + (rd & 3)] = (uint8_t)tcode[1 - dside];
      const uint64_t x = (uint64_t)(rd ^ ro);
      D0 ^= f5_eq(D0, rd) * x;
      D1 ^= f5_eq(D1, rd) * x;
      if (!lp) inconsistent = true;
    }
  }
  if (inconsistent) atomicOr(status, kErrInconsistent);

  // the record
  Rec r;
  r.w[0] = (nl > 0 ? (uint32_t)nib(B, 0) : (uint32_t)kVnextMin) | (crit_edges << 4) |
           ((uint32_t)(crit_tris & 0x3FFFull) << 18);
  r.w[1] = (uint32_t)((crit_tris >> 14) & 0x3FFFFFull);
#pragma unroll
  for (int i = 2; i < 8; ++i) r.w[i] = 0;
  bool has_max = false;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const uint32_t w = sm.code[k][tid];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int t = 4 * k + b;
      const uint32_t c = (w >> (8 * b)) & 0x7Fu;
      has_max |= c == (uint32_t)kCodeMax;
      const int off = 56 + 7 * t, wi = off >> 5, bi = off & 31;
      r.w[wi] |= c << bi;
      if (bi > 25) r.w[wi + 1] |= c >> (32 - bi);
    }
  }
  r.w[1] |= (has_max ? 1u : 0u) << 22;
  uint4* dst = reinterpret_cast<uint4*>(rec + v);
  dst[0] = make_uint4(r.w[0], r.w[1], r.w[2], r.w[3]);
  dst[1] = make_uint4(r.w[4], r.w[5], r.w[6], r.w[7]);
  vnext8[v] = (uint8_t)(r.w[0] & 15u);

  if (tab) {
    unsigned long long q[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = 0;
    unsigned long long ends = ~0ull;
#pragma unroll
    for (int x = 0; x < 14; ++x) {
      if ((lower >> x) & 1u) {
        const int p = nib(P, x);
        const unsigned long long c = sm.rp[p][tid];
        const int root = nib(L, p);
        const int e = root == 0 ? 15 : nib(B, root);
        const int off = 36 * x, wi = off >> 6, bi = off & 63;
        q[wi] |= c << bi;
        if (bi > 28) q[wi + 1] |= c >> (64 - bi);
        ends = (ends & ~(15ull << (4 * x))) | ((unsigned long long)e << (4 * x));
      }
    }
    // (a, b) is oriented when a is lower and b ranks below it (then b is lower too)
    const unsigned long long orient = below36 & edges_from_lower(lower, std::make_integer_sequence<int, 14>{});
    uint4* dst4 = reinterpret_cast<uint4*>(tab + v);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      dst4[k] = make_uint4((uint32_t)q[2 * k], (uint32_t)(q[2 * k] >> 32), (uint32_t)q[2 * k + 1],
                           (uint32_t)(q[2 * k + 1] >> 32));
    dst4[4] = make_uint4((uint32_t)ends, (uint32_t)(ends >> 32), (uint32_t)orient, (uint32_t)(orient >> 32));
    uint32_t nk[16];
    const int64_t sy = d.lx, sz = (int64_t)d.lx * d.ly;
#pragma unroll
    for (int i = 0; i < 14; ++i)
      nk[i] = ((valid >> i) & 1u)
                  ? value_key(__ldg(values + v + c_geo.off[i][0] + sy * c_geo.off[i][1] + sz * c_geo.off[i][2]))
                  : 0u;
    nk[14] = nk[15] = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) dst4[5 + k] = make_uint4(nk[4 * k], nk[4 * k + 1], nk[4 * k + 2], nk[4 * k + 3]);
  }
}

// Every lower star (the first diagram of a field, or without the fast update).
template <int MINB>
__global__ void __launch_bounds__(kGT, MINB) k_gradient(Dims d, const uint32_t* __restrict__ rank, const float* __restrict__ values,
                           Rec* __restrict__ rec, uint8_t* __restrict__ vnext8, D1Tab* __restrict__ tab,
                           uint32_t* status) {
  __shared__ GradGeo sg;
  __shared__ GradSmem sm;
  grad_geo_to_shared(sg);
  int64_t v = (int64_t)blockIdx.x * kGT + threadIdx.x;
  if (v < d.nv) gradient_star(d, rank, values, v, rec, vnext8, tab, status, sg, sm);
}

// Section 4.2, fast persistence update: only the lower stars whose closed
// star holds a vertex the last gradient step updated can change (the vertex
// itself and its 14 neighbours); the others keep their records, which stay
// exact.  Each such star is listed once (a generation mark, so the marks are
// never cleared), then recomputed by one thread of a dense launch.
__global__ void k_gradient_expand(Dims d, const uint32_t* __restrict__ upd, int64_t nu, uint32_t* __restrict__ mark,
                                  uint32_t gen, uint32_t* __restrict__ list, unsigned long long* count) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nu * 15) return;
  uint32_t u = upd[t / 15];
  int i = (int)(t % 15);
  uint32_t w = u;
  if (i < 14) {
    int x, y, z, nx, ny, nz;
    vxyz(d, u, x, y, z);
    if (!nbr_xyz(d, x, y, z, i, nx, ny, nz)) return;
    w = vid(d, nx, ny, nz);
  }
  if (atomicExch(mark + w, gen) != gen) list[atomicAdd(count, 1ull)] = w;
}

template <int MINB>
__global__ void __launch_bounds__(kGT, MINB) k_gradient_list(Dims d, const uint32_t* __restrict__ rank, const float* __restrict__ values,
                                const uint32_t* __restrict__ list, const unsigned long long* __restrict__ count,
                                Rec* __restrict__ rec, uint8_t* __restrict__ vnext8, D1Tab* __restrict__ tab,
                                uint32_t* status) {
  __shared__ GradGeo sg;
  __shared__ GradSmem sm;
  grad_geo_to_shared(sg);
  int64_t i = (int64_t)blockIdx.x * kGT + threadIdx.x;
  if (i < (int64_t)*count) gradient_star(d, rank, values, list[i], rec, vnext8, tab, status, sg, sm);
}


// ---------------------------------------------------------------------------
// Compaction of critical cells, in increasing rank of their highest vertex
// (then the lexicographic order inside one lower star), which is the
// lexicographic order of Section 2.2 restricted to critical cells.
// ---------------------------------------------------------------------------
constexpr int kCT = 256;  // threads per block
constexpr int kCI = 8;    // rounds per block
constexpr int kCTile = kCT * kCI;

struct Cnt4 {
  int a, b, c, d;
};

__device__ __forceinline__ Cnt4 rec_counts(const Rec& r) {
  Cnt4 c;
  c.a = rec_vnext(r) == kVnextMin;
  c.b = __popc(rec_crit_edges(r));
  c.c = __popcll(rec_crit_tris(r));
  c.d = rec_has_max(r) ? 1 : 0;
  return c;
}

__device__ __forceinline__ Rec load_rec(const Rec* rec, uint32_t v) {
  const uint4* p = reinterpret_cast<const uint4*>(rec + v);
  uint4 a = __ldg(p), b = __ldg(p + 1);
  Rec r;
  r.w[0] = a.x; r.w[1] = a.y; r.w[2] = a.z; r.w[3] = a.w;
  r.w[4] = b.x; r.w[5] = b.y; r.w[6] = b.z; r.w[7] = b.w;
  return r;
}

// block-wide exclusive scan of 4 counters (warp shuffles + shared memory)
__device__ __forceinline__ Cnt4 block_scan4(Cnt4 v, Cnt4& total) {
  __shared__ int sw[kCT / 32][4];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Cnt4 inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int a = __shfl_up_sync(0xFFFFFFFFu, inc.a, o), b = __shfl_up_sync(0xFFFFFFFFu, inc.b, o);
    int c = __shfl_up_sync(0xFFFFFFFFu, inc.c, o), d = __shfl_up_sync(0xFFFFFFFFu, inc.d, o);
    if (lane >= o) {
      inc.a += a; inc.b += b; inc.c += c; inc.d += d;
    }
  }
  if (lane == 31) {
    sw[wid][0] = inc.a; sw[wid][1] = inc.b; sw[wid][2] = inc.c; sw[wid][3] = inc.d;
  }
  __syncthreads();
  Cnt4 base = {0, 0, 0, 0};
  total = {0, 0, 0, 0};
  for (int w = 0; w < kCT / 32; ++w) {
    if (w < wid) {
      base.a += sw[w][0]; base.b += sw[w][1]; base.c += sw[w][2]; base.d += sw[w][3];
    }
    total.a += sw[w][0]; total.b += sw[w][1]; total.c += sw[w][2]; total.d += sw[w][3];
  }
  __syncthreads();
  Cnt4 ex = {base.a + inc.a - v.a, base.b + inc.b - v.b, base.c + inc.c - v.c, base.d + inc.d - v.d};
  return ex;
}

__global__ void k_crit_count(int64_t nv, const uint32_t* __restrict__ order, const Rec* __restrict__ rec,
                             int4* __restrict__ tile_counts) {
  Cnt4 acc = {0, 0, 0, 0};
  int64_t base = (int64_t)blockIdx.x * kCTile;
  for (int i = 0; i < kCI; ++i) {
    int64_t r = base + (int64_t)i * kCT + threadIdx.x;
    if (r < nv) {
      Cnt4 c = rec_counts(load_rec(rec, __ldg(order + r)));
      acc.a += c.a; acc.b += c.b; acc.c += c.c; acc.d += c.d;
    }
  }
  Cnt4 tot;
  block_scan4(acc, tot);
  if (threadIdx.x == 0) tile_counts[blockIdx.x] = make_int4(tot.a, tot.b, tot.c, tot.d);
}

// exclusive scan of the tile counters, single block; also writes the totals
__global__ void k_crit_scan(int ntiles, int4* __restrict__ tile_counts, int4* __restrict__ totals) {
  __shared__ int4 carry;
  if (threadIdx.x == 0) carry = make_int4(0, 0, 0, 0);
  __syncthreads();
  for (int b = 0; b < ntiles; b += kCT) {
    int i = b + threadIdx.x;
    Cnt4 v = {0, 0, 0, 0};
    if (i < ntiles) {
      int4 t = tile_counts[i];
      v = {t.x, t.y, t.z, t.w};
    }
    Cnt4 tot;
    Cnt4 ex = block_scan4(v, tot);
    int4 c = carry;
    if (i < ntiles) tile_counts[i] = make_int4(c.x + ex.a, c.y + ex.b, c.z + ex.c, c.w + ex.d);
    __syncthreads();
    if (threadIdx.x == 0) carry = make_int4(c.x + tot.a, c.y + tot.b, c.z + tot.c, c.w + tot.d);
    __syncthreads();
  }
  if (threadIdx.x == 0) *totals = carry;
}

__global__ void k_crit_write(Dims d, const uint32_t* __restrict__ order, const uint32_t* __restrict__ rank,
                             const Rec* __restrict__ rec, const int4* __restrict__ tile_off, CritLists L,
                             uint32_t* __restrict__ cidx, uint32_t* __restrict__ c1base,
                             uint32_t* __restrict__ c2base, uint32_t* status) {
  const Geo& sg = c_geo;
  int4 t = tile_off[blockIdx.x];
  Cnt4 run = {t.x, t.y, t.z, t.w};
  int64_t base = (int64_t)blockIdx.x * kCTile;
  for (int i = 0; i < kCI; ++i) {
    int64_t r = base + (int64_t)i * kCT + threadIdx.x;
    Cnt4 c = {0, 0, 0, 0};
    uint32_t v = 0;
    Rec rc;
    if (r < d.nv) {
      v = __ldg(order + r);
      rc = load_rec(rec, v);
      c = rec_counts(rc);
    }
    Cnt4 tot;
    Cnt4 ex = block_scan4(c, tot);
    if (r < d.nv && (c.a | c.b | c.c | c.d)) {
      int o0 = run.a + ex.a, o1 = run.b + ex.b, o2 = run.c + ex.c, o3 = run.d + ex.d;
      if (c.a) {
        if (o0 < L.cap0) L.c0[o0] = v;
        cidx[v] = (uint32_t)o0;
      }
      if (c.d) {
        int tau = 0;
        for (int k = 0; k < 24; ++k)
          if (rec_tet_code(rc, k) == kCodeMax) tau = k;
        if (o3 < L.cap3) L.c3[o3] = (v << 5) | (uint32_t)tau;
        cidx[v] = (uint32_t)o3;
      }
      if (c.b | c.c) {
        int x, y, z;
        vxyz(d, v, x, y, z);
        uint32_t nr[14];
#pragma unroll
        for (int k = 0; k < 14; ++k) {
          int nx, ny, nz;
          nr[k] = nbr_xyz(d, x, y, z, k, nx, ny, nz) ? __ldg(rank + vid(d, nx, ny, nz)) : 0xFFFFFFFFu;
        }
        uint32_t rv = __ldg(rank + v);
        if (c.b) {
          c1base[v] = (uint32_t)o1;
          uint32_t m = rec_crit_edges(rc);
          // emit by increasing rank of the lower endpoint
          for (int k = 0; k < c.b; ++k) {
            int best = -1;
            for (int j = 0; j < 14; ++j)
              if (((m >> j) & 1u) && (best < 0 || nr[j] < nr[best])) best = j;
            m &= ~(1u << best);
            int o = o1 + k;
            if (o < L.cap1) {
              L.c1_key[o] = ((uint64_t)rv << 32) | nr[best];
              L.c1_vn[o] = (v << 4) | (uint32_t)best;
            }
          }
        }
        if (c.c) {
          c2base[v] = (uint32_t)o2;
          uint64_t m = rec_crit_tris(rc);
          for (int k = 0; k < c.c; ++k) {
            int best = -1;
            uint64_t bk = 0;
            for (uint64_t mm = m; mm; mm &= mm - 1) {
              int e = __ffsll((long long)mm) - 1;
              uint32_t ra = nr[sg.edge[e][0]], rb = nr[sg.edge[e][1]];
              uint64_t kk = ((uint64_t)max(ra, rb) << 32) | min(ra, rb);
              if (best < 0 || kk < bk) {
                best = e;
                bk = kk;
              }
            }
            m &= ~(1ull << best);
            int o = o2 + k;
            if (o < L.cap2) L.c2_ve[o] = (v << 6) | (uint32_t)best;
          }
        }
      }
    }
    run.a += tot.a; run.b += tot.b; run.c += tot.c; run.d += tot.d;
  }
}

// Every zero-persistence pair of every lower star, as (birth cell, death
// cell).  Test support: lets the local pairing be checked cell by cell.
__global__ void k_zero_pairs(Dims d, const uint32_t* __restrict__ rank, unsigned long long* __restrict__ out,
                             int64_t cap, unsigned long long* __restrict__ count, uint32_t* status) {
  const Geo& sg = c_geo;
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.nv) return;
  Star s;
  star_load(s, d, (uint32_t)v, rank);
  Fwd f;
  star_forward(s, f, sg);
  Dual du;
  star_dual(s, f, du, sg);
  if (du.inconsistent) atomicOr(status, kErrInconsistent);
  int x, y, z;
  vxyz(d, (uint32_t)v, x, y, z);
  auto P = [&](int k, int* o) {
    o[0] = x + sg.off[k][0];
    o[1] = y + sg.off[k][1];
    o[2] = z + sg.off[k][2];
  };
  auto emit = [&](uint64_t a, uint64_t b) {
    unsigned long long i = atomicAdd(count, 1ull);
    if ((int64_t)i < cap) {
      out[2 * i] = a;
      out[2 * i + 1] = b;
    }
  };
  int xs[4][3];
  xs[0][0] = x; xs[0][1] = y; xs[0][2] = z;
  if (s.nl > 0) {
    P(s.by_pos[0], xs[1]);
    emit(cell_id_of(d, 1, xs), cell_id_of(d, 2, xs));
  }
  for (int a = 0; a < 14; ++a) {
    int e = f.killer[a];
    if (e < 0) continue;
    P(a, xs[1]);
    uint64_t cb = cell_id_of(d, 2, xs);
    P(sg.edge[e][0], xs[1]);
    P(sg.edge[e][1], xs[2]);
    emit(cb, cell_id_of(d, 3, xs));
  }
  for (int t = 0; t < 24; ++t) {
    int e = du.killer[t];
    if (e < 0) continue;
    P(sg.edge[e][0], xs[1]);
    P(sg.edge[e][1], xs[2]);
    uint64_t cb = cell_id_of(d, 3, xs);
    P(sg.tri[t][0], xs[1]);
    P(sg.tri[t][1], xs[2]);
    P(sg.tri[t][2], xs[3]);
    emit(cb, cell_id_of(d, 4, xs));
  }
}

}  // namespace tsf

namespace tsf {

// Blocks per SM of the gradient kernels' register budget (tuning knob 8).
static int gradient_blocks() { return (int)get_knob(8); }

void launch_gradient(const Dims& d, const uint32_t* rank, const float* f, Rec* rec, uint8_t* vnext8, D1Tab* tab,
                     uint32_t* status, cudaStream_t st) {
  unsigned nb = (unsigned)((d.nv + kGT - 1) / kGT);
  switch (gradient_blocks()) {
    case 1: k_gradient<1><<<nb, kGT, 0, st>>>(d, rank, f, rec, vnext8, tab, status); break;
    case 2: k_gradient<5><<<nb, kGT, 0, st>>>(d, rank, f, rec, vnext8, tab, status); break;
    default: k_gradient<6><<<nb, kGT, 0, st>>>(d, rank, f, rec, vnext8, tab, status); break;
  }
  note_launch();
}

void launch_gradient_incremental(const Dims& d, const uint32_t* rank, const float* f, const uint32_t* upd, int64_t nu,
                                 uint32_t* mark, uint32_t gen, uint32_t* list, unsigned long long* count, Rec* rec,
                                 uint8_t* vnext8, D1Tab* tab, uint32_t* status, cudaStream_t st) {
  cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
  if (nu <= 0) return;
  unsigned nb = (unsigned)((nu * 15 + 255) / 256);
  k_gradient_expand<<<nb, 256, 0, st>>>(d, upd, nu, mark, gen, list, count); note_launch();
  unsigned nl = (unsigned)((std::min<int64_t>(nu * 15, d.nv) + kGT - 1) / kGT);
  switch (gradient_blocks()) {
    case 1: k_gradient_list<1><<<nl, kGT, 0, st>>>(d, rank, f, list, count, rec, vnext8, tab, status); break;
    case 2: k_gradient_list<5><<<nl, kGT, 0, st>>>(d, rank, f, list, count, rec, vnext8, tab, status); break;
    default: k_gradient_list<6><<<nl, kGT, 0, st>>>(d, rank, f, list, count, rec, vnext8, tab, status); break;
  }
  note_launch();
}

int crit_tiles(int64_t nv) { return (int)((nv + kCTile - 1) / kCTile); }

void launch_crit_count(const Dims& d, const uint32_t* order, const Rec* rec, int4* tile_counts, int4* totals,
                       cudaStream_t st) {
  int nt = crit_tiles(d.nv);
  k_crit_count<<<nt, kCT, 0, st>>>(d.nv, order, rec, tile_counts); note_launch();
  k_crit_scan<<<1, kCT, 0, st>>>(nt, tile_counts, totals); note_launch();
}

void launch_crit_write(const Dims& d, const uint32_t* order, const uint32_t* rank, const Rec* rec,
                       const int4* tile_off, const CritLists& L, uint32_t* cidx, uint32_t* c1base, uint32_t* c2base,
                       uint32_t* status, cudaStream_t st) {
  k_crit_write<<<crit_tiles(d.nv), kCT, 0, st>>>(d, order, rank, rec, tile_off, L, cidx, c1base, c2base, status); note_launch();
}

void launch_zero_pairs(const Dims& d, const uint32_t* rank, unsigned long long* out, int64_t cap,
                       unsigned long long* count, uint32_t* status, cudaStream_t st) {
  k_zero_pairs<<<(unsigned)((d.nv + 127) / 128), 128, 0, st>>>(d, rank, out, cap, count, status); note_launch();
}

}  // namespace tsf
