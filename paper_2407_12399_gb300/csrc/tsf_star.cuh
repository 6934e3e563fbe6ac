// tsf_star.cuh -- the lower star of one vertex and its zero-persistence pairs.
//
// Paper Section 4.2: the discrete gradient is local to the lower star of each
// vertex (its cofaces whose other vertices all come earlier in the vertex
// order).  In the lexicographic filtration (Section 2.2) all simplices of the
// lower star of v come in one consecutive block, and the zero-persistence
// pairs (v_b = v_d = v) are exactly the pairs of the block's own reduction,
// i.e. the persistence of the *lower link* of v (augmented by v itself):
//   * v pairs with its lowest edge v*a (a = the lowest lower neighbour);
//   * an edge v*x pairs with the triangle v*(a,b) when the link edge (a,b)
//     merges two components of the lower link whose younger representative
//     is x (0-dimensional persistence of the lower link, elder rule);
//   * a triangle v*e pairs with the tetrahedron v*tau when, sweeping the
//     dual graph of the lower link backwards (link triangles as nodes, link
//     edges as arcs, everything outside the lower star as one oldest node),
//     the arc e kills the component represented by tau.
// Cells left unpaired are critical.  Note that v*x need not be a face of
// v*(a,b), nor v*e a face of v*tau: these pairs are not always facet pairs,
// so the integral lines below follow "the component a cell merges into",
// not the cell's partner.
#pragma once
#include <utility>
#include "tsf_internal.cuh"

namespace tsf {

struct Star {
  uint32_t rv;        // rank of v
  uint32_t nr[14];    // ranks of the neighbours (undefined where invalid)
  uint32_t valid;     // in-grid neighbours
  uint32_t lower;     // neighbours ranked below v
  int8_t pos[14];     // rank position among the lower neighbours, -1
  int8_t by_pos[14];  // inverse of pos
  uint16_t adjn[14];  // lower neighbour i: bit q = linked to the lower neighbour at position q
  int nl;
};

// Link adjacency of neighbour I (compile time) in rank-position space.
template <int I>
__device__ __forceinline__ void star_adj_of(Star& s) {
  uint32_t r = 0;
#pragma unroll
  for (int j = 0; j < 14; ++j)
    if ((geo_adj(I) >> j) & 1u)
      if ((s.lower >> j) & 1u) r |= 1u << s.pos[j];
  s.adjn[I] = (uint16_t)r;
}
template <int... I>
__device__ __forceinline__ void star_adj(Star& s, std::integer_sequence<int, I...>) {
  (star_adj_of<I>(s), ...);
}

__device__ inline void star_load(Star& s, const Dims& d, uint32_t v, const uint32_t* __restrict__ rank) {
  int x, y, z;
  vxyz(d, v, x, y, z);
  s.rv = __ldg(rank + v);
  s.valid = 0;
  s.lower = 0;
#pragma unroll
  for (int i = 0; i < 14; ++i) {
    int nx, ny, nz;
    s.nr[i] = 0xFFFFFFFFu;
    if (nbr_xyz(d, x, y, z, i, nx, ny, nz)) {
      s.valid |= 1u << i;
      uint32_t r = __ldg(rank + vid(d, nx, ny, nz));
      s.nr[i] = r;
      if (r < s.rv) s.lower |= 1u << i;
    }
  }
  s.nl = 0;
#pragma unroll
  for (int i = 0; i < 14; ++i) {
    s.pos[i] = -1;
    if ((s.lower >> i) & 1u) {
      int p = 0;
#pragma unroll
      for (int j = 0; j < 14; ++j)
        if (((s.lower >> j) & 1u) && s.nr[j] < s.nr[i]) ++p;
      s.pos[i] = (int8_t)p;
      s.by_pos[p] = (int8_t)i;
      ++s.nl;
    }
  }
  star_adj(s, std::make_integer_sequence<int, 14>{});
}

__device__ __forceinline__ int uf_find(int8_t* par, int x) {
  while (par[x] != x) {
    par[x] = par[par[x]];
    x = par[x];
  }
  return x;
}

// Forward sweep of the lower link in lexicographic order: link vertices by
// rank, then each new vertex's link edges to earlier ones by increasing rank.
struct Fwd {
  uint64_t lower_edges;  // link edges of the lower link
  uint64_t link_pos;     // lower link edges that close a cycle (did not merge)
  uint32_t crit_edges;   // surviving link components but the oldest: v*a critical
  int8_t killer[14];     // link edge that killed neighbour a's component, -1
};

// The forward sweep; with CHAINS it also gives, for every killed lower
// neighbour x, y_of[x] = the older representative its component merged
// with and path_of[x] = the link edges of the forest path x ... y through
// the killing edge (a forest path never changes as the forest grows, so the
// paths are taken in the final forest, as xors of paths to the tree roots).
template <bool CHAINS>
__device__ inline void star_forward_impl(const Star& s, Fwd& f, const Geo& G, int8_t* y_of, uint64_t* path_of) {
  int8_t par[14];
  uint32_t tadj[14];
  int8_t in_x[14], other[14];
  f.lower_edges = 0;
  f.link_pos = 0;
  f.crit_edges = 0;
  for (int i = 0; i < 14; ++i) {
    par[i] = (int8_t)i;
    f.killer[i] = -1;
    if (CHAINS) {
      tadj[i] = 0;
      y_of[i] = -1;
      path_of[i] = 0;
    }
  }
  for (int p = 1; p < s.nl; ++p) {
    int a = s.by_pos[p];
    for (uint32_t qm = s.adjn[a] & ((1u << p) - 1u); qm; qm &= qm - 1) {
      int q = __ffs(qm) - 1;
      int b = s.by_pos[q];
      int e = G.edge_idx[a][b];
      f.lower_edges |= 1ull << e;
      int ra = uf_find(par, p), rb = uf_find(par, q);
      if (ra == rb) {
        f.link_pos |= 1ull << e;
      } else {
        int young = ra > rb ? ra : rb, old = ra > rb ? rb : ra;
        int x = s.by_pos[young];
        par[young] = (int8_t)old;
        f.killer[x] = (int8_t)e;
        if (CHAINS) {
          y_of[x] = s.by_pos[old];
          in_x[x] = (int8_t)(ra == young ? a : b);
          other[x] = (int8_t)(ra == young ? b : a);
          tadj[a] |= 1u << b;
          tadj[b] |= 1u << a;
        }
      }
    }
  }
  for (int p = 1; p < s.nl; ++p)
    if (uf_find(par, p) == p) f.crit_edges |= 1u << s.by_pos[p];
  if (CHAINS) {
    // link edges from every vertex to the root of its tree (the vertex of
    // rank position 0 of its component, any root works): the forest path
    // between two vertices of one tree is the xor of their root paths
    uint64_t rp[14];
    uint32_t done = 0;
    for (int p = 0; p < s.nl; ++p) {
      int r = s.by_pos[p];
      if ((done >> r) & 1u) continue;
      rp[r] = 0;
      done |= 1u << r;
      uint32_t frontier = 1u << r;
      while (frontier) {
        uint32_t nf = 0;
        for (uint32_t fm = frontier; fm; fm &= fm - 1) {
          int u = __ffs(fm) - 1;
          for (uint32_t m = tadj[u] & ~done; m; m &= m - 1) {
            int w2 = __ffs(m) - 1;
            rp[w2] = rp[u] ^ (1ull << G.edge_idx[u][w2]);
            done |= 1u << w2;
            nf |= 1u << w2;
          }
        }
        frontier = nf;
      }
    }
    for (int x = 0; x < 14; ++x)
      if (y_of[x] >= 0)
        path_of[x] = rp[x] ^ rp[in_x[x]] ^ (1ull << f.killer[x]) ^ rp[other[x]] ^ rp[y_of[x]];
  }
}

__device__ inline void star_forward(const Star& s, Fwd& f, const Geo& G) {
  star_forward_impl<false>(s, f, G, nullptr, nullptr);
}

// Key of a link triangle for the backward sweep (larger = later in the
// filtration = older in the backward sweep).
__device__ __forceinline__ int star_tri_key(const Star& s, int tau, const Geo& G) {
  int p0 = s.pos[G.tri[tau][0]], p1 = s.pos[G.tri[tau][1]], p2 = s.pos[G.tri[tau][2]];
  int hi = max(p0, max(p1, p2)), lo = min(p0, min(p1, p2));
  int mid = p0 + p1 + p2 - hi - lo;
  return hi * 196 + mid * 14 + lo;
}

struct Dual {
  uint8_t code[24];     // record code per link triangle (see Rec)
  int8_t killer[24];    // link edge whose triangle killed tau, -1
  uint64_t crit_tris;   // critical triangles v*e by link edge
  bool has_max;
  bool inconsistent;
};

__device__ inline void star_dual(const Star& s, const Fwd& f, Dual& du, const Geo& G) {
  const int OUT = 24;
  int8_t par[25];
  int key[24];
  du.crit_tris = 0;
  du.has_max = false;
  du.inconsistent = false;
  for (int t = 0; t < 24; ++t) {
    par[t] = (int8_t)t;
    du.killer[t] = -1;
    uint32_t m = (1u << G.tri[t][0]) | (1u << G.tri[t][1]) | (1u << G.tri[t][2]);
    bool low = (s.lower & m) == m;
    du.code[t] = low ? (uint8_t)kCodeMax : (uint8_t)kCodeNone;
    key[t] = low ? star_tri_key(s, t, G) : 0;
  }
  par[OUT] = OUT;
  for (int p = s.nl - 1; p >= 1; --p) {
    int a = s.by_pos[p];
    for (uint32_t qm = s.adjn[a] & ((1u << p) - 1u); qm;) {
      int q = 31 - __clz(qm);
      qm ^= 1u << q;
      int b = s.by_pos[q];
      int e = G.edge_idx[a][b];
      int node[2], tcode[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        int t = G.edge_tri[e][k];
        int j = G.edge_third[e][k];
        int c = G.tri[t][j];
        if (!((s.valid >> c) & 1u)) {
          node[k] = OUT;
          tcode[k] = kCodeOut;
        } else if ((s.lower >> c) & 1u) {
          node[k] = t;
          tcode[k] = t;
        } else {
          node[k] = OUT;
          tcode[k] = 24 + 3 * t + j;
        }
      }
      int r0 = uf_find(par, node[0]), r1 = uf_find(par, node[1]);
      if (r0 == r1) {
        if ((f.link_pos >> e) & 1ull) du.crit_tris |= 1ull << e;
      } else {
        int k0 = (r0 == OUT) ? 0x7FFFFFFF : key[r0];
        int k1 = (r1 == OUT) ? 0x7FFFFFFF : key[r1];
        int dside = (k0 < k1) ? 0 : 1;
        int rd = dside == 0 ? r0 : r1, ro = dside == 0 ? r1 : r0;
        du.code[rd] = (uint8_t)tcode[1 - dside];
        du.killer[rd] = (int8_t)e;
        par[rd] = (int8_t)ro;
        if (!((f.link_pos >> e) & 1ull)) du.inconsistent = true;
      }
    }
  }
  for (int t = 0; t < 24; ++t)
    if (du.code[t] == kCodeMax) du.has_max = true;
}

__device__ inline Rec star_record(const Star& s, const Fwd& f, const Dual& du) {
  Rec r;
#pragma unroll
  for (int i = 0; i < 8; ++i) r.w[i] = 0;
  uint32_t vnext = s.nl > 0 ? (uint32_t)s.by_pos[0] : (uint32_t)kVnextMin;
  r.w[0] = vnext | (f.crit_edges << 4) | ((uint32_t)(du.crit_tris & 0x3FFFull) << 18);
  r.w[1] = (uint32_t)((du.crit_tris >> 14) & 0x3FFFFFull) | ((du.has_max ? 1u : 0u) << 22);
  for (int t = 0; t < 24; ++t) rec_set(r, 56 + 7 * t, 7, du.code[t]);
  return r;
}

// Lexicographic key of a link edge (a, b) of the lower link: (higher rank
// position, lower rank position).
__device__ __forceinline__ int star_edge_key(const Star& s, int e, const Geo& G) {
  int pa = s.pos[G.edge[e][0]], pb = s.pos[G.edge[e][1]];
  return max(pa, pb) * 14 + min(pa, pb);
}

}  // namespace tsf

namespace tsf {

}  // namespace tsf

namespace tsf {

// For every lower neighbour x killed in the forward sweep: y_of[x] = the
// older representative its component merged with, path_of[x] = the link
// edges (bitmask) of the forest path x ... y through the killing edge.  The
// reduced column of the triangle paired with w*x is w*x + w*y + path.
__device__ inline void star_chains(const Star& s, int8_t* y_of, uint64_t* path_of, const Geo& G) {
  Fwd f;
  star_forward_impl<true>(s, f, G, y_of, path_of);
}

}  // namespace tsf
