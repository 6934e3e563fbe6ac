// tsf_geo.cuh -- the Freudenthal triangulation of a regular grid, seen from
// one vertex (paper Section 2.1: the implicit triangulation of the grid).
//
// Every vertex v has 14 neighbours v + o, where o (or -o) is a non-zero 0/1
// vector.  Three points form a triangle, four a tetrahedron, exactly when they
// are pairwise neighbours (the triangulation is a flag complex: pairwise
// comparable corners of one cube form a chain).  The *link* of v is a
// triangulated sphere with 14 vertices, 36 edges and 24 triangles; the
// simplices containing v are v itself, 14 edges v*a, 36 triangles v*(a,b) and
// 24 tetrahedra v*(a,b,c) for link vertices a, link edges (a,b) and link
// triangles (a,b,c).  All tables below are computed at compile time from that
// definition.
#pragma once
#include <cstdint>

namespace tsf {

struct Geo {
  int8_t off[14][3];        // neighbour offsets; 0..6 = +mask(1..7), 7..13 = -mask(1..7)
  int8_t edge[36][2];       // link edge -> neighbour indices (a < b)
  int8_t edge_idx[14][14];  // neighbour pair -> link edge, -1 if not adjacent
  int8_t tri[24][3];        // link triangle -> neighbour indices (a < b < c)
  int8_t tri_edge[24][3];   // link triangle -> its three link edges
  int8_t edge_tri[36][2];   // link edge -> the two link triangles containing it
  int8_t edge_third[36][2]; // ... and the slot (0..2) of each triangle's third vertex
  uint16_t adj[14];         // link adjacency bitmask per neighbour
  int8_t nbr_of[27];        // (dx+1) + 3 (dy+1) + 9 (dz+1) -> neighbour index, -1
  int8_t tri_of3[14][14][14];  // neighbour triple -> link triangle, -1
};

constexpr bool geo_is_nbr(int dx, int dy, int dz) {
  if (dx == 0 && dy == 0 && dz == 0) return false;
  if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) return false;
  return (dx >= 0 && dy >= 0 && dz >= 0) || (dx <= 0 && dy <= 0 && dz <= 0);
}

constexpr Geo make_geo() {
  Geo g{};
  for (int m = 1; m < 8; ++m) {
    g.off[m - 1][0] = (int8_t)(m & 1);
    g.off[m - 1][1] = (int8_t)((m >> 1) & 1);
    g.off[m - 1][2] = (int8_t)((m >> 2) & 1);
    g.off[m + 6][0] = (int8_t)(-(m & 1));
    g.off[m + 6][1] = (int8_t)(-((m >> 1) & 1));
    g.off[m + 6][2] = (int8_t)(-((m >> 2) & 1));
  }
  for (int i = 0; i < 27; ++i) g.nbr_of[i] = -1;
  for (int i = 0; i < 14; ++i) g.nbr_of[(g.off[i][0] + 1) + 3 * (g.off[i][1] + 1) + 9 * (g.off[i][2] + 1)] = (int8_t)i;
  for (int i = 0; i < 14; ++i) {
    g.adj[i] = 0;
    for (int j = 0; j < 14; ++j) g.edge_idx[i][j] = -1;
  }
  int ne = 0;
  for (int i = 0; i < 14; ++i)
    for (int j = i + 1; j < 14; ++j)
      if (geo_is_nbr(g.off[j][0] - g.off[i][0], g.off[j][1] - g.off[i][1], g.off[j][2] - g.off[i][2])) {
        g.edge[ne][0] = (int8_t)i;
        g.edge[ne][1] = (int8_t)j;
        g.edge_idx[i][j] = g.edge_idx[j][i] = (int8_t)ne;
        g.adj[i] = (uint16_t)(g.adj[i] | (1u << j));
        g.adj[j] = (uint16_t)(g.adj[j] | (1u << i));
        ++ne;
      }
  for (int e = 0; e < 36; ++e) g.edge_tri[e][0] = g.edge_tri[e][1] = -1;
  for (int i = 0; i < 14; ++i)
    for (int j = 0; j < 14; ++j)
      for (int k = 0; k < 14; ++k) g.tri_of3[i][j][k] = -1;
  int nt = 0;
  for (int i = 0; i < 14; ++i)
    for (int j = i + 1; j < 14; ++j)
      for (int k = j + 1; k < 14; ++k)
        if (g.edge_idx[i][j] >= 0 && g.edge_idx[i][k] >= 0 && g.edge_idx[j][k] >= 0) {
          g.tri[nt][0] = (int8_t)i;
          g.tri[nt][1] = (int8_t)j;
          g.tri[nt][2] = (int8_t)k;
          int es[3] = {g.edge_idx[i][j], g.edge_idx[i][k], g.edge_idx[j][k]};
          for (int s = 0; s < 3; ++s) {
            g.tri_edge[nt][s] = (int8_t)es[s];
            if (g.edge_tri[es[s]][0] < 0) g.edge_tri[es[s]][0] = (int8_t)nt;
            else g.edge_tri[es[s]][1] = (int8_t)nt;
          }
          int p[3] = {i, j, k};
          for (int s2 = 0; s2 < 3; ++s2) {
            int ee = es[s2], slot = g.edge_tri[ee][1] == nt ? 1 : 0;
            for (int q = 0; q < 3; ++q)
              if (p[q] != g.edge[ee][0] && p[q] != g.edge[ee][1]) g.edge_third[ee][slot] = (int8_t)q;
          }
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
              for (int c = 0; c < 3; ++c)
                if (a != b && a != c && b != c) g.tri_of3[p[a]][p[b]][p[c]] = (int8_t)nt;
          ++nt;
        }
  return g;
}

constexpr Geo kGeo = make_geo();

// Compile-time lookups for fully unrolled device code: link edge `le`'s
// endpoints, and the neighbour index of b - a as seen from neighbour a.
__host__ __device__ constexpr int geo_edge(int le, int k) { return kGeo.edge[le][k]; }
__host__ __device__ constexpr uint32_t geo_adj(int a) { return kGeo.adj[a]; }
__host__ __device__ constexpr int geo_dir(int a, int b) {
  return kGeo.nbr_of[(kGeo.off[b][0] - kGeo.off[a][0] + 1) + 3 * (kGeo.off[b][1] - kGeo.off[a][1] + 1) +
                     9 * (kGeo.off[b][2] - kGeo.off[a][2] + 1)];
}

// Crossing into the next lower star on an ascending dual line: the
// tetrahedron v*tau whose record code is 24 + 3 t + j continues as the
// tetrahedron of neighbour c = tri[t][j]'s star opposite the same triangle:
// its link triangle there is (v, p, q) seen from c.  up_step[code - 24] =
// {c, that link triangle}, or {-1, -1} if the geometry has none.
struct UpStep {
  int8_t c, tau;
};
struct UpSteps {
  UpStep s[72];
};
constexpr UpSteps make_up_steps() {
  UpSteps u{};
  for (int code = 0; code < 72; ++code) {
    int t2 = code / 3, j = code % 3;
    int c = kGeo.tri[t2][j], p = kGeo.tri[t2][(j + 1) % 3], q = kGeo.tri[t2][(j + 2) % 3];
    auto idx = [](int dx, int dy, int dz) { return kGeo.nbr_of[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)]; };
    int i0 = idx(-kGeo.off[c][0], -kGeo.off[c][1], -kGeo.off[c][2]);
    int i1 = idx(kGeo.off[p][0] - kGeo.off[c][0], kGeo.off[p][1] - kGeo.off[c][1], kGeo.off[p][2] - kGeo.off[c][2]);
    int i2 = idx(kGeo.off[q][0] - kGeo.off[c][0], kGeo.off[q][1] - kGeo.off[c][1], kGeo.off[q][2] - kGeo.off[c][2]);
    int tau = (i0 >= 0 && i1 >= 0 && i2 >= 0) ? kGeo.tri_of3[i0][i1][i2] : -1;
    u.s[code].c = (int8_t)(tau >= 0 ? c : -1);
    u.s[code].tau = (int8_t)tau;
  }
  return u;
}
constexpr UpSteps kUpSteps = make_up_steps();
constexpr bool up_steps_complete() {
  for (int k = 0; k < 72; ++k)
    if (kUpSteps.s[k].c < 0) return false;
  return true;
}
static_assert(up_steps_complete(), "every link triangle of a neighbour star continues across the shared face");

constexpr bool geo_link_dirs_valid() {
  for (int e = 0; e < 36; ++e)
    if (geo_dir(geo_edge(e, 0), geo_edge(e, 1)) < 0 || geo_dir(geo_edge(e, 1), geo_edge(e, 0)) < 0) return false;
  return true;
}
static_assert(geo_link_dirs_valid(), "the endpoints of a link edge are neighbours of each other");

constexpr int geo_count_edges() {
  int n = 0;
  for (int i = 0; i < 14; ++i)
    for (int j = i + 1; j < 14; ++j) n += kGeo.edge_idx[i][j] >= 0;
  return n;
}
constexpr bool geo_edges_have_two_triangles() {
  for (int e = 0; e < 36; ++e)
    if (kGeo.edge_tri[e][0] < 0 || kGeo.edge_tri[e][1] < 0) return false;
  return true;
}
static_assert(geo_count_edges() == 36, "the link of a Freudenthal vertex has 36 edges");
static_assert(geo_edges_have_two_triangles(), "the link is a closed surface: 24 triangles, 2 per edge");
constexpr bool geo_third_vertices_valid() {
  for (int e = 0; e < 36; ++e)
    for (int k = 0; k < 2; ++k) {
      int c = kGeo.tri[kGeo.edge_tri[e][k]][kGeo.edge_third[e][k]];
      if (c == kGeo.edge[e][0] || c == kGeo.edge[e][1]) return false;
    }
  return true;
}
static_assert(geo_third_vertices_valid(), "edge_third names the vertex of each triangle off the edge");

}  // namespace tsf
