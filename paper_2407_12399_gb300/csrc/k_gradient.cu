// k_gradient.cu -- lower-star discrete gradient (Section 4.2) and compaction
// of the critical cells in lexicographic order.
#include <algorithm>

#include "tsf_kernels.cuh"
#include "tsf_star.cuh"

namespace tsf {

// The lower star of v (Section 4.2): its gradient record, the byte naming
// the edge v is paired with, and (tab non-null) the saddle-saddle table row.
__device__ __forceinline__ void gradient_star(const Dims& d, const uint32_t* __restrict__ rank,
                                              const float* __restrict__ values, int64_t v, Rec* __restrict__ rec,
                                              uint8_t* __restrict__ vnext8, D1Tab* __restrict__ tab,
                                              uint32_t* status, const Geo& sg) {
  Star s;
  star_load(s, d, (uint32_t)v, rank);
  Fwd f;
  int8_t y_of[14];
  uint64_t path_of[14];
  if (tab) star_forward_impl<true>(s, f, sg, y_of, path_of);
  else star_forward(s, f, sg);
  Dual du;
  star_dual(s, f, du, sg);
  if (du.inconsistent) atomicOr(status, kErrInconsistent);
  Rec r = star_record(s, f, du);
  uint4* dst = reinterpret_cast<uint4*>(rec + v);
  dst[0] = make_uint4(r.w[0], r.w[1], r.w[2], r.w[3]);
  dst[1] = make_uint4(r.w[4], r.w[5], r.w[6], r.w[7]);
  vnext8[v] = (uint8_t)(r.w[0] & 15u);
  if (tab) {
    // closures by increasing rank position: v*y (pos(y) < pos(x)) is done
    // before the v*x whose chain continues there
    uint32_t crit = rec_crit_edges(r);
    uint64_t cl[14];
    int8_t end[14];
    D1Tab t;
#pragma unroll
    for (int k = 0; k < 10; ++k) t.q[k] = 0;
    unsigned long long ends = ~0ull;
    for (int p = 0; p < s.nl; ++p) {
      int x = s.by_pos[p];
      uint64_t c = 0;
      int e = 15;
      if (p > 0) {
        if ((crit >> x) & 1u) {
          e = x;
        } else {
          int y = y_of[x];
          if (y < 0) {
            atomicOr(status, kErrInconsistent);
          } else {
            c = path_of[x];
            if (y != s.by_pos[0]) {
              c ^= cl[y];
              e = end[y];
            }
          }
        }
      }
      cl[x] = c;
      end[x] = (int8_t)e;
      tab_set_closure(t, x, c);
      ends = (ends & ~(15ull << (4 * x))) | ((unsigned long long)e << (4 * x));
    }
    unsigned long long orient = 0;
    for (int le = 0; le < 36; ++le) {
      int a = sg.edge[le][0], b = sg.edge[le][1];
      if (((s.lower >> a) & (s.lower >> b) & 1u) && s.pos[a] > s.pos[b]) orient |= 1ull << le;
    }
    t.q[8] = ends;
    t.q[9] = orient;
    {
      int x, y, z;
      vxyz(d, (uint32_t)v, x, y, z);
#pragma unroll
      for (int i = 0; i < 14; ++i) {
        int nx, ny, nz;
        t.nkey[i] = nbr_xyz(d, x, y, z, i, nx, ny, nz) ? value_key(__ldg(values + vid(d, nx, ny, nz))) : 0u;
      }
      t.pad[0] = t.pad[1] = 0;
    }
    uint4* dst4 = reinterpret_cast<uint4*>(tab + v);
    const uint4* src4 = reinterpret_cast<const uint4*>(&t);
#pragma unroll
    for (int k = 0; k < 9; ++k) dst4[k] = src4[k];
  }
}

// Every lower star (the first diagram of a field, or without the fast update).
__global__ void k_gradient(Dims d, const uint32_t* __restrict__ rank, const float* __restrict__ values,
                           Rec* __restrict__ rec, uint8_t* __restrict__ vnext8, D1Tab* __restrict__ tab,
                           uint32_t* status) {
  __shared__ Geo sg;
  geo_to_shared(sg);
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < d.nv) gradient_star(d, rank, values, v, rec, vnext8, tab, status, sg);
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

__global__ void k_gradient_list(Dims d, const uint32_t* __restrict__ rank, const float* __restrict__ values,
                                const uint32_t* __restrict__ list, const unsigned long long* __restrict__ count,
                                Rec* __restrict__ rec, uint8_t* __restrict__ vnext8, D1Tab* __restrict__ tab,
                                uint32_t* status) {
  __shared__ Geo sg;
  geo_to_shared(sg);
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (int64_t)*count) gradient_star(d, rank, values, list[i], rec, vnext8, tab, status, sg);
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

void launch_gradient(const Dims& d, const uint32_t* rank, const float* f, Rec* rec, uint8_t* vnext8, D1Tab* tab,
                     uint32_t* status, cudaStream_t st) {
  unsigned nb = (unsigned)((d.nv + 127) / 128);
  k_gradient<<<nb, 128, 0, st>>>(d, rank, f, rec, vnext8, tab, status); note_launch();
}

void launch_gradient_incremental(const Dims& d, const uint32_t* rank, const float* f, const uint32_t* upd, int64_t nu,
                                 uint32_t* mark, uint32_t gen, uint32_t* list, unsigned long long* count, Rec* rec,
                                 uint8_t* vnext8, D1Tab* tab, uint32_t* status, cudaStream_t st) {
  cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
  if (nu <= 0) return;
  unsigned nb = (unsigned)((nu * 15 + 255) / 256);
  k_gradient_expand<<<nb, 256, 0, st>>>(d, upd, nu, mark, gen, list, count); note_launch();
  unsigned nl = (unsigned)((std::min<int64_t>(nu * 15, d.nv) + 127) / 128);
  k_gradient_list<<<nl, 128, 0, st>>>(d, rank, f, list, count, rec, vnext8, tab, status); note_launch();
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
