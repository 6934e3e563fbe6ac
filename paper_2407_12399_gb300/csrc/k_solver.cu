// k_solver.cu -- diagram assembly (Section 2.2), diagram order (Section 2.4),
// target diagram (Section 3), still pairs and the reduced assignment
// (Section 4.3, Eq. 1), the direct gradient step (Section 4.1) and the loss
// (Eq. 2).
#include <atomic>
#include "tsf_kernels.cuh"
#include "tsf_grid.cuh"
#include "tsf_solver.cuh"

namespace tsf {

// ---------------------------------------------------------------------------
// Merge sort of an index array by a comparator (bottom-up, stable; each pass
// places every element by a binary search in its partner run).
// ---------------------------------------------------------------------------
template <class Less>
__global__ void k_merge_pass(int n, const int* __restrict__ n_dev, int width, const int32_t* __restrict__ in,
                             int32_t* __restrict__ out, Less less) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (n_dev) n = min(*n_dev, n);
  if (i >= n) return;
  int run = i / width;
  int pair_start = (run & ~1) * width;
  bool left = (run & 1) == 0;
  int own_start = run * width;
  int p = i - own_start;
  int o_start = left ? own_start + width : own_start - width;
  int o_len = left ? max(0, min(width, n - o_start)) : width;
  int x = in[i];
  int lo = 0, hi = o_len;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    int y = in[o_start + mid];
    // left-run elements go before equal right-run elements (stability)
    bool before = left ? less(y, x) : !less(x, y);
    if (before) lo = mid + 1;
    else hi = mid;
  }
  out[pair_start + p + lo] = x;
}

// The first log2(kTile) merge levels run as one launch: every block sorts a
// tile of kTile indices with a bitonic network in shared memory over
// (primary key, index).  Each comparator supplies key(i), a 64-bit
// coarsening of its order (key(a) < key(b) implies a before b); equal keys
// fall back to the comparator.  The comparators here are total orders, or
// order equal values only, so the tiles need no stability; the merge passes
// above them are stable.  With n_dev non-null the count is read on the
// device and n is only its upper bound.
constexpr int kTileT = 1024, kTile = 2 * kTileT;

template <class Less>
__global__ void __launch_bounds__(kTileT) k_tile_sort(int n, const int* __restrict__ n_dev, int32_t* __restrict__ out,
                                                      Less less) {
  __shared__ unsigned long long K[kTile];
  __shared__ int32_t I[kTile];
  if (n_dev) n = min(*n_dev, n);
  const int base = blockIdx.x * kTile;
  const int m = min(kTile, n - base);
  if (m <= 0) return;
  int n2 = 1;
  while (n2 < m) n2 <<= 1;
  for (int i = threadIdx.x; i < n2; i += kTileT) {
    K[i] = i < m ? less.key(base + i) : ~0ull;
    I[i] = i < m ? base + i : -1;  // -1 sorts after everything
  }
  __syncthreads();
  for (int size = 2; size <= n2; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < n2; i += kTileT) {
        int j = i ^ stride;
        if (j > i) {
          bool up = (i & size) == 0;
          unsigned long long kx = K[i], ky = K[j];
          int x = I[i], y = I[j];
          bool x_after_y = kx != ky ? kx > ky : (x < 0 ? y >= 0 : (y >= 0 && less(y, x)));
          if (x_after_y == up) {
            K[i] = ky;
            K[j] = kx;
            I[i] = y;
            I[j] = x;
          }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < m; i += kTileT) out[base + i] = I[i];
}

template <class Less>
static int32_t* merge_sort(int n, int32_t* a, int32_t* b, Less less, cudaStream_t st, const int* n_dev = nullptr) {
  if (n <= 0) return a;
  k_tile_sort<<<(n + kTile - 1) / kTile, kTileT, 0, st>>>(n, n_dev, a, less); note_launch();
  for (int w = kTile; w < n; w *= 2) {
    k_merge_pass<<<(n + 255) / 256, 256, 0, st>>>(n, n_dev, w, a, b, less); note_launch();
    int32_t* t = a;
    a = b;
    b = t;
  }
  return a;
}

// ---------------------------------------------------------------------------
// Stable order of n items by a 64-bit key: two stable LSD radix sorts of the
// 32-bit halves (low, then high), each four onesweep passes.  Items at or
// beyond *n_dev (when given) get the largest key.  Equal keys keep their
// index order, like the merge sort above.  Returns out (n indices).
// ---------------------------------------------------------------------------
template <class KeyFn>
__global__ void k_key64(int n, const int* __restrict__ n_dev, KeyFn kf, uint32_t* __restrict__ lo,
                        uint32_t* __restrict__ hi, uint32_t* __restrict__ iota) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int m = n_dev ? min(*n_dev, n) : n;
  const unsigned long long k = i < m ? kf(i) : ~0ull;
  lo[i] = (uint32_t)k;
  hi[i] = (uint32_t)(k >> 32);
  iota[i] = (uint32_t)i;
}

__global__ void k_gather_u32(int n, const uint32_t* __restrict__ src, const uint32_t* __restrict__ perm,
                             uint32_t* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[perm[i]];
}

template <class KeyFn>
static int32_t* radix_sort64(int n, const int* n_dev, KeyFn kf, uint32_t* rs, int32_t* tmp, int32_t* out,
                             uint32_t* status, cudaStream_t st) {
  if (n <= 0) return out;
  uint32_t* lo = rs;
  uint32_t* hi = lo + n;
  uint32_t* hi2 = hi + n;
  uint32_t* iota = hi2 + n;
  uint32_t* scratch = iota + n;
  const unsigned nb = (unsigned)((n + 255) / 256);
  k_key64<<<nb, 256, 0, st>>>(n, n_dev, kf, lo, hi, iota); note_launch();
  uint32_t* p1 = reinterpret_cast<uint32_t*>(tmp);
  sort_u32_pairs(lo, iota, n, nullptr, p1, scratch, status, st);
  k_gather_u32<<<nb, 256, 0, st>>>(n, hi, p1, hi2); note_launch();
  sort_u32_pairs(hi2, p1, n, nullptr, reinterpret_cast<uint32_t*>(out), scratch, status, st);
  return out;
}

int64_t radix_sort64_words(int64_t n) { return 4 * n + sort_scratch_words(n); }

// ---------------------------------------------------------------------------
// diagram assembly
// ---------------------------------------------------------------------------
__device__ __forceinline__ void xyz_of(const Dims& d, uint32_t v, int* o) { vxyz(d, v, o[0], o[1], o[2]); }

__global__ void k_build_points(Dims d, NbrDelta nd, CritLists L, int n1, int n2, int n3, const int32_t* __restrict__ d0_min,
                               const int32_t* __restrict__ d1_edge, const int32_t* __restrict__ d2_max,
                               const uint32_t* __restrict__ order, const float* __restrict__ f, Pt* __restrict__ pts,
                               int* __restrict__ count, int cap) {
  __shared__ Geo sg;
  geo_to_shared(sg);
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int xs[4][3];
  auto put = [&](Pt& p) {
    int k = atomicAdd(count, 1);
    if (k < cap) pts[k] = p;
  };
  if (i < n1) {  // D0: (minimum, critical edge)
    int m = d0_min[i];
    if (m >= 0) {
      Pt p;
      uint32_t vn = L.c1_vn[i];
      uint32_t v = vn >> 4;
      uint32_t u = (uint32_t)((int32_t)v + nd.d[vn & 15u]);
      p.vb = L.c0[m];
      p.vd = v;
      xyz_of(d, p.vb, xs[0]);
      p.cb = cell_id_of(d, 1, xs);
      xyz_of(d, v, xs[0]);
      xyz_of(d, u, xs[1]);
      p.cd = cell_id_of(d, 2, xs);
      p.dim = 0;
      p.ess = 0;
      p.b = f[p.vb];
      p.d = f[p.vd];
      p.tgt = -1;
      p.still = 0;
      put(p);
    }
  }
  if (i < n2) {
    uint32_t ve = L.c2_ve[i];
    uint32_t v = ve >> 6;
    int e = (int)(ve & 63u);
    xyz_of(d, v, xs[0]);
    xyz_of(d, (uint32_t)((int32_t)v + nd.d[sg.edge[e][0]]), xs[1]);
    xyz_of(d, (uint32_t)((int32_t)v + nd.d[sg.edge[e][1]]), xs[2]);
    uint64_t tri = cell_id_of(d, 3, xs);
    int ce = d1_edge[i], mx = d2_max[i];
    if (ce >= 0) {  // D1: (critical edge, critical triangle)
      Pt p;
      uint32_t vn = L.c1_vn[ce];
      uint32_t w = vn >> 4;
      int ys[4][3];
      xyz_of(d, w, ys[0]);
      xyz_of(d, (uint32_t)((int32_t)w + nd.d[vn & 15u]), ys[1]);
      p.cb = cell_id_of(d, 2, ys);
      p.cd = tri;
      p.vb = w;
      p.vd = v;
      p.dim = 1;
      p.ess = 0;
      p.b = f[w];
      p.d = f[v];
      p.tgt = -1;
      p.still = 0;
      put(p);
    } else if (mx >= 0 && mx < n3) {  // D2: (critical triangle, maximum)
      Pt p;
      uint32_t c3 = L.c3[mx];
      uint32_t w = c3 >> 5;
      int tau = (int)(c3 & 31u);
      int ys[4][3];
      xyz_of(d, w, ys[0]);
      for (int k = 0; k < 3; ++k) xyz_of(d, (uint32_t)((int32_t)w + nd.d[sg.tri[tau][k]]), ys[k + 1]);
      p.cb = tri;
      p.cd = cell_id_of(d, 4, ys);
      p.vb = v;
      p.vd = w;
      p.dim = 2;
      p.ess = 0;
      p.b = f[v];
      p.d = f[w];
      p.tgt = -1;
      p.still = 0;
      put(p);
    }
  }
  if (i == 0) {  // the essential class, at (f(v_min), f(v_max))
    Pt p;
    p.vb = order[0];
    p.vd = order[d.nv - 1];
    xyz_of(d, p.vb, xs[0]);
    p.cb = cell_id_of(d, 1, xs);
    p.cd = ~0ull;
    p.dim = 0;
    p.ess = 1;
    p.b = f[p.vb];
    p.d = f[p.vd];
    p.tgt = -1;
    p.still = 0;
    put(p);
  }
}

struct DiagLess {
  const Pt* p;
  __device__ unsigned long long key(int i) const {
    return ((unsigned long long)value_key(p[i].b) << 32) | value_key(p[i].d);
  }
  __device__ bool operator()(int a, int b) const {
    const Pt& x = p[a];
    const Pt& y = p[b];
    uint32_t xb = value_key(x.b), yb = value_key(y.b);
    if (xb != yb) return xb < yb;
    uint32_t xd = value_key(x.d), yd = value_key(y.d);
    if (xd != yd) return xd < yd;
    if (x.vb != y.vb) return x.vb < y.vb;
    if (x.vd != y.vd) return x.vd < y.vd;
    return x.cb < y.cb;
  }
};

struct KeyLess {  // (essential, dim, v_b, v_d, birth cell)
  const Pt* p;
  __device__ unsigned long long key(int i) const {  // (essential, dim, v_b, v_d >> 3)
    const Pt& x = p[i];
    return ((unsigned long long)(x.ess != 0) << 63) | ((unsigned long long)(x.dim & 3) << 61) |
           ((unsigned long long)x.vb << 29) | (unsigned long long)(x.vd >> 3);
  }
  __device__ bool operator()(int a, int b) const {
    const Pt& x = p[a];
    const Pt& y = p[b];
    if (x.ess != y.ess) return x.ess < y.ess;
    if (x.dim != y.dim) return x.dim < y.dim;
    if (x.vb != y.vb) return x.vb < y.vb;
    if (x.vd != y.vd) return x.vd < y.vd;
    return x.cb < y.cb;
  }
};

// KeyLess as one 64-bit key when vertex ids fit 30 bits: (essential, dim,
// v_b, v_d); equal keys keep index order, which is birth-cell order in a
// diagram (points with the same vertices share their values, and diagram
// order then goes by birth cell).
struct KeyBits {
  const Pt* p;
  __device__ unsigned long long operator()(int i) const {
    const Pt& x = p[i];
    return ((unsigned long long)(x.ess != 0) << 62) | ((unsigned long long)(x.dim & 3) << 60) |
           ((unsigned long long)x.vb << 30) | (unsigned long long)x.vd;
  }
};

__global__ void k_gather_pts(int n, const int32_t* __restrict__ idx, const Pt* __restrict__ in, Pt* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[idx[i]];
}

int build_diagram(const Dims& d, const NbrDelta& nd, const CritLists& L, int n1, int n2, int n3, const PairOut& P,
                  const uint32_t* order, const float* f, SolverBufs& B, Pt* out, int cap, cudaStream_t st) {
  cudaMemsetAsync(B.count, 0, sizeof(int), st);
  int n = max(max(n1, n2), 1);
  k_build_points<<<(n + 255) / 256, 256, 0, st>>>(d, nd, L, n1, n2, n3, P.d0_min, P.d1_edge, P.d2_max, order, f,
                                                  B.tmp_pts, B.count, cap); note_launch();
  int np = 0;
  cudaMemcpyAsync(&np, B.count, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  if (np > cap) return -np;
  int32_t* idx = merge_sort(np, B.idxA, B.idxB, DiagLess{B.tmp_pts}, st);
  k_gather_pts<<<(np + 255) / 256, 256, 0, st>>>(np, idx, B.tmp_pts, out); note_launch();
  return np;
}

// ---------------------------------------------------------------------------
// target diagram from a persistence threshold (Section 3)
// ---------------------------------------------------------------------------
// Signal threshold of Section 3: theta = fl(fraction * fl(max f - min f)),
// the extreme values read through the vertex order (first and last vertex).
__device__ __forceinline__ float signal_theta(const uint32_t* __restrict__ order, const float* __restrict__ f,
                                              int64_t nv, float fraction) {
  const float lo = f[order[0]], hi = f[order[nv - 1]];
  return __fmul_rn(fraction, __fsub_rn(hi, lo));
}

__global__ void k_select_targets(int np, const Pt* __restrict__ pts, const uint32_t* __restrict__ order,
                                 const float* __restrict__ f, int64_t nv, float fraction,
                                 uint32_t* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < np) {
    const float theta = signal_theta(order, f, nv, fraction);
    float pers = __fsub_rn(pts[i].d, pts[i].b);
    flag[i] = (pts[i].ess || pers >= theta) ? 1u : 0u;
  }
}
__global__ void k_write_targets(int np, const Pt* __restrict__ pts, const uint32_t* __restrict__ flag,
                                const uint32_t* __restrict__ pos, Tg* __restrict__ T) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < np && flag[i]) {
    Tg t;
    t.b = pts[i].b;
    t.d = pts[i].d;
    t.vb = pts[i].vb;
    t.vd = pts[i].vd;
    t.src = pts[i].cb;
    t.dim = pts[i].dim;
    t.ess = pts[i].ess;
    T[pos[i]] = t;
  }
}

int make_targets(int np, const Pt* pts, const uint32_t* order, const float* f, int64_t nv, float fraction,
                 SolverBufs& B, Tg* T, cudaStream_t st) {
  uint32_t* flag = B.u32a;
  uint32_t* pos = B.u32b;
  k_select_targets<<<(np + 255) / 256, 256, 0, st>>>(np, pts, order, f, nv, fraction, flag); note_launch();
  exclusive_scan_u32(flag, pos, np, B.u32c, st);
  k_write_targets<<<(np + 255) / 256, 256, 0, st>>>(np, pts, flag, pos, T); note_launch();
  uint32_t tail[2];
  cudaMemcpyAsync(&tail[0], pos + np - 1, 4, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&tail[1], flag + np - 1, 4, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return (int)(tail[0] + tail[1]);
}

// ---------------------------------------------------------------------------
// still pairs (Section 4.3)
// ---------------------------------------------------------------------------
__global__ void k_targets_as_points(int nt, const Tg* __restrict__ T, Pt* __restrict__ R) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nt) {
    Pt p;
    p.b = T[t].b;
    p.d = T[t].d;
    p.vb = T[t].vb;
    p.vd = T[t].vd;
    p.cb = T[t].src;
    p.cd = 0;
    p.dim = T[t].dim;
    p.ess = T[t].ess;
    p.tgt = t;
    p.still = 0;
    R[t] = p;
  }
}

__device__ __forceinline__ int key_cmp(const Pt& x, const Pt& y) {
  if (x.ess != y.ess) return x.ess < y.ess ? -1 : 1;
  if (x.dim != y.dim) return x.dim < y.dim ? -1 : 1;
  if (x.vb != y.vb) return x.vb < y.vb ? -1 : 1;
  if (x.vd != y.vd) return x.vd < y.vd ? -1 : 1;
  return 0;
}

// For each current point (in key order) the k-th point with its key is still
// if the reference list has at least k points with that key; it inherits the
// reference point's assignment.
__global__ void k_still(int np, const Pt* __restrict__ cur, const int32_t* __restrict__ ck, int nr,
                        const Pt* __restrict__ ref, const int32_t* __restrict__ rk, Pt* __restrict__ out,
                        uint8_t* __restrict__ taken) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= np) return;
  int i = ck[r];
  const Pt& x = cur[i];
  // first index with this key in the current key order
  int lo = 0, hi = r;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (key_cmp(cur[ck[mid]], x) < 0) lo = mid + 1;
    else hi = mid;
  }
  int rank_in_key = r - lo;
  int a = 0, b = nr;
  while (a < b) {
    int mid = (a + b) >> 1;
    if (key_cmp(ref[rk[mid]], x) < 0) a = mid + 1;
    else b = mid;
  }
  int j = a + rank_in_key;
  Pt p = x;
  p.tgt = -1;
  p.still = 0;
  if (j < nr && key_cmp(ref[rk[j]], x) == 0) {
    p.still = 1;
    p.tgt = ref[rk[j]].tgt;
    if (p.tgt >= 0) taken[p.tgt] = 1;
  }
  out[i] = p;
}

// ---------------------------------------------------------------------------
// reduced assignment (Eq. 1, q = 2), one finite group
// ---------------------------------------------------------------------------
__device__ __forceinline__ double cost_pt(float pb, float pd, float tb, float td) {
  double db = __dsub_rn((double)pb, (double)tb);
  double dd = __dsub_rn((double)pd, (double)td);
  return __dadd_rn(__dmul_rn(db, db), __dmul_rn(dd, dd));
}
__device__ __forceinline__ double cost_diag(float b, float d) {
  double e = __dsub_rn((double)d, (double)b);
  return __dmul_rn(__dmul_rn(e, e), 0.5);
}

__global__ void k_group_flags(int np, const Pt* __restrict__ pts, int g, uint32_t* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < np) {
    int grp = pts[i].ess ? 3 : pts[i].dim;
    flag[i] = (!pts[i].still && grp == g) ? 1u : 0u;
  }
}
__global__ void k_tgroup_flags(int nt, const Tg* __restrict__ T, const uint8_t* __restrict__ taken, int g,
                               uint32_t* __restrict__ flag) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nt) {
    int grp = T[t].ess ? 3 : T[t].dim;
    flag[t] = (!taken[t] && grp == g) ? 1u : 0u;
  }
}
__global__ void k_compact(int n, const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                          int32_t* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flag[i]) out[pos[i]] = i;
}

// candidates of target t: points p with w(p,t) = c(p,t) - diag(p) < diag(t)
__global__ void k_cand_count(int npg, const int32_t* __restrict__ plist, const Pt* __restrict__ pts, int k,
                             const int32_t* __restrict__ tlist, const Tg* __restrict__ T, uint32_t* __restrict__ cnt) {
  int t = blockIdx.x;
  const Tg tg = T[tlist[t]];
  double dt = cost_diag(tg.b, tg.d);
  uint32_t c = 0;
  for (int i = threadIdx.x; i < npg; i += blockDim.x) {
    const Pt& p = pts[plist[i]];
    double w = __dsub_rn(cost_pt(p.b, p.d, tg.b, tg.d), cost_diag(p.b, p.d));
    c += (w < dt) ? 1u : 0u;
  }
  for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
  __shared__ uint32_t s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) atomicAdd(&s, c);
  __syncthreads();
  if (threadIdx.x == 0) cnt[t] = s;
}

__global__ void k_cand_fill(int npg, const int32_t* __restrict__ plist, const Pt* __restrict__ pts, int k,
                            const int32_t* __restrict__ tlist, const Tg* __restrict__ T,
                            const uint32_t* __restrict__ off, Cand* __restrict__ cands) {
  int t = blockIdx.x;
  const Tg tg = T[tlist[t]];
  double dt = cost_diag(tg.b, tg.d);
  __shared__ uint32_t fill;
  if (threadIdx.x == 0) fill = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < npg; i += blockDim.x) {
    const Pt& p = pts[plist[i]];
    double w = __dsub_rn(cost_pt(p.b, p.d, tg.b, tg.d), cost_diag(p.b, p.d));
    if (w < dt) {
      uint32_t s = atomicAdd(&fill, 1u);
      Cand c;
      c.w = w;
      c.p = i;
      c.t = t;
      cands[off[t] + s] = c;
    }
  }
}

struct CandLess {
  const Cand* c;
  __device__ unsigned long long key(int i) const {  // (target, high half of the monotone image of w)
    unsigned long long u = (unsigned long long)__double_as_longlong(c[i].w);
    u = (u >> 63) ? ~u : (u | (1ull << 63));
    return ((unsigned long long)(uint32_t)c[i].t << 32) | (u >> 32);
  }
  __device__ bool operator()(int a, int b) const {
    const Cand& x = c[a];
    const Cand& y = c[b];
    if (x.t != y.t) return x.t < y.t;
    if (x.w != y.w) return x.w < y.w;
    return x.p < y.p;
  }
};

// keep the k cheapest candidates of each target; mark their points as columns
__global__ void k_cand_keep(int nc, const int32_t* __restrict__ idx, const Cand* __restrict__ cands,
                            const uint32_t* __restrict__ off, int k, uint32_t* __restrict__ is_col,
                            Cand* __restrict__ kept, uint32_t* __restrict__ nkept) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nc) return;
  const Cand c = cands[idx[r]];
  int rank = r - (int)off[c.t];
  if (rank < k) {
    kept[off[c.t] + rank] = c;
    is_col[c.p] = 1u;
    atomicMax(&nkept[c.t], (uint32_t)(rank + 1));
  }
}

constexpr int kHT = 1024;

__device__ __forceinline__ int block_exscan_int1024(int v, int& total) {
  __shared__ int sw[33];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sw[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int s = lane < (int)(blockDim.x >> 5) ? sw[lane] : 0;
    int si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xFFFFFFFFu, si, o);
      if (lane >= o) si += t;
    }
    sw[lane] = si - s;
    if (lane == 31) sw[32] = si;
  }
  __syncthreads();
  int res = sw[wid] + inc - v;
  total = sw[32];
  __syncthreads();
  return res;
}

// Shortest augmenting path (Hungarian algorithm with potentials): rows =
// targets in target order, columns = candidate points (point order) and one
// private diagonal column per target; ties go to the lowest column index.
//
// A row's search only ever reaches the candidate columns of the rows in its
// tree and their diagonal columns; every other column keeps minv = +inf
// (inf - delta = inf) and never takes part in a decision.  So each step works
// on the list of reached columns instead of all m columns: the same
// arithmetic on the same columns, O(reached) per step.  Once a row's search
// has reached more than m/8 columns it sweeps all m columns instead (cheaper
// than gathering through the list; identical results).  Rows: count(r) and
// get(r, c, j, w) give row r's c-th candidate as 1-based column j, weight w.
// The textbook dense form of the same search, for problems small enough
// that sweeping all m columns per step is cheaper than gathering the
// reached ones: row i0's costs are scattered into a dense row (H.aw, +inf
// elsewhere), then one pass relaxes and takes the argmin, one pass moves
// the potentials.  Identical arithmetic and ties.
constexpr int kSapDenseMax = 16384;

template <class Rows>
__device__ bool sap_dense(int k, int mc, const Rows& R, const double* __restrict__ diag_t, HungWork H,
                          uint32_t* status) {
  const int m = mc + k;
  const double INF = __longlong_as_double(0x7FF0000000000000ll);
  double* row = H.aw;
  __shared__ int s_j0;
  __shared__ double s_val[kHT / 32];
  __shared__ int s_idx[kHT / 32];
  __shared__ double s_delta;
  __shared__ int s_j1;
  for (int j = threadIdx.x; j <= m; j += kHT) {
    H.v[j] = 0.0;
    H.pm[j] = 0;
    H.way[j] = 0;
  }
  for (int i = threadIdx.x; i <= k; i += kHT) H.u[i] = 0.0;
  __syncthreads();
  for (int i = 1; i <= k; ++i) {
    for (int j = threadIdx.x; j <= m; j += kHT) {
      H.minv[j] = INF;
      H.used[j] = 0;
    }
    if (threadIdx.x == 0) {
      H.pm[0] = i;
      s_j0 = 0;
    }
    __syncthreads();
    for (int guard = 0;; ++guard) {
      if (guard > m + 2) {
        if (threadIdx.x == 0) atomicOr(status, kErrRounds);
        return false;
      }
      const int j0 = s_j0;
      if (threadIdx.x == 0) H.used[j0] = 1;
      const int i0 = H.pm[j0];
      for (int j = 1 + threadIdx.x; j <= m; j += kHT) row[j] = INF;
      __syncthreads();
      const int n = R.count(i0 - 1);
      for (int c = threadIdx.x; c < n; c += kHT) {
        int j;
        double w;
        R.get(i0 - 1, c, j, w);
        row[j] = w;
      }
      if (threadIdx.x == 0) row[1 + mc + (i0 - 1)] = diag_t[i0 - 1];
      __syncthreads();
      const double ui0 = H.u[i0];
      double bv = INF;
      int bj = 0x7FFFFFFF;
      for (int j = 1 + threadIdx.x; j <= m; j += kHT) {
        if (H.used[j]) continue;
        double cur = __dsub_rn(__dsub_rn(row[j], ui0), H.v[j]);
        double mv = H.minv[j];
        if (cur < mv) {
          mv = cur;
          H.minv[j] = cur;
          H.way[j] = j0;
        }
        if (mv < bv || (mv == bv && j < bj)) {
          bv = mv;
          bj = j;
        }
      }
      for (int o = 16; o; o >>= 1) {
        double ov = __shfl_down_sync(0xFFFFFFFFu, bv, o);
        int oj = __shfl_down_sync(0xFFFFFFFFu, bj, o);
        if (ov < bv || (ov == bv && oj < bj)) {
          bv = ov;
          bj = oj;
        }
      }
      if ((threadIdx.x & 31) == 0) {
        s_val[threadIdx.x >> 5] = bv;
        s_idx[threadIdx.x >> 5] = bj;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double v0 = s_val[0];
        int j1 = s_idx[0];
        for (int w = 1; w < kHT / 32; ++w)
          if (s_val[w] < v0 || (s_val[w] == v0 && s_idx[w] < j1)) {
            v0 = s_val[w];
            j1 = s_idx[w];
          }
        s_delta = v0;
        s_j1 = j1;
      }
      __syncthreads();
      const double delta = s_delta;
      const int j1 = s_j1;
      if (j1 == 0x7FFFFFFF) {
        if (threadIdx.x == 0) atomicOr(status, kErrInconsistent);
        return false;
      }
      for (int j = threadIdx.x; j <= m; j += kHT) {
        if (H.used[j]) {
          int r = H.pm[j];
          H.u[r] = __dadd_rn(H.u[r], delta);
          H.v[j] = __dsub_rn(H.v[j], delta);
        } else {
          H.minv[j] = __dsub_rn(H.minv[j], delta);
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) s_j0 = j1;
      __syncthreads();
      if (H.pm[j1] == 0) break;
    }
    if (threadIdx.x == 0) {
      int j0 = s_j0;
      do {
        int j1 = H.way[j0];
        H.pm[j0] = H.pm[j1];
        j0 = j1;
      } while (j0);
    }
    __syncthreads();
  }
  return true;
}

template <class Rows>
__device__ bool sap_solve(int k, int mc, const Rows& R, const double* __restrict__ diag_t, HungWork H,
                          uint32_t* status) {
  if (mc + k <= kSapDenseMax) return sap_dense(k, mc, R, diag_t, H, status);
  const int m = mc + k;
  const double INF = __longlong_as_double(0x7FF0000000000000ll);
  __shared__ int s_nl;
  __shared__ double s_val[kHT / 32];
  __shared__ int s_idx[kHT / 32];
  const int dense_at = m / 8;
  for (int j = threadIdx.x; j <= m; j += kHT) {
    H.v[j] = 0.0;
    H.pm[j] = 0;
    H.way[j] = 0;
    H.minv[j] = INF;
    H.used[j] = 0;
  }
  for (int i = threadIdx.x; i <= k; i += kHT) H.u[i] = 0.0;
  if (threadIdx.x == 0) s_nl = 0;
  __syncthreads();
  for (int i = 1; i <= k; ++i) {
    if (threadIdx.x == 0) H.pm[0] = i;
    __syncthreads();
    int j0 = 0;
    bool dense = false;
    for (int guard = 0;; ++guard) {
      if (guard > m + 2) {
        if (threadIdx.x == 0) atomicOr(status, kErrRounds);
        return false;
      }
      // relax the columns of row i0 = pm[j0] (its candidates, then its diagonal)
      const int i0 = H.pm[j0];
      const double ui0 = H.u[i0];
      const int n = R.count(i0 - 1);
      for (int c0 = 0; c0 <= n; c0 += kHT) {  // whole warps iterate: the appends are warp-aggregated
        const int c = c0 + threadIdx.x;
        int j = 0;
        bool app = false;
        if (c <= n) {
          double w;
          if (c < n) {
            R.get(i0 - 1, c, j, w);
          } else {
            j = 1 + mc + (i0 - 1);
            w = diag_t[i0 - 1];
          }
          if (j != j0 && !H.used[j]) {
            double cur = __dsub_rn(__dsub_rn(w, ui0), H.v[j]);
            double mv = H.minv[j];
            app = mv == INF && !dense;
            if (cur < mv) {
              H.minv[j] = cur;
              H.way[j] = j0;
            }
          }
        }
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, app);
        if (bal) {
          const int lane = threadIdx.x & 31, leader = __ffs(bal) - 1;
          int base = 0;
          if (lane == leader) base = atomicAdd(&s_nl, __popc(bal));
          base = __shfl_sync(0xFFFFFFFFu, base, leader);
          if (app) H.list[base + __popc(bal & ((1u << lane) - 1u))] = j;
        }
      }
      if (threadIdx.x == 0) H.used[j0] = 1;
      __syncthreads();
      // argmin of minv over the reached unused columns, lowest index on ties
      const int nl = s_nl;
      if (!dense && nl > dense_at) dense = true;  // uniform: every thread reads the same s_nl
      double bv = INF;
      int bj = 0x7FFFFFFF;
      if (dense) {
        for (int j = 1 + threadIdx.x; j <= m; j += kHT) {
          if (H.used[j]) continue;
          double mv = H.minv[j];
          if (mv < bv) {  // unreached columns (minv = inf) never win
            bv = mv;
            bj = j;
          }
        }
      } else {
        for (int q = threadIdx.x; q < nl; q += kHT) {
          int j = H.list[q];
          if (H.used[j]) continue;
          double mv = H.minv[j];
          if (mv < bv || (mv == bv && j < bj)) {
            bv = mv;
            bj = j;
          }
        }
      }
      for (int o = 16; o; o >>= 1) {
        double ov = __shfl_down_sync(0xFFFFFFFFu, bv, o);
        int oj = __shfl_down_sync(0xFFFFFFFFu, bj, o);
        if (ov < bv || (ov == bv && oj < bj)) {
          bv = ov;
          bj = oj;
        }
      }
      if ((threadIdx.x & 31) == 0) {
        s_val[threadIdx.x >> 5] = bv;
        s_idx[threadIdx.x >> 5] = bj;
      }
      __syncthreads();
      double delta = s_val[0];
      int j1 = s_idx[0];
      for (int w = 1; w < kHT / 32; ++w)
        if (s_val[w] < delta || (s_val[w] == delta && s_idx[w] < j1)) {
          delta = s_val[w];
          j1 = s_idx[w];
        }
      if (j1 == 0x7FFFFFFF) {
        if (threadIdx.x == 0) atomicOr(status, kErrInconsistent);
        return false;
      }
      // potentials: the tree's columns (the root column 0 and the used
      // reached ones) and their rows move by delta, the others' minv drop
      if (threadIdx.x == 0) {
        int r = H.pm[0];
        H.u[r] = __dadd_rn(H.u[r], delta);
        H.v[0] = __dsub_rn(H.v[0], delta);
      }
      if (dense) {
        for (int j = 1 + threadIdx.x; j <= m; j += kHT) {
          if (H.used[j]) {
            int r = H.pm[j];
            H.u[r] = __dadd_rn(H.u[r], delta);
            H.v[j] = __dsub_rn(H.v[j], delta);
          } else if (H.minv[j] != INF) {
            H.minv[j] = __dsub_rn(H.minv[j], delta);
          }
        }
      } else {
        for (int q = threadIdx.x; q < nl; q += kHT) {
          int j = H.list[q];
          if (H.used[j]) {
            int r = H.pm[j];
            H.u[r] = __dadd_rn(H.u[r], delta);
            H.v[j] = __dsub_rn(H.v[j], delta);
          } else {
            H.minv[j] = __dsub_rn(H.minv[j], delta);
          }
        }
      }
      __syncthreads();
      j0 = j1;
      if (H.pm[j1] == 0) break;
    }
    if (threadIdx.x == 0) {
      int j = j0;
      do {
        int jp = H.way[j];
        H.pm[j] = H.pm[jp];
        j = jp;
      } while (j);
    }
    // back to the untouched state for the next row
    if (dense) {
      for (int j = 1 + threadIdx.x; j <= m; j += kHT) {
        H.minv[j] = INF;
        H.used[j] = 0;
      }
    } else {
      const int nl = s_nl;
      for (int q = threadIdx.x; q < nl; q += kHT) {
        int j = H.list[q];
        H.minv[j] = INF;
        H.used[j] = 0;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      H.used[0] = 0;
      s_nl = 0;
    }
  }
  __syncthreads();
  return true;
}

struct KeptRows {
  const Cand* kept;
  const uint32_t* koff;
  const uint32_t* nkept;
  const uint32_t* colpos;
  __device__ int count(int r) const { return (int)nkept[r]; }
  __device__ void get(int r, int c, int& j, double& w) const {
    const Cand& cd = kept[koff[r] + c];
    j = 1 + (int)colpos[cd.p];
    w = cd.w;
  }
};

__global__ void __launch_bounds__(kHT, 1) k_hungarian(int k, int mc, const Cand* __restrict__ kept,
                                                   const uint32_t* __restrict__ koff,
                                                   const uint32_t* __restrict__ nkept,
                                                   const uint32_t* __restrict__ colpos,
                                                   const double* __restrict__ diag_t, HungWork H,
                                                   int32_t* __restrict__ col_to_row, uint32_t* status) {
  if (!sap_solve(k, mc, KeptRows{kept, koff, nkept, colpos}, diag_t, H, status)) return;
  for (int j = 1 + threadIdx.x; j <= mc; j += kHT) col_to_row[j - 1] = H.pm[j] - 1;
}


// ---------------------------------------------------------------------------
// Auction variant of the reduced assignment (the paper's implementation,
// Section 5, solves it with the Auction algorithm at relative precision
// 0.01).  Same rows and options as sap_solve; net cost of an option
// w(r,j) + price(j).  Forward auction in synchronous (Jacobi) rounds: every
// unassigned row finds its cheapest net cost n1 (ties: lowest column) at j1
// and the cheapest among its other options n2, and bids
// price(j1) + ((n2 - n1) + eps); each point column takes its highest bid
// (ties: lowest row) and its previous row is unassigned; a bid for the row's
// own diagonal always wins.  eps-scaling: eps = max diag(t) / 4, divided by
// 5 per phase; a later phase keeps the assignment and prices, except that
// (until nothing changes) columns without a row get price 0 and rows whose
// net cost exceeds their cheapest by more than the new eps are released.
// Phase end: every column without a row has price 0, so
// LB = sum_r n1_r - sum_j price(j) bounds the optimum from below and
// W - LB <= k eps for the assignment's cost W; the auction stops once
// W + D <= (1 + prec)(LB + D), D = sum of diag(p) over the group's points
// (the reduced W2^2 within a factor (1 + prec) of its minimum), or once eps
// reaches 2^-40 max diag(t).  The sums run on one thread in row order,
// prices in column order (points, then diagonals).  Rounds work on the list
// of rows that bid.  On return H.pm[j] (j < mc) is the row owning point
// column j, or -1.
// Scratch: H.v = prices (m), H.minv = a column's highest bid (bits), H.key =
// its round-tagged winner, H.u = bids / cheapest net costs (k), H.aw = costs
// of the assigned options (k), H.pm = owners (mc); aux (4 x stride ints) =
// a row's column, its bid column (-2: released), two row lists.
// ---------------------------------------------------------------------------
constexpr int kAuctionRounds = 1 << 24;

// Options of a row are scanned by one warp in chunks of 32, in the kept
// list's order (increasing w); prices are >= 0, so once a chunk's largest w
// exceeds the running second-cheapest net cost no later option can change
// the cheapest (n1, j1) or the second-cheapest n2, and the scan stops.  The
// row's own diagonal is the first option.  Lane states merge by a
// butterfly, so every lane ends with the warp's result.
struct AucBest {
  double n1, w1, n2;
  int j1;
};

__device__ __forceinline__ void auc_take(AucBest& s, double v, int j, double w) {
  if (v < s.n1 || (v == s.n1 && j < s.j1)) {
    s.n2 = s.n1;
    s.n1 = v;
    s.j1 = j;
    s.w1 = w;
  } else if (v < s.n2) {
    s.n2 = v;
  }
}

__device__ __forceinline__ AucBest auc_warp_merge(AucBest s) {
  for (int o = 16; o; o >>= 1) {
    AucBest b;
    b.n1 = __shfl_xor_sync(0xFFFFFFFFu, s.n1, o);
    b.w1 = __shfl_xor_sync(0xFFFFFFFFu, s.w1, o);
    b.n2 = __shfl_xor_sync(0xFFFFFFFFu, s.n2, o);
    b.j1 = __shfl_xor_sync(0xFFFFFFFFu, s.j1, o);
    if (b.n1 < s.n1 || (b.n1 == s.n1 && b.j1 < s.j1)) {
      s.n2 = fmin(s.n1, b.n2);
      s.n1 = b.n1;
      s.j1 = b.j1;
      s.w1 = b.w1;
    } else {
      s.n2 = fmin(s.n2, b.n1);
    }
  }
  return s;
}

template <class Rows>
__device__ __forceinline__ AucBest auction_best(const Rows& R, int r, int mc, const double* __restrict__ diag_t,
                                                const double* price) {
  const double INF = __longlong_as_double(0x7FF0000000000000ll);
  const int lane = threadIdx.x & 31;
  const int n = R.count(r);
  AucBest s{INF, INF, INF, 0x7FFFFFFF};
  if (lane == 0) auc_take(s, __dadd_rn(diag_t[r], price[mc + r]), mc + r, diag_t[r]);
  for (int base = 0; base < n; base += 32) {
    const int c = base + lane;
    double w = 0.0;
    if (c < n) {
      int j;
      R.get(r, c, j, w);
      auc_take(s, __dadd_rn(w, price[j - 1]), j - 1, w);
    }
    const double wlast = __shfl_sync(0xFFFFFFFFu, w, min(31, n - 1 - base));
    const AucBest m = auc_warp_merge(s);
    if (wlast > m.n2) break;
  }
  return auc_warp_merge(s);
}

// Cheapest net cost of row r (all lanes), with the same early stop.
template <class Rows>
__device__ __forceinline__ double auction_min(const Rows& R, int r, int mc, const double* __restrict__ diag_t,
                                              const double* price) {
  const int lane = threadIdx.x & 31;
  const int n = R.count(r);
  double m = __dadd_rn(diag_t[r], price[mc + r]);
  for (int base = 0; base < n; base += 32) {
    const int c = base + lane;
    double w = 0.0, v = m;
    if (c < n) {
      int j;
      R.get(r, c, j, w);
      v = __dadd_rn(w, price[j - 1]);
    }
    for (int o = 16; o; o >>= 1) v = fmin(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    m = fmin(m, v);
    const double wlast = __shfl_sync(0xFFFFFFFFu, w, min(31, n - 1 - base));
    if (wlast > m) break;
  }
  return m;
}

// Cheapest net cost of row r with the tightened prices pt (double bits,
// every one >= 0), all lanes, with the same early stop.
template <class Rows>
__device__ __forceinline__ double auction_min_bits(const Rows& R, int r, int mc, const double* __restrict__ diag_t,
                                                   const unsigned long long* pt, bool l2) {
  const int lane = threadIdx.x & 31;
  const int n = R.count(r);
  auto P = [&](int j) { return __longlong_as_double((long long)(l2 ? __ldcg(pt + j) : pt[j])); };
  double m = __dadd_rn(diag_t[r], P(mc + r));
  for (int base = 0; base < n; base += 32) {
    const int c = base + lane;
    double w = 0.0, v = m;
    if (c < n) {
      int j;
      R.get(r, c, j, w);
      v = __dadd_rn(w, P(j - 1));
    }
    for (int o = 16; o; o >>= 1) v = fmin(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    m = fmin(m, v);
    const double wlast = __shfl_sync(0xFFFFFFFFu, w, min(31, n - 1 - base));
    if (wlast > m) break;
  }
  return m;
}

// One warp: raise pt(j) to u - w(r,j) over row r's options (scatter-max).
template <class Rows>
__device__ __forceinline__ void auction_need(const Rows& R, int r, int mc, const double* __restrict__ diag_t,
                                             double u, unsigned long long* pt) {
  const int lane = threadIdx.x & 31;
  const int n = R.count(r);
  for (int c = lane; c <= n; c += 32) {
    int j;
    double w;
    if (c < n) {
      R.get(r, c, j, w);
      j -= 1;
    } else {
      j = mc + r;
      w = diag_t[r];
    }
    const double need = __dsub_rn(u, w);
    if (need > 0.0) atomicMax(pt + j, (unsigned long long)__double_as_longlong(need));
  }
}

template <class Rows>
__device__ bool auction_solve(int k, int mc, const Rows& R, const double* __restrict__ diag_t, double prec,
                              const Pt* __restrict__ pts, const int32_t* __restrict__ gpts, int npg, HungWork H,
                              int32_t* aux, int stride, int32_t* rounds_out, uint32_t* status) {
  const int m = mc + k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t* rowcol = aux;
  int32_t* bidcol = aux + stride;
  int32_t* lists[2] = {aux + 2 * stride, aux + 3 * stride};
  double* price = H.v;
  unsigned long long* colbid = reinterpret_cast<unsigned long long*>(H.minv);
  unsigned long long* colkey = H.key;
  double* bidval = H.u;
  double* bidw = H.bw;
  double* aw = H.aw;
  int32_t* owner = H.pm;
  __shared__ int s_n[2];
  __shared__ int s_nv;
  __shared__ int s_stop;
  __shared__ double s_chunk[kHT];
  __shared__ double s_eps;
  if (threadIdx.x == 0) {
    s_n[0] = 0;
    s_n[1] = 0;
  }
  for (int j = threadIdx.x; j < m; j += kHT) price[j] = 0.0;
  for (int j = threadIdx.x; j < mc; j += kHT) {
    owner[j] = -1;
    colbid[j] = 0ull;
    colkey[j] = ~0ull;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < k; r += kHT) {
    bidcol[r] = -1;
    if (R.count(r) > 0) {
      rowcol[r] = -1;
      lists[0][atomicAdd(&s_n[0], 1)] = r;
    } else {
      rowcol[r] = mc + r;
      aw[r] = diag_t[r];
    }
  }
  // D = sum of diag(p) in point order; the largest diag(t)
  double dsum = 0.0, cmax = 0.0;
  for (int c0 = 0; c0 < npg; c0 += kHT) {
    int i = c0 + threadIdx.x;
    if (i < npg) s_chunk[threadIdx.x] = cost_diag(pts[gpts[i]].b, pts[gpts[i]].d);
    __syncthreads();
    if (threadIdx.x == 0) {
      int n = min(kHT, npg - c0);
      for (int q = 0; q < n; ++q) dsum = __dadd_rn(dsum, s_chunk[q]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int r = 0; r < k; ++r) cmax = fmax(cmax, diag_t[r]);
    double emin = ldexp(cmax, -40);
    if (!(emin > 0.0)) emin = 2.2250738585072014e-308;  // smallest normal double
    double e = __dmul_rn(cmax, 0.25);
    s_eps = e < emin ? emin : e;
  }
  __syncthreads();
  double eps = s_eps;
  double onep = __dadd_rn(1.0, prec);  // the precision is on sqrt(W2^2)
  onep = __dmul_rn(onep, onep);
  int cur = 0;
  unsigned round = 0;
  int phase = 0, checks = 0;
  for (;; ++phase) {
    if (phase > 0) {
      for (;; ++checks) {  // release the rows that break eps-complementary slackness
        for (int j = threadIdx.x; j < mc; j += kHT)
          if (owner[j] < 0) price[j] = 0.0;
        for (int r = threadIdx.x; r < k; r += kHT)
          if (rowcol[r] != mc + r) price[mc + r] = 0.0;
        if (threadIdx.x == 0) s_nv = 0;
        __syncthreads();
        for (int r = warp; r < k; r += kHT / 32) {
          const int jr = rowcol[r];
          if (jr < 0) continue;
          const double n1 = auction_min(R, r, mc, diag_t, price);
          if (lane == 0 && __dadd_rn(aw[r], price[jr]) > __dadd_rn(n1, eps)) {
            bidcol[r] = -2;
            atomicAdd(&s_nv, 1);
          }
        }
        __syncthreads();
        if (s_nv == 0) break;
        for (int r = threadIdx.x; r < k; r += kHT) {
          if (bidcol[r] != -2) continue;
          bidcol[r] = -1;
          if (rowcol[r] < mc) owner[rowcol[r]] = -1;
          rowcol[r] = -1;
          lists[cur][atomicAdd(&s_n[cur], 1)] = r;
        }
        __syncthreads();
      }
    }
    for (;; ++round) {
      if (round >= (unsigned)kAuctionRounds) {
        if (threadIdx.x == 0) atomicOr(status, kErrRounds);
        return false;
      }
      const int ncur = s_n[cur];
      const int nxt = cur ^ 1;
      if (ncur == 0) break;
      const int32_t* L = lists[cur];
      int32_t* LN = lists[nxt];
      // bids: one warp per listed row
      for (int idx = warp; idx < ncur; idx += kHT / 32) {
        const int r = L[idx];
        const AucBest b = auction_best(R, r, mc, diag_t, price);
        if (lane == 0) {
          double g = __dsub_rn(b.n2, b.n1);
          g = __dadd_rn(g, eps);
          const double bid = __dadd_rn(price[b.j1], g);
          if (b.j1 >= mc) {  // the row's own diagonal: nobody else bids for it
            price[b.j1] = bid;
            rowcol[r] = b.j1;
            aw[r] = b.w1;
          } else {
            bidcol[r] = b.j1;
            bidval[r] = bid;
            bidw[r] = b.w1;
            atomicMax(&colbid[b.j1], (unsigned long long)__double_as_longlong(bid));
          }
        }
      }
      __syncthreads();
      // ties: the lowest row among a column's highest bids
      const unsigned long long tag = (unsigned long long)(0xFFFFFFFFu - round) << 32;
      for (int idx = threadIdx.x; idx < ncur; idx += kHT) {
        const int r = L[idx];
        const int j = bidcol[r];
        if (j >= 0 && colbid[j] == (unsigned long long)__double_as_longlong(bidval[r]))
          atomicMin(&colkey[j], tag | (unsigned)r);
      }
      __syncthreads();
      // winners take their column; losers and displaced rows bid again
      for (int idx = threadIdx.x; idx < ncur; idx += kHT) {
        const int r = L[idx];
        const int j = bidcol[r];
        if (j < 0) continue;
        bidcol[r] = -1;
        if (colkey[j] == (tag | (unsigned)r)) {
          const int old = owner[j];
          if (old >= 0) {
            rowcol[old] = -1;
            LN[atomicAdd(&s_n[nxt], 1)] = old;
          }
          owner[j] = r;
          rowcol[r] = j;
          aw[r] = bidw[r];
          price[j] = bidval[r];
          colbid[j] = 0ull;
        } else {
          LN[atomicAdd(&s_n[nxt], 1)] = r;
        }
      }
      if (threadIdx.x == 0) s_n[cur] = 0;
      __syncthreads();
      cur = nxt;
    }
    // phase end: W, LB and the stop test
    for (int r = warp; r < k; r += kHT / 32) {
      const double n1 = auction_min(R, r, mc, diag_t, price);
      if (lane == 0) bidval[r] = n1;
    }
    __syncthreads();
    // W, U (row order) and P (column order): chunks staged in shared memory,
    // added by one thread in order
    __shared__ double s_w[kHT];
    double W = 0.0, U = 0.0, P = 0.0;
    for (int c0 = 0; c0 < k; c0 += kHT) {
      const int r = c0 + threadIdx.x;
      if (r < k) {
        s_w[threadIdx.x] = aw[r];
        s_chunk[threadIdx.x] = bidval[r];
      }
      __syncthreads();
      if (threadIdx.x == 0)
        for (int i = 0, n = min(kHT, k - c0); i < n; ++i) {
          W = __dadd_rn(W, s_w[i]);
          U = __dadd_rn(U, s_chunk[i]);
        }
      __syncthreads();
    }
    for (int c0 = 0; c0 < m; c0 += kHT) {
      const int j = c0 + threadIdx.x;
      if (j < m) s_chunk[threadIdx.x] = price[j];
      __syncthreads();
      if (threadIdx.x == 0)
        for (int i = 0, n = min(kHT, m - c0); i < n; ++i) P = __dadd_rn(P, s_chunk[i]);
      __syncthreads();
    }
    // a second dual bound: prices down to what the row values u_r (in bidval)
    // need, then the row values up to their new minima (colbid is zero here)
    unsigned long long* pt = colbid;
    for (int r = warp; r < k; r += kHT / 32) auction_need(R, r, mc, diag_t, bidval[r], pt);
    __syncthreads();
    for (int r = warp; r < k; r += kHT / 32) {
      const double u2 = auction_min_bits(R, r, mc, diag_t, pt, false);
      if (lane == 0) bidw[r] = u2;
    }
    __syncthreads();
    double U2 = 0.0, P2 = 0.0;
    for (int c0 = 0; c0 < k; c0 += kHT) {
      const int r = c0 + threadIdx.x;
      if (r < k) s_chunk[threadIdx.x] = bidw[r];
      __syncthreads();
      if (threadIdx.x == 0)
        for (int i = 0, n = min(kHT, k - c0); i < n; ++i) U2 = __dadd_rn(U2, s_chunk[i]);
      __syncthreads();
    }
    for (int c0 = 0; c0 < m; c0 += kHT) {
      const int j = c0 + threadIdx.x;
      if (j < m) s_chunk[threadIdx.x] = __longlong_as_double((long long)pt[j]);
      __syncthreads();
      if (threadIdx.x == 0)
        for (int i = 0, n = min(kHT, m - c0); i < n; ++i) P2 = __dadd_rn(P2, s_chunk[i]);
      __syncthreads();
    }
    for (int j = threadIdx.x; j < m; j += kHT) pt[j] = 0ull;
    if (threadIdx.x == 0) {
      double lb = __dsub_rn(U, P);
      const double lb2 = __dsub_rn(U2, P2);
      if (lb2 > lb) lb = lb2;
      double lhs = __dadd_rn(W, dsum);
      double rhs = __dadd_rn(lb, dsum);
      rhs = __dmul_rn(rhs, onep);
      double emin = ldexp(cmax, -40);
      if (!(emin > 0.0)) emin = 2.2250738585072014e-308;
      int stop = (lhs <= rhs || !(eps > emin)) ? 1 : 0;
      if (!stop) {
        double e = __ddiv_rn(eps, 5.0);
        s_eps = e < emin ? emin : e;
      }
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) break;
    eps = s_eps;
  }
  if (threadIdx.x == 0 && rounds_out) {
    atomicAdd(rounds_out, (int)round);
    atomicAdd(rounds_out + 1, phase + 1);
    atomicAdd(rounds_out + 2, checks);
  }
  __syncthreads();
  return true;
}

__global__ void __launch_bounds__(kHT, 1) k_auction(int k, int mc, const Cand* __restrict__ kept,
                                                 const uint32_t* __restrict__ koff, const uint32_t* __restrict__ nkept,
                                                 const uint32_t* __restrict__ colpos,
                                                 const double* __restrict__ diag_t, double prec,
                                                 const Pt* __restrict__ pts, const int32_t* __restrict__ plist,
                                                 int npg, HungWork H, int32_t* aux, int stride,
                                                 int32_t* __restrict__ col_to_row, int32_t* rounds_out,
                                                 uint32_t* status) {
  if (!auction_solve(k, mc, KeptRows{kept, koff, nkept, colpos}, diag_t, prec, pts, plist, npg, H, aux, stride,
                     rounds_out, status))
    return;
  for (int j = threadIdx.x; j < mc; j += kHT) col_to_row[j] = H.pm[j];
}

// ---------------------------------------------------------------------------
// The same auction over the whole GPU: one cooperative launch of
// co-resident blocks, the steps of auction_solve separated by a grid
// barrier instead of a block barrier, rows and columns spread over every
// warp of the grid.  Identical arithmetic in identical order (the sums still
// run on one thread); a large reduced problem then bids with thousands of
// warps instead of 32.  State shared between blocks is read through L2
// (__ldcg); the barrier (tsf_grid.cuh) gives up after ~2^24 polls, sets
// kErrSpin and the auction returns false on every block.
// ---------------------------------------------------------------------------
constexpr int kGT = 512;        // threads per block of the grid auction
constexpr int kGridMin = 192;   // fewer rows: the single-block auction

struct AucCtl {
  unsigned bar[2];  // arrivals, generation
  int n[2];         // lengths of the two row lists
  int nv;           // rows released by the current check
  int stop;
  int pad[2];
  double eps;
};

template <class Rows>
__device__ __forceinline__ AucBest auction_best_cg(const Rows& R, int r, int mc, const double* __restrict__ diag_t,
                                                   const double* price) {
  const double INF = __longlong_as_double(0x7FF0000000000000ll);
  const int lane = threadIdx.x & 31;
  const int n = R.count(r);
  AucBest s{INF, INF, INF, 0x7FFFFFFF};
  if (lane == 0) auc_take(s, __dadd_rn(diag_t[r], __ldcg(price + mc + r)), mc + r, diag_t[r]);
  for (int base = 0; base < n; base += 32) {
    const int c = base + lane;
    double w = 0.0;
    if (c < n) {
      int j;
      R.get(r, c, j, w);
      auc_take(s, __dadd_rn(w, __ldcg(price + j - 1)), j - 1, w);
    }
    const double wlast = __shfl_sync(0xFFFFFFFFu, w, min(31, n - 1 - base));
    const AucBest m = auc_warp_merge(s);
    if (wlast > m.n2) break;
  }
  return auc_warp_merge(s);
}

template <class Rows>
__device__ __forceinline__ double auction_min_cg(const Rows& R, int r, int mc, const double* __restrict__ diag_t,
                                                 const double* price) {
  const int lane = threadIdx.x & 31;
  const int n = R.count(r);
  double m = __dadd_rn(diag_t[r], __ldcg(price + mc + r));
  for (int base = 0; base < n; base += 32) {
    const int c = base + lane;
    double w = 0.0, v = m;
    if (c < n) {
      int j;
      R.get(r, c, j, w);
      v = __dadd_rn(w, __ldcg(price + j - 1));
    }
    for (int o = 16; o; o >>= 1) v = fmin(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    m = fmin(m, v);
    const double wlast = __shfl_sync(0xFFFFFFFFu, w, min(31, n - 1 - base));
    if (wlast > m) break;
  }
  return m;
}

template <class Rows>
__device__ bool auction_grid(int k, int mc, const Rows& R, const double* __restrict__ diag_t, double prec,
                             const Pt* __restrict__ pts, const int32_t* __restrict__ gpts, int npg, HungWork H,
                             int32_t* aux, int stride, AucCtl* ctl, int32_t* rounds_out, uint32_t* status) {
  const int m = mc + k;
  const unsigned nb = gridDim.x;
  const int lane = threadIdx.x & 31;
  const int gtid = blockIdx.x * kGT + threadIdx.x, gthreads = nb * kGT;
  const int gwarp = gtid >> 5, gwarps = gthreads >> 5;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  int32_t* rowcol = aux;
  int32_t* bidcol = aux + stride;
  int32_t* lists[2] = {aux + 2 * stride, aux + 3 * stride};
  double* price = H.v;
  unsigned long long* colbid = reinterpret_cast<unsigned long long*>(H.minv);
  unsigned long long* colkey = H.key;
  double* bidval = H.u;
  double* bidw = H.bw;
  double* aw = H.aw;
  int32_t* owner = H.pm;
  volatile int* vn = ctl->n;
  __shared__ double s_chunk[kGT];
  __shared__ double s_w[kGT];
  for (int j = gtid; j < m; j += gthreads) price[j] = 0.0;
  for (int j = gtid; j < mc; j += gthreads) {
    owner[j] = -1;
    colbid[j] = 0ull;
    colkey[j] = ~0ull;
  }
  if (!grid_barrier(ctl->bar, nb, status)) return false;
  for (int r = gtid; r < k; r += gthreads) {
    bidcol[r] = -1;
    if (R.count(r) > 0) {
      rowcol[r] = -1;
      lists[0][atomicAdd(&ctl->n[0], 1)] = r;
    } else {
      rowcol[r] = mc + r;
      aw[r] = diag_t[r];
    }
  }
  // D = sum of diag(p) in point order, the largest diag(t), eps: block 0
  double dsum = 0.0, cmax = 0.0;
  if (blockIdx.x == 0) {
    for (int c0 = 0; c0 < npg; c0 += kGT) {
      int i = c0 + threadIdx.x;
      if (i < npg) s_chunk[threadIdx.x] = cost_diag(pts[gpts[i]].b, pts[gpts[i]].d);
      __syncthreads();
      if (threadIdx.x == 0)
        for (int q = 0, n = min(kGT, npg - c0); q < n; ++q) dsum = __dadd_rn(dsum, s_chunk[q]);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      for (int r = 0; r < k; ++r) cmax = fmax(cmax, diag_t[r]);
      double emin = ldexp(cmax, -40);
      if (!(emin > 0.0)) emin = 2.2250738585072014e-308;  // smallest normal double
      double e = __dmul_rn(cmax, 0.25);
      ctl->eps = e < emin ? emin : e;
    }
  }
  if (!grid_barrier(ctl->bar, nb, status)) return false;
  double eps = __ldcg(&ctl->eps);
  double onep = __dadd_rn(1.0, prec);  // the precision is on sqrt(W2^2)
  onep = __dmul_rn(onep, onep);
  int cur = 0;
  unsigned round = 0;
  int phase = 0, checks = 0;
  for (;; ++phase) {
    if (phase > 0) {
      for (;; ++checks) {  // release the rows that break eps-complementary slackness
        for (int j = gtid; j < mc; j += gthreads)
          if (__ldcg(owner + j) < 0) price[j] = 0.0;
        for (int r = gtid; r < k; r += gthreads)
          if (__ldcg(rowcol + r) != mc + r) price[mc + r] = 0.0;
        if (lead) ctl->nv = 0;
        if (!grid_barrier(ctl->bar, nb, status)) return false;
        for (int r = gwarp; r < k; r += gwarps) {
          const int jr = __ldcg(rowcol + r);
          if (jr < 0) continue;
          const double n1 = auction_min_cg(R, r, mc, diag_t, price);
          if (lane == 0 && __dadd_rn(__ldcg(aw + r), __ldcg(price + jr)) > __dadd_rn(n1, eps)) {
            bidcol[r] = -2;
            atomicAdd(&ctl->nv, 1);
          }
        }
        if (!grid_barrier(ctl->bar, nb, status)) return false;
        if (*(volatile int*)&ctl->nv == 0) break;
        for (int r = gtid; r < k; r += gthreads) {
          if (__ldcg(bidcol + r) != -2) continue;
          bidcol[r] = -1;
          const int jr = __ldcg(rowcol + r);
          if (jr < mc) owner[jr] = -1;
          rowcol[r] = -1;
          lists[cur][atomicAdd(&ctl->n[cur], 1)] = r;
        }
        if (!grid_barrier(ctl->bar, nb, status)) return false;
      }
    }
    for (;; ++round) {
      if (round >= (unsigned)kAuctionRounds) {
        if (lead) atomicOr(status, kErrRounds);
        return false;
      }
      const int ncur = vn[cur];
      const int nxt = cur ^ 1;
      if (ncur == 0) break;
      const int32_t* L = lists[cur];
      int32_t* LN = lists[nxt];
      for (int idx = gwarp; idx < ncur; idx += gwarps) {
        const int r = __ldcg(L + idx);
        const AucBest b = auction_best_cg(R, r, mc, diag_t, price);
        if (lane == 0) {
          double g = __dsub_rn(b.n2, b.n1);
          g = __dadd_rn(g, eps);
          const double bid = __dadd_rn(__ldcg(price + b.j1), g);
          if (b.j1 >= mc) {
            price[b.j1] = bid;
            rowcol[r] = b.j1;
            aw[r] = b.w1;
          } else {
            bidcol[r] = b.j1;
            bidval[r] = bid;
            bidw[r] = b.w1;
            atomicMax(&colbid[b.j1], (unsigned long long)__double_as_longlong(bid));
          }
        }
      }
      if (!grid_barrier(ctl->bar, nb, status)) return false;
      const unsigned long long tag = (unsigned long long)(0xFFFFFFFFu - round) << 32;
      for (int idx = gtid; idx < ncur; idx += gthreads) {
        const int r = __ldcg(L + idx);
        const int j = __ldcg(bidcol + r);
        if (j >= 0 && __ldcg(colbid + j) == (unsigned long long)__double_as_longlong(__ldcg(bidval + r)))
          atomicMin(&colkey[j], tag | (unsigned)r);
      }
      if (!grid_barrier(ctl->bar, nb, status)) return false;
      for (int idx = gtid; idx < ncur; idx += gthreads) {
        const int r = __ldcg(L + idx);
        const int j = __ldcg(bidcol + r);
        if (j < 0) continue;
        bidcol[r] = -1;
        if (__ldcg(colkey + j) == (tag | (unsigned)r)) {
          const int old = __ldcg(owner + j);
          if (old >= 0) {
            rowcol[old] = -1;
            LN[atomicAdd(&ctl->n[nxt], 1)] = old;
          }
          owner[j] = r;
          rowcol[r] = j;
          aw[r] = __ldcg(bidw + r);
          price[j] = __ldcg(bidval + r);
          colbid[j] = 0ull;
        } else {
          LN[atomicAdd(&ctl->n[nxt], 1)] = r;
        }
      }
      if (lead) ctl->n[cur] = 0;
      if (!grid_barrier(ctl->bar, nb, status)) return false;
      cur = nxt;
    }
    // phase end: W, LB and the stop test
    for (int r = gwarp; r < k; r += gwarps) {
      const double n1 = auction_min_cg(R, r, mc, diag_t, price);
      if (lane == 0) bidval[r] = n1;
    }
    if (!grid_barrier(ctl->bar, nb, status)) return false;
    // a second dual bound (see auction_solve): colbid is zero here
    unsigned long long* pt = colbid;
    for (int r = gwarp; r < k; r += gwarps) auction_need(R, r, mc, diag_t, __ldcg(bidval + r), pt);
    if (!grid_barrier(ctl->bar, nb, status)) return false;
    for (int r = gwarp; r < k; r += gwarps) {
      const double u2 = auction_min_bits(R, r, mc, diag_t, pt, true);
      if (lane == 0) bidw[r] = u2;
    }
    if (!grid_barrier(ctl->bar, nb, status)) return false;
    if (blockIdx.x == 0) {
      double W = 0.0, U = 0.0, P = 0.0, U2 = 0.0, P2 = 0.0;
      for (int c0 = 0; c0 < k; c0 += kGT) {
        const int r = c0 + threadIdx.x;
        if (r < k) {
          s_w[threadIdx.x] = __ldcg(aw + r);
          s_chunk[threadIdx.x] = __ldcg(bidval + r);
        }
        __syncthreads();
        if (threadIdx.x == 0)
          for (int i = 0, n = min(kGT, k - c0); i < n; ++i) {
            W = __dadd_rn(W, s_w[i]);
            U = __dadd_rn(U, s_chunk[i]);
          }
        __syncthreads();
      }
      for (int c0 = 0; c0 < m; c0 += kGT) {
        const int j = c0 + threadIdx.x;
        if (j < m) s_chunk[threadIdx.x] = __ldcg(price + j);
        __syncthreads();
        if (threadIdx.x == 0)
          for (int i = 0, n = min(kGT, m - c0); i < n; ++i) P = __dadd_rn(P, s_chunk[i]);
        __syncthreads();
      }
      for (int c0 = 0; c0 < k; c0 += kGT) {
        const int r = c0 + threadIdx.x;
        if (r < k) s_chunk[threadIdx.x] = __ldcg(bidw + r);
        __syncthreads();
        if (threadIdx.x == 0)
          for (int i = 0, n = min(kGT, k - c0); i < n; ++i) U2 = __dadd_rn(U2, s_chunk[i]);
        __syncthreads();
      }
      for (int c0 = 0; c0 < m; c0 += kGT) {
        const int j = c0 + threadIdx.x;
        if (j < m) s_chunk[threadIdx.x] = __longlong_as_double((long long)__ldcg(pt + j));
        __syncthreads();
        if (threadIdx.x == 0)
          for (int i = 0, n = min(kGT, m - c0); i < n; ++i) P2 = __dadd_rn(P2, s_chunk[i]);
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        double lb = __dsub_rn(U, P);
        const double lb2 = __dsub_rn(U2, P2);
        if (lb2 > lb) lb = lb2;
        double lhs = __dadd_rn(W, dsum);
        double rhs = __dadd_rn(lb, dsum);
        rhs = __dmul_rn(rhs, onep);
        double emin = ldexp(cmax, -40);
        if (!(emin > 0.0)) emin = 2.2250738585072014e-308;
        int stop = (lhs <= rhs || !(eps > emin)) ? 1 : 0;
        if (!stop) {
          double e = __ddiv_rn(eps, 5.0);
          ctl->eps = e < emin ? emin : e;
        }
        ctl->stop = stop;
      }
    }
    if (!grid_barrier(ctl->bar, nb, status)) return false;
    if (*(volatile int*)&ctl->stop) break;
    eps = __ldcg(&ctl->eps);
    // zero again before the next phase's bids (a barrier comes first)
    for (int j = gtid; j < m; j += gthreads) pt[j] = 0ull;
  }
  if (lead && rounds_out) {
    atomicAdd(rounds_out, (int)round);
    atomicAdd(rounds_out + 1, phase + 1);
    atomicAdd(rounds_out + 2, checks);
  }
  return grid_barrier(ctl->bar, nb, status);
}

// Group g of the fused path, when it has at least kGridMin free targets (the
// single-block k_asg_solve prepared its columns and left it to this launch).
__global__ void __launch_bounds__(kGT) k_auction_grid_group(AsgDev A, Pt* __restrict__ pts, int g, double prec,
                                                            AucCtl* ctl, uint32_t* status) {
  if (A.counts[8]) return;
  // an earlier group's launch gave up at a barrier: the call already fails
  // with a timeout, so later groups do not spend their own barrier limits
  if (*static_cast<volatile uint32_t*>(status) & kErrSpin) return;
  const int npg = A.counts[g], k = A.counts[4 + g];
  if (k < kGridMin || npg == 0) return;
  int pbase = 0, tbase = 0, wbase = 0;
  for (int gg = 0; gg < g; ++gg) {
    pbase += A.counts[gg];
    tbase += A.counts[4 + gg];
    wbase += A.counts[gg] + A.counts[4 + gg] + 2;
  }
  const int mc = A.counts[13 + g];
  HungWork H;
  H.u = A.H.u + wbase;
  H.v = A.H.v + wbase;
  H.minv = A.H.minv + wbase;
  H.list = A.H.list + wbase;
  H.pm = A.H.pm + wbase;
  H.way = A.H.way + wbase;
  H.used = A.H.used + wbase;
  H.key = A.H.key + wbase;
  H.aw = A.H.aw + wbase;
  H.bw = A.H.bw + wbase;
  const int wg = npg + k + 2;
  if (!auction_grid(k, mc, KeptRows{A.kept, A.kept_off + tbase, A.nkept + tbase, A.colpos + pbase},
                    A.diag_t + tbase, prec, pts, A.plist + pbase, npg, H, A.aux + 4 * wbase, wg, ctl + g,
                    A.counts + 10, status))
    return;
  for (int j = blockIdx.x * kGT + threadIdx.x; j < mc; j += gridDim.x * kGT) {
    const int r = __ldcg(H.pm + j);
    if (r >= 0) pts[A.plist[pbase + A.col_point[wbase + j]]].tgt = A.tlist[tbase + r];
  }
}

// The group-by-group path's problem, over the whole GPU.
__global__ void __launch_bounds__(kGT) k_auction_grid(int k, int mc, const Cand* __restrict__ kept,
                                                      const uint32_t* __restrict__ koff,
                                                      const uint32_t* __restrict__ nkept,
                                                      const uint32_t* __restrict__ colpos,
                                                      const double* __restrict__ diag_t, double prec,
                                                      const Pt* __restrict__ pts, const int32_t* __restrict__ plist,
                                                      int npg, HungWork H, int32_t* aux, int stride, AucCtl* ctl,
                                                      int32_t* __restrict__ col_to_row, int32_t* rounds_out,
                                                      uint32_t* status) {
  if (!auction_grid(k, mc, KeptRows{kept, koff, nkept, colpos}, diag_t, prec, pts, plist, npg, H, aux, stride, ctl,
                    rounds_out, status))
    return;
  for (int j = blockIdx.x * kGT + threadIdx.x; j < mc; j += gridDim.x * kGT) col_to_row[j] = __ldcg(H.pm + j);
}

__global__ void k_colpos(int npg, const uint32_t* __restrict__ is_col, const uint32_t* __restrict__ pos,
                         uint32_t* __restrict__ colpos, int32_t* __restrict__ col_point) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < npg) {
    colpos[i] = pos[i];
    if (is_col[i]) col_point[pos[i]] = i;
  }
}

__global__ void k_diag_t(int k, const int32_t* __restrict__ tlist, const Tg* __restrict__ T, double* __restrict__ dt) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < k) dt[t] = cost_diag(T[tlist[t]].b, T[tlist[t]].d);
}

__global__ void k_apply_assignment(int mc, const int32_t* __restrict__ col_to_row, const int32_t* __restrict__ col_point,
                                   const int32_t* __restrict__ plist, const int32_t* __restrict__ tlist,
                                   Pt* __restrict__ pts) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < mc) {
    int r = col_to_row[j];
    if (r >= 0) pts[plist[col_point[j]]].tgt = tlist[r];
  }
}

__global__ void k_essential(int npg, const int32_t* __restrict__ plist, int k, const int32_t* __restrict__ tlist,
                            Pt* __restrict__ pts) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < npg && i < k) pts[plist[i]].tgt = tlist[i];
}

static uint32_t read_tail(const uint32_t* flag, const uint32_t* pos, int n, cudaStream_t st) {
  uint32_t tail[2] = {0, 0};
  if (n == 0) return 0;
  cudaMemcpyAsync(&tail[0], pos + n - 1, 4, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&tail[1], flag + n - 1, 4, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return tail[0] + tail[1];
}

// ---------------------------------------------------------------------------
// Reduced assignment without host round-trips (used when every target's
// candidate list fits a shared-memory tile; otherwise `assign_groups` runs).
// ---------------------------------------------------------------------------
constexpr int kCandTile = 2048;



// Stable partition of the non-still points and the free targets by group
// (finite dimension 0/1/2, essential = 3) over many blocks.  Items are the np
// points, then the nt targets; group 0..3 for a non-still point, 4..7 for a
// free target.  k_part_count counts per block and group,
// k_part_scan turns the counts into output offsets (and the group sizes),
// k_part_scatter writes every item in its block's order, k_part_essential
// matches the essential class in order.
constexpr int kPartT = 1024;

__device__ __forceinline__ int part_group(int i, int np, const Pt* __restrict__ pts, int nt, const Tg* __restrict__ T,
                                          const uint8_t* __restrict__ taken) {
  if (i < np) return pts[i].still ? -1 : (pts[i].ess ? 3 : pts[i].dim);
  const int t = i - np;
  if (t < nt) return taken[t] ? -1 : 4 + (T[t].ess ? 3 : T[t].dim);
  return -1;
}

__global__ void __launch_bounds__(kPartT) k_part_count(int np, const Pt* __restrict__ pts, int nt,
                                                       const Tg* __restrict__ T, const uint8_t* __restrict__ taken,
                                                       int32_t* __restrict__ bc) {
  __shared__ int c[8];
  if (threadIdx.x < 8) c[threadIdx.x] = 0;
  __syncthreads();
  const int g = part_group(blockIdx.x * kPartT + threadIdx.x, np, pts, nt, T, taken);
  const int lane = threadIdx.x & 31;
  for (int gg = 0; gg < 8; ++gg) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, g == gg);
    if (lane == 0 && m) atomicAdd(&c[gg], __popc(m));
  }
  __syncthreads();
  if (threadIdx.x < 8) bc[blockIdx.x * 8 + threadIdx.x] = c[threadIdx.x];
}

__global__ void __launch_bounds__(kPartT) k_part_scan(int nblk, int32_t* __restrict__ bc, AsgDev A) {
  __shared__ int sw[kPartT / 32 + 1];
  __shared__ int tot[8];
  const int per = (nblk + kPartT - 1) / kPartT;
  const int b0 = threadIdx.x * per, b1 = min(nblk, b0 + per);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int g = 0; g < 8; ++g) {
    int v = 0;
    for (int b = b0; b < b1; ++b) v += bc[b * 8 + g];
    int inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) sw[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      const int x = sw[lane];
      int xi = x;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, xi, o);
        if (lane >= o) xi += t;
      }
      sw[lane] = xi - x;
      if (lane == 31) tot[g] = xi;
    }
    __syncthreads();
    int run = sw[wid] + inc - v;
    for (int b = b0; b < b1; ++b) {
      const int c = bc[b * 8 + g];
      bc[b * 8 + g] = run;  // offset inside the group, added to the group base below
      run += c;
    }
    __syncthreads();
  }
  // group bases: points 0..3 in plist, targets 4..7 in tlist
  __shared__ int base[8];
  if (threadIdx.x == 0) {
    int b = 0, c = 0;
    for (int g = 0; g < 4; ++g) {
      base[g] = b;
      b += tot[g];
      base[4 + g] = c;
      c += tot[4 + g];
      A.counts[g] = tot[g];
      A.counts[4 + g] = tot[4 + g];
    }
    A.counts[8] = 0;
    A.counts[9] = 0;
    A.counts[10] = 0;  // auction rounds, phases, release passes
    A.counts[11] = 0;
    A.counts[12] = 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nblk * 8; i += kPartT) bc[i] += base[i & 7];
}

__global__ void __launch_bounds__(kPartT) k_part_scatter(int np, const Pt* __restrict__ pts, int nt,
                                                         const Tg* __restrict__ T, const uint8_t* __restrict__ taken,
                                                         const int32_t* __restrict__ bc, AsgDev A) {
  __shared__ int wc[kPartT / 32][8];
  const int i = blockIdx.x * kPartT + threadIdx.x;
  const int g = part_group(i, np, pts, nt, T, taken);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int myoff = 0;
  for (int gg = 0; gg < 8; ++gg) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, g == gg);
    if (lane == 0) wc[w][gg] = __popc(m);
    if (g == gg) myoff = __popc(m & ((1u << lane) - 1u));
  }
  __syncthreads();
  if (g >= 0) {
    int o = bc[blockIdx.x * 8 + g] + myoff;
    for (int ww = 0; ww < w; ++ww) o += wc[ww][g];
    if (g < 4) A.plist[o] = i;
    else A.tlist[o] = i - np;
  }
}

__global__ void k_part_essential(AsgDev A, Pt* __restrict__ pw) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int b3 = A.counts[0] + A.counts[1] + A.counts[2], b7 = A.counts[4] + A.counts[5] + A.counts[6];
  const int n3 = min(A.counts[3], A.counts[7]);
  for (int i = 0; i < n3; ++i) pw[A.plist[b3 + i]].tgt = A.tlist[b7 + i];
}

__device__ __forceinline__ void group_of_target(const int32_t* counts, int t, int& g, int& local, int& pbase,
                                                int& tbase) {
  int tb = 0, pb = 0;
  g = -1;
  for (int gg = 0; gg < 3; ++gg) {
    int k = counts[4 + gg];
    if (t < tb + k) {
      g = gg;
      local = t - tb;
      tbase = tb;
      pbase = pb;
      return;
    }
    tb += k;
    pb += counts[gg];
  }
}

// Bitonic sort of n (w, point) pairs in shared memory by (w, point),
// ascending; entries from n up to the next power of two are padding.
__device__ void cand_sort(double* sw, int* sp, int n) {
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  for (int i = n + threadIdx.x; i < n2; i += blockDim.x) {
    sw[i] = __longlong_as_double(0x7FF0000000000000ll);
    sp[i] = 0x7FFFFFFF;
  }
  __syncthreads();
  for (int size = 2; size <= n2; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        int j = i ^ stride;
        if (j > i) {
          bool up = (i & size) == 0;
          bool gt = sw[i] > sw[j] || (sw[i] == sw[j] && sp[i] > sp[j]);
          if (gt == up) {
            double tw = sw[i];
            sw[i] = sw[j];
            sw[j] = tw;
            int tp = sp[i];
            sp[i] = sp[j];
            sp[j] = tp;
          }
        }
      }
      __syncthreads();
    }
}

// one block per free finite target: its k cheapest candidates p (w(p,t) <
// diag(t), ordered by (w, point index)).  Points are scanned in chunks of
// the block size in increasing index; whenever the shared buffer could
// overflow, it is sorted and cut to the k cheapest, whose largest (w, p)
// becomes the bar a later point must beat (later points have larger
// indices, so w below the bar's w).  Groups with more than kCandTile - 512
// free targets leave the problem to the general path.
__global__ void __launch_bounds__(512) k_asg_candidates(const Pt* __restrict__ pts, const Tg* __restrict__ T,
                                                        AsgDev A) {
  __shared__ double sw[kCandTile];
  __shared__ int sp[kCandTile];
  __shared__ int fill;
  __shared__ double bar;
  int g, local, pbase, tbase;
  group_of_target(A.counts, blockIdx.x, g, local, pbase, tbase);
  if (g < 0) return;
  int npg = A.counts[g], k = A.counts[4 + g];
  if (k > kCandTile - 512) {
    if (threadIdx.x == 0) A.counts[8] = 1;  // the general path takes over
    return;
  }
  const Tg tg = T[A.tlist[tbase + local]];
  const double dt = cost_diag(tg.b, tg.d);
  if (threadIdx.x == 0) {
    fill = 0;
    bar = dt;
  }
  __syncthreads();
  for (int base = 0; base < npg; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const double b = bar;
    if (i < npg) {
      const Pt& p = pts[A.plist[pbase + i]];
      const double w = __dsub_rn(cost_pt(p.b, p.d, tg.b, tg.d), cost_diag(p.b, p.d));
      if (w < b) {
        const int s = atomicAdd(&fill, 1);
        sw[s] = w;
        sp[s] = i;
      }
    }
    __syncthreads();
    const int n = fill;
    __syncthreads();  // every thread has read fill before the next chunk appends
    if (n > kCandTile - (int)blockDim.x && base + (int)blockDim.x < npg) {
      cand_sort(sw, sp, n);
      if (threadIdx.x == 0) {
        fill = min(n, k);
        if (n >= k) bar = sw[k - 1];
      }
      __syncthreads();
    }
  }
  const int n = fill;
  cand_sort(sw, sp, n);
  int keep = min(n, k);
  __shared__ uint32_t off;
  if (threadIdx.x == 0) {
    off = (uint32_t)atomicAdd(&A.counts[9], keep);
    A.kept_off[tbase + local] = off;
    A.nkept[tbase + local] = (uint32_t)keep;
    if ((int)off + keep > A.cap_kept) A.counts[8] = 1;
  }
  __syncthreads();
  if ((int)off + keep > A.cap_kept) return;
  for (int i = threadIdx.x; i < keep; i += blockDim.x) {
    Cand c;
    c.w = sw[i];
    c.p = sp[i];
    c.t = local;
    A.kept[off + i] = c;
    A.is_col[pbase + sp[i]] = 1u;
  }
}

// one block per finite group: column map (candidate points in point order,
// then one private diagonal column per target) and the shortest augmenting
// path solve, exactly as k_hungarian
// AUCTION: the auction (prec > 0) instead of the exact search; two kernels so
// that neither carries the other's registers.
template <bool AUCTION>
__global__ void __launch_bounds__(kHT, 1) k_asg_solve(AsgDev A, Pt* __restrict__ pts, const Tg* __restrict__ T,
                                                      double prec, uint32_t* status) {
  const int g = blockIdx.x;
  if (A.counts[8]) return;
  int npg = A.counts[g], k = A.counts[4 + g];
  if (k == 0 || npg == 0) return;
  int pbase = 0, tbase = 0, wbase = 0;
  for (int gg = 0; gg < g; ++gg) {
    pbase += A.counts[gg];
    tbase += A.counts[4 + gg];
    wbase += A.counts[gg] + A.counts[4 + gg] + 2;
  }
  // column positions of the candidate points of this group
  __shared__ int s_mc;
  {
    int run = 0;
    for (int b0 = 0; b0 < npg; b0 += kHT) {
      int i = b0 + threadIdx.x;
      int f = (i < npg && A.is_col[pbase + i]) ? 1 : 0;
      int tot;
      int ex = block_exscan_int1024(f, tot);
      if (i < npg) A.colpos[pbase + i] = (uint32_t)(run + ex);
      if (f) A.col_point[wbase + run + ex] = i;
      run += tot;
    }
    if (threadIdx.x == 0) s_mc = run;
    __syncthreads();
  }
  int mc = s_mc;
  HungWork H;
  H.u = A.H.u + wbase;
  H.v = A.H.v + wbase;
  H.minv = A.H.minv + wbase;
  H.list = A.H.list + wbase;
  H.pm = A.H.pm + wbase;
  H.way = A.H.way + wbase;
  H.used = A.H.used + wbase;
  H.key = A.H.key + wbase;
  H.aw = A.H.aw + wbase;
  H.bw = A.H.bw + wbase;
  double* diag_t = A.diag_t + tbase;
  for (int t = threadIdx.x; t < k; t += kHT) diag_t[t] = cost_diag(T[A.tlist[tbase + t]].b, T[A.tlist[tbase + t]].d);
  __syncthreads();
  if constexpr (AUCTION) {
    if (k >= kGridMin) {  // k_auction_grid_group solves it over the whole GPU
      if (threadIdx.x == 0) A.counts[13 + g] = mc;
      return;
    }
    const int wg = npg + k + 2;
    if (!auction_solve(k, mc, KeptRows{A.kept, A.kept_off + tbase, A.nkept + tbase, A.colpos + pbase}, diag_t, prec,
                       pts, A.plist + pbase, npg, H, A.aux + 4 * wbase, wg, A.counts + 10, status))
      return;
    for (int j = threadIdx.x; j < mc; j += kHT) {
      int r = H.pm[j];
      if (r >= 0) pts[A.plist[pbase + A.col_point[wbase + j]]].tgt = A.tlist[tbase + r];
    }
    return;
  } else {
  if (!sap_solve(k, mc, KeptRows{A.kept, A.kept_off + tbase, A.nkept + tbase, A.colpos + pbase}, diag_t, H, status))
    return;
  for (int j = 1 + threadIdx.x; j <= mc; j += kHT) {
    int r = H.pm[j] - 1;
    if (r >= 0) pts[A.plist[pbase + A.col_point[wbase + j - 1]]].tgt = A.tlist[tbase + r];
  }
  }
}

int assign_groups(int np, Pt* pts, int nt, const Tg* T, double prec, SolverBufs& B, uint32_t* status,
                  AssignStats* as, cudaStream_t st);

// Assignment phi*_j.  `ref` is the previous diagram (or the targets at j = 0,
// each assigned to itself).  Returns 0, or a negative value when a scratch
// buffer is too small (the caller grows it and retries).
int assign(int np, Pt* pts, int nr, const Pt* ref, int nt, const Tg* T, double prec, SolverBufs& B,
           uint32_t* status, AssignStats* as, cudaStream_t st) {
  // 1) still pairs
  cudaMemsetAsync(B.taken, 0, (size_t)max(nt, 1), st);
  const bool radix = B.ids30 && np <= B.cap_rsort && nr <= B.cap_rsort;
  int32_t* ck = radix ? radix_sort64(np, nullptr, KeyBits{pts}, B.rsort, B.idxB, B.idxA, status, st)
                      : merge_sort(np, B.idxA, B.idxB, KeyLess{pts}, st);
  int32_t* rk = B.idxC;
  if (nr > 0) {
    // the reference is the previous assignment's points: their key order
    // was kept (the keys of an array do not change once it is built)
    if (ref == B.keyord_for && nr == B.keyord_n) rk = B.keyord;
    else if (radix) rk = radix_sort64(nr, nullptr, KeyBits{ref}, B.rsort, B.idxD, B.idxC, status, st);
    else rk = merge_sort(nr, B.idxC, B.idxD, KeyLess{ref}, st);
  }
  k_still<<<(np + 255) / 256, 256, 0, st>>>(np, pts, ck, nr, ref, rk, B.tmp_pts, B.taken); note_launch();
  cudaMemcpyAsync(pts, B.tmp_pts, sizeof(Pt) * (size_t)np, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(B.keyord, ck, sizeof(int32_t) * (size_t)np, cudaMemcpyDeviceToDevice, st);
  B.keyord_for = pts;
  B.keyord_n = np;
  // 2) reduced problems: three launches, no host round-trip; the general
  // group-by-group path runs only when a candidate list overflows its tile
  cudaMemsetAsync(B.A.is_col, 0, sizeof(uint32_t) * (size_t)np, st);
  {
    const int nblk = max(1, (np + nt + kPartT - 1) / kPartT);
    int32_t* bc = reinterpret_cast<int32_t*>(B.u32a);  // 8 counters per block
    k_part_count<<<nblk, kPartT, 0, st>>>(np, pts, nt, T, B.taken, bc); note_launch();
    k_part_scan<<<1, kPartT, 0, st>>>(nblk, bc, B.A); note_launch();
    k_part_scatter<<<nblk, kPartT, 0, st>>>(np, pts, nt, T, B.taken, bc, B.A); note_launch();
    k_part_essential<<<1, 32, 0, st>>>(B.A, pts); note_launch();
  }
  k_asg_candidates<<<max(nt, 1), 512, 0, st>>>(pts, T, B.A); note_launch();
  if (prec > 0.0) {
    k_asg_solve<true><<<3, kHT, 0, st>>>(B.A, pts, T, prec, status);
  } else {
    k_asg_solve<false><<<3, kHT, 0, st>>>(B.A, pts, T, prec, status);
  }
  note_launch();
  if (prec > 0.0) {  // groups with many free targets: the auction over the whole GPU
    const int nb = cooperative_blocks((const void*)k_auction_grid_group, kGT);
    if (nb == 0) return -4;
    cudaMemsetAsync(B.actl, 0, 3 * sizeof(AucCtl), st);
    for (int g = 0; g < 3; ++g) {
      AsgDev A = B.A;
      Pt* p = pts;
      int gg = g;
      double pr = prec;
      AucCtl* c = static_cast<AucCtl*>(B.actl);
      void* args[] = {&A, &p, &gg, &pr, &c, &status};
      if (cooperative_launch((const void*)k_auction_grid_group, dim3(nb), dim3(kGT), args, st) != cudaSuccess)
        return -4;
    }
  }
  int32_t hc[13];
  cudaMemcpyAsync(hc, B.A.counts, sizeof(hc), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&as->status, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  as->status_valid = !hc[8];
  as->rounds = hc[10];
  as->phases = hc[11];
  as->checks = hc[12];
  for (int g = 0; g < 4; ++g) as->k[g] = hc[4 + g];
  if (!hc[8]) return 0;
  return assign_groups(np, pts, nt, T, prec, B, status, as, st);
}

// General path: group by group with host-sized buffers.
int assign_groups(int np, Pt* pts, int nt, const Tg* T, double prec, SolverBufs& B, uint32_t* status,
                  AssignStats* as, cudaStream_t st) {
  // 2) reduced problems, group by group
  as->k[0] = as->k[1] = as->k[2] = as->k[3] = 0;
  for (int g = 0; g < 4; ++g) {
    k_group_flags<<<(np + 255) / 256, 256, 0, st>>>(np, pts, g, B.u32a); note_launch();
    exclusive_scan_u32(B.u32a, B.u32b, np, B.u32c, st);
    int npg = (int)read_tail(B.u32a, B.u32b, np, st);
    k_compact<<<(np + 255) / 256, 256, 0, st>>>(np, B.u32a, B.u32b, B.plist); note_launch();
    int k = 0;
    if (nt > 0) {
      k_tgroup_flags<<<(nt + 255) / 256, 256, 0, st>>>(nt, T, B.taken, g, B.u32a); note_launch();
      exclusive_scan_u32(B.u32a, B.u32b, nt, B.u32c, st);
      k = (int)read_tail(B.u32a, B.u32b, nt, st);
      k_compact<<<(nt + 255) / 256, 256, 0, st>>>(nt, B.u32a, B.u32b, B.tlist); note_launch();
    }
    as->k[g] = k;
    if (k == 0 || npg == 0) continue;
    if (g == 3) {
      k_essential<<<(npg + 255) / 256, 256, 0, st>>>(npg, B.plist, k, B.tlist, pts); note_launch();
      continue;
    }
    if (k > B.cap_k) return -1;
    k_cand_count<<<k, 256, 0, st>>>(npg, B.plist, pts, k, B.tlist, T, B.u32a); note_launch();
    exclusive_scan_u32(B.u32a, B.u32b, k, B.u32c, st);
    int nc = (int)read_tail(B.u32a, B.u32b, k, st);
    if (nc > B.cap_cand) return -2;
    if (nc == 0) continue;
    k_cand_fill<<<k, 256, 0, st>>>(npg, B.plist, pts, k, B.tlist, T, B.u32b, B.cands); note_launch();
    int32_t* ci = merge_sort(nc, B.idxC, B.idxD, CandLess{B.cands}, st);
    cudaMemsetAsync(B.is_col, 0, sizeof(uint32_t) * (size_t)npg, st);
    cudaMemsetAsync(B.nkept, 0, sizeof(uint32_t) * (size_t)k, st);
    k_cand_keep<<<(nc + 255) / 256, 256, 0, st>>>(nc, ci, B.cands, B.u32b, k, B.is_col, B.kept, B.nkept); note_launch();
    exclusive_scan_u32(B.is_col, B.colpos, npg, B.u32c, st);
    int mc = (int)read_tail(B.is_col, B.colpos, npg, st);
    if (mc + k + 1 > B.cap_cols) return -3;
    k_colpos<<<(npg + 255) / 256, 256, 0, st>>>(npg, B.is_col, B.colpos, B.colpos, B.col_point); note_launch();
    k_diag_t<<<(k + 255) / 256, 256, 0, st>>>(k, B.tlist, T, B.diag_t); note_launch();
    if (prec > 0.0 && k >= kGridMin) {
      const int nb = cooperative_blocks((const void*)k_auction_grid, kGT);
      if (nb == 0) return -4;
      cudaMemsetAsync(B.actl, 0, sizeof(AucCtl), st);
      const Cand* kept = B.kept;
      const uint32_t *koff = B.u32b, *nk = B.nkept, *cp = B.colpos;
      const double* dt = B.diag_t;
      const Pt* cpts = pts;
      const int32_t* pl = B.plist;
      HungWork H = B.H;
      int32_t* aux = B.aux;
      int stride = B.cap_cols + 1;
      AucCtl* c = static_cast<AucCtl*>(B.actl);
      int32_t* ctr = B.col_to_row;
      int32_t* ro = B.A.counts + 10;
      int kk = k, mm = mc, nn = npg;
      double pr = prec;
      void* args[] = {&kk, &mm, &kept, &koff, &nk, &cp, &dt, &pr, &cpts, &pl, &nn, &H, &aux, &stride, &c, &ctr, &ro,
                      &status};
      if (cooperative_launch((const void*)k_auction_grid, dim3(nb), dim3(kGT), args, st) != cudaSuccess) return -4;
    } else if (prec > 0.0) {
      k_auction<<<1, kHT, 0, st>>>(k, mc, B.kept, B.u32b, B.nkept, B.colpos, B.diag_t, prec, pts, B.plist, npg, B.H,
                                   B.aux, B.cap_cols + 1, B.col_to_row, B.A.counts + 10, status); note_launch();
    } else {
      k_hungarian<<<1, kHT, 0, st>>>(k, mc, B.kept, B.u32b, B.nkept, B.colpos, B.diag_t, B.H, B.col_to_row, status); note_launch();
    }
    k_apply_assignment<<<(mc + 255) / 256, 256, 0, st>>>(mc, B.col_to_row, B.col_point, B.plist, B.tlist, pts); note_launch();
  }
  if (prec > 0.0) {  // rounds of the fused attempt plus these
    int32_t r[3] = {0, 0, 0};
    cudaMemcpyAsync(r, B.A.counts + 10, sizeof(r), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    as->rounds = r[0];
    as->phases = r[1];
    as->checks = r[2];
  }
  return 0;
}

// ---------------------------------------------------------------------------
// loss (Eq. 2) and stop counters
// ---------------------------------------------------------------------------
__global__ void k_loss_terms(int np, const Pt* __restrict__ pts, int nt, const Tg* __restrict__ T,
                             float cancel_eps, double* __restrict__ terms, uint8_t* __restrict__ tused,
                             unsigned long long* __restrict__ counters) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < np) {
    const Pt& p = pts[i];
    double c;
    if (p.tgt >= 0) {
      c = cost_pt(p.b, p.d, T[p.tgt].b, T[p.tgt].d);
      tused[p.tgt] = 1;
      if (!p.still) atomicAdd(&counters[2], 1ull);
    } else {
      c = cost_diag(p.b, p.d);
      if (__fsub_rn(p.d, p.b) > cancel_eps) atomicAdd(&counters[0], 1ull);
    }
    if (p.still) atomicAdd(&counters[1], 1ull);
    terms[i] = c;
  }
}
__global__ void k_loss_tterms(int np, int nt, const Tg* __restrict__ T, const uint8_t* __restrict__ tused,
                              double* __restrict__ terms) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nt) terms[np + t] = tused[t] ? 0.0 : cost_diag(T[t].b, T[t].d);
}
// deterministic pairwise sum (fixed tree), one block
__global__ void k_sum(int n, const double* __restrict__ terms, double* __restrict__ out) {
  __shared__ double s[1024];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 1024) acc = __dadd_rn(acc, terms[i]);
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 512; w; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] = __dadd_rn(s[threadIdx.x], s[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

void loss_and_counts(int np, const Pt* pts, int nt, const Tg* T, float cancel_eps, SolverBufs& B, double* h_loss,
                     unsigned long long* h_counts, cudaStream_t st) {
  cudaMemsetAsync(B.counters, 0, sizeof(unsigned long long) * 4, st);
  cudaMemsetAsync(B.taken, 0, (size_t)max(nt, 1), st);
  if (np > 0)
    k_loss_terms<<<(np + 255) / 256, 256, 0, st>>>(np, pts, nt, T, cancel_eps, B.terms, B.taken, B.counters); note_launch();
  if (nt > 0) k_loss_tterms<<<(nt + 255) / 256, 256, 0, st>>>(np, nt, T, B.taken, B.terms); note_launch();
  k_sum<<<1, 1024, 0, st>>>(np + nt, B.terms, B.dsum); note_launch();
  cudaMemcpyAsync(h_loss, B.dsum, sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(h_counts, B.counters, sizeof(unsigned long long) * 4, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
}

// ---------------------------------------------------------------------------
// gradient step (Section 4.1)
// ---------------------------------------------------------------------------
__global__ void k_contrib(int np, const Pt* __restrict__ pts, const Tg* __restrict__ T, float alpha_b, float alpha_d,
                          Contrib* __restrict__ C, int* __restrict__ count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const Pt& p = pts[i];
  float tb, td;
  if (p.tgt >= 0) {
    tb = T[p.tgt].b;
    td = T[p.tgt].d;
  } else {
    float m = __fmul_rn(__fadd_rn(p.b, p.d), 0.5f);
    tb = m;
    td = m;
  }
  float gb = __fmul_rn(2.0f, __fsub_rn(p.b, tb));
  float cb = __fmul_rn(alpha_b, gb);
  int k = atomicAdd(count, p.ess ? 1 : 2);
  C[k].v = p.vb;
  C[k].key = value_key(cb);
  C[k].c = cb;
  if (!p.ess) {
    float gd = __fmul_rn(2.0f, __fsub_rn(p.d, td));
    float cd = __fmul_rn(alpha_d, gd);
    C[k + 1].v = p.vd;
    C[k + 1].key = value_key(cd);
    C[k + 1].c = cd;
  }
}

struct ContribLess {
  const Contrib* c;
  __device__ unsigned long long key(int i) const { return ((unsigned long long)c[i].v << 32) | c[i].key; }
  __device__ bool operator()(int a, int b) const {
    const Contrib& x = c[a];
    const Contrib& y = c[b];
    if (x.v != y.v) return x.v < y.v;
    return x.key < y.key;
  }
};

struct ContribBits {  // ContribLess as one 64-bit key
  const Contrib* c;
  __device__ unsigned long long operator()(int i) const { return ((unsigned long long)c[i].v << 32) | c[i].key; }
};

// one thread per vertex segment: acc = +0, acc += c in increasing value order
__global__ void k_apply_step(int nc, const int* __restrict__ nc_dev, const int32_t* __restrict__ idx,
                             const Contrib* __restrict__ C, float* __restrict__ f, uint32_t* __restrict__ upd,
                             unsigned long long* __restrict__ nupd) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (nc_dev) nc = min(*nc_dev, nc);
  if (r >= nc) return;
  uint32_t v = C[idx[r]].v;
  if (r > 0 && C[idx[r - 1]].v == v) return;
  float acc = 0.0f;
  for (int s = r; s < nc && C[idx[s]].v == v; ++s) acc = __fadd_rn(acc, C[idx[s]].c);
  float old = f[v];
  float nw = __fsub_rn(old, acc);
  if (__float_as_uint(nw) != __float_as_uint(old)) {
    f[v] = nw;
    unsigned long long k = atomicAdd(nupd, 1ull);
    if (upd) upd[k] = v;
  }
}

int64_t gradient_step(int np, const Pt* pts, const Tg* T, float alpha_b, float alpha_d, float* f, uint32_t* upd,
                      SolverBufs& B, uint32_t* status, cudaStream_t st) {
  cudaMemsetAsync(B.count, 0, sizeof(int), st);
  cudaMemsetAsync(B.counters, 0, sizeof(unsigned long long), st);
  if (np == 0) return 0;
  k_contrib<<<(np + 255) / 256, 256, 0, st>>>(np, pts, T, alpha_b, alpha_d, B.contrib, B.count); note_launch();
  // at most two contributions per point: sized by 2 np, counted on the device
  int32_t* idx = 2 * np <= B.cap_rsort
                     ? radix_sort64(2 * np, B.count, ContribBits{B.contrib}, B.rsort, B.idxB, B.idxA, status, st)
                     : merge_sort(2 * np, B.idxA, B.idxB, ContribLess{B.contrib}, st, B.count);
  k_apply_step<<<(2 * np + 255) / 256, 256, 0, st>>>(2 * np, B.count, idx, B.contrib, f, upd, B.counters);
  note_launch();
  unsigned long long nupd = 0;
  cudaMemcpyAsync(&nupd, B.counters, sizeof(nupd), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return (int64_t)nupd;
}

// ---------------------------------------------------------------------------
// Gradient of the topological loss (Eq. 2, q = 2) with respect to the field,
// for a fixed diagram and matching, in fp64: a point matched to target t
// contributes 2 (b - t_b) at v_b and 2 (d - t_d) at v_d (the essential class
// too), a diagonal-matched point b - d at v_b and d - b at v_d.  Per vertex
// the contributions are added in diagram order, birth before death.
// ---------------------------------------------------------------------------
struct Grad64 {
  uint32_t v;
  uint32_t idx;  // 2 * point + (0 birth, 1 death)
  double g;
};
static_assert(sizeof(Grad64) == sizeof(Contrib), "gradient entries reuse the contribution buffer");

__global__ void k_loss_grad_contrib(int np, const Pt* __restrict__ pts, const Tg* __restrict__ T,
                                    Grad64* __restrict__ G) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const Pt& p = pts[i];
  double b = (double)p.b, d = (double)p.d, gb, gd;
  if (p.tgt >= 0) {
    gb = __dmul_rn(2.0, __dsub_rn(b, (double)T[p.tgt].b));
    gd = __dmul_rn(2.0, __dsub_rn(d, (double)T[p.tgt].d));
  } else {
    gb = __dsub_rn(b, d);
    gd = __dsub_rn(d, b);
  }
  G[2 * i].v = p.vb;
  G[2 * i].idx = 2u * (uint32_t)i;
  G[2 * i].g = gb;
  G[2 * i + 1].v = p.vd;
  G[2 * i + 1].idx = 2u * (uint32_t)i + 1u;
  G[2 * i + 1].g = gd;
}

struct Grad64Less {
  const Grad64* c;
  __device__ unsigned long long key(int i) const { return ((unsigned long long)c[i].v << 32) | c[i].idx; }
  __device__ bool operator()(int a, int b) const { return key(a) < key(b); }
};

__global__ void k_loss_grad_apply(int n, const int32_t* __restrict__ idx, const Grad64* __restrict__ G,
                                  double* __restrict__ grad) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  uint32_t v = G[idx[r]].v;
  if (r > 0 && G[idx[r - 1]].v == v) return;
  double acc = 0.0;
  for (int s = r; s < n && G[idx[s]].v == v; ++s) acc = __dadd_rn(acc, G[idx[s]].g);
  grad[v] = acc;
}

void loss_gradient(int np, const Pt* pts, const Tg* T, SolverBufs& B, double* grad, int64_t nv, cudaStream_t st) {
  cudaMemsetAsync(grad, 0, sizeof(double) * (size_t)nv, st);
  if (np == 0) return;
  Grad64* G = reinterpret_cast<Grad64*>(B.contrib);
  k_loss_grad_contrib<<<(np + 255) / 256, 256, 0, st>>>(np, pts, T, G); note_launch();
  int32_t* idx = merge_sort(2 * np, B.idxA, B.idxB, Grad64Less{G}, st);
  k_loss_grad_apply<<<(2 * np + 255) / 256, 256, 0, st>>>(2 * np, idx, G, grad); note_launch();
}

// New field values: copies the changed ones and lists their vertices, so
// that the next diagram can be updated incrementally (Section 4.2).
__global__ void k_replace_values(int64_t nv, const float* __restrict__ in, float* __restrict__ f,
                                 uint32_t* __restrict__ upd, unsigned long long* __restrict__ count) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  float x = in[v];
  if (__float_as_uint(x) != __float_as_uint(f[v])) {
    f[v] = x;
    upd[atomicAdd(count, 1ull)] = (uint32_t)v;
  }
}

void replace_values(int64_t nv, const float* in, float* f, uint32_t* upd, unsigned long long* count,
                    cudaStream_t st) {
  cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
  k_replace_values<<<(unsigned)((nv + 255) / 256), 256, 0, st>>>(nv, in, f, upd, count); note_launch();
}

void targets_as_points(int nt, const Tg* T, Pt* R, cudaStream_t st) {
  if (nt > 0) k_targets_as_points<<<(nt + 255) / 256, 256, 0, st>>>(nt, T, R); note_launch();
}

}  // namespace tsf
