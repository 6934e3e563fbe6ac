// k_solver.cu -- diagram assembly (Section 2.2), diagram order (Section 2.4),
// target diagram (Section 3), still pairs and the reduced assignment
// (Section 4.3, Eq. 1), the direct gradient step (Section 4.1) and the loss
// (Eq. 2).
#include "tsf_kernels.cuh"
#include "tsf_solver.cuh"

namespace tsf {

// ---------------------------------------------------------------------------
// Stable merge sort of an index array by a comparator (bottom-up; each pass
// places every element by a binary search in its partner run).
// ---------------------------------------------------------------------------
template <class Less>
__global__ void k_merge_pass(int n, int width, const int32_t* __restrict__ in, int32_t* __restrict__ out, Less less) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
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

__global__ void k_iota(int n, int32_t* a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = i;
}

template <class Less>
static int32_t* merge_sort(int n, int32_t* a, int32_t* b, Less less, cudaStream_t st) {
  if (n <= 0) return a;
  k_iota<<<(n + 255) / 256, 256, 0, st>>>(n, a); note_launch();
  for (int w = 1; w < n; w *= 2) {
    k_merge_pass<<<(n + 255) / 256, 256, 0, st>>>(n, w, a, b, less); note_launch();
    int32_t* t = a;
    a = b;
    b = t;
  }
  return a;
}

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
__global__ void k_select_targets(int np, const Pt* __restrict__ pts, float theta, uint32_t* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < np) {
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

int make_targets(int np, const Pt* pts, float theta, SolverBufs& B, Tg* T, cudaStream_t st) {
  uint32_t* flag = B.u32a;
  uint32_t* pos = B.u32b;
  k_select_targets<<<(np + 255) / 256, 256, 0, st>>>(np, pts, theta, flag); note_launch();
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

// Shortest augmenting path (Hungarian algorithm with potentials): rows =
// targets in target order, columns = candidate points (point order) and one
// private diagonal column per target; ties go to the lowest column index.
__global__ void __launch_bounds__(kHT) k_hungarian(int k, int mc, const Cand* __restrict__ kept,
                                                   const uint32_t* __restrict__ koff,
                                                   const uint32_t* __restrict__ nkept,
                                                   const uint32_t* __restrict__ colpos,
                                                   const double* __restrict__ diag_t, HungWork H,
                                                   int32_t* __restrict__ col_to_row, uint32_t* status) {
  const int m = mc + k;
  const double INF = __longlong_as_double(0x7FF0000000000000ll);
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
        return;
      }
      int j0 = s_j0;
      if (threadIdx.x == 0) H.used[j0] = 1;
      int i0 = H.pm[j0];
      for (int j = 1 + threadIdx.x; j <= m; j += kHT) H.row[j] = INF;
      __syncthreads();
      for (int c = threadIdx.x; c < (int)nkept[i0 - 1]; c += kHT) {
        const Cand& cd = kept[koff[i0 - 1] + c];
        H.row[1 + colpos[cd.p]] = cd.w;
      }
      if (threadIdx.x == 0) H.row[1 + mc + (i0 - 1)] = diag_t[i0 - 1];
      __syncthreads();
      double ui0 = H.u[i0];
      double bv = INF;
      int bj = 0x7FFFFFFF;
      for (int j = 1 + threadIdx.x; j <= m; j += kHT) {
        if (H.used[j]) continue;
        double cur = __dsub_rn(__dsub_rn(H.row[j], ui0), H.v[j]);
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
      // block argmin, lowest index on ties
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
      double delta = s_delta;
      int j1 = s_j1;
      if (j1 == 0x7FFFFFFF) {
        if (threadIdx.x == 0) atomicOr(status, kErrInconsistent);
        return;
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
  for (int j = 1 + threadIdx.x; j <= mc; j += kHT) col_to_row[j - 1] = H.pm[j] - 1;
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

// Assignment phi*_j.  `ref` is the previous diagram (or the targets at j = 0,
// each assigned to itself).  Returns 0, or a negative value when a scratch
// buffer is too small (the caller grows it and retries).
int assign(int np, Pt* pts, int nr, const Pt* ref, int nt, const Tg* T, SolverBufs& B, uint32_t* status,
           AssignStats* as, cudaStream_t st) {
  // 1) still pairs
  cudaMemsetAsync(B.taken, 0, (size_t)max(nt, 1), st);
  int32_t* ck = merge_sort(np, B.idxA, B.idxB, KeyLess{pts}, st);
  int32_t* rk = nr > 0 ? merge_sort(nr, B.idxC, B.idxD, KeyLess{ref}, st) : B.idxC;
  k_still<<<(np + 255) / 256, 256, 0, st>>>(np, pts, ck, nr, ref, rk, B.tmp_pts, B.taken); note_launch();
  cudaMemcpyAsync(pts, B.tmp_pts, sizeof(Pt) * (size_t)np, cudaMemcpyDeviceToDevice, st);
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
    k_hungarian<<<1, kHT, 0, st>>>(k, mc, B.kept, B.u32b, B.nkept, B.colpos, B.diag_t, B.H, B.col_to_row, status); note_launch();
    k_apply_assignment<<<(mc + 255) / 256, 256, 0, st>>>(mc, B.col_to_row, B.col_point, B.plist, B.tlist, pts); note_launch();
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
  __device__ bool operator()(int a, int b) const {
    const Contrib& x = c[a];
    const Contrib& y = c[b];
    if (x.v != y.v) return x.v < y.v;
    return x.key < y.key;
  }
};

// one thread per vertex segment: acc = +0, acc += c in increasing value order
__global__ void k_apply_step(int nc, const int32_t* __restrict__ idx, const Contrib* __restrict__ C,
                             float* __restrict__ f, uint8_t* __restrict__ dirty, unsigned long long* __restrict__ nupd) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nc) return;
  uint32_t v = C[idx[r]].v;
  if (r > 0 && C[idx[r - 1]].v == v) return;
  float acc = 0.0f;
  for (int s = r; s < nc && C[idx[s]].v == v; ++s) acc = __fadd_rn(acc, C[idx[s]].c);
  float old = f[v];
  float nw = __fsub_rn(old, acc);
  if (__float_as_uint(nw) != __float_as_uint(old)) {
    f[v] = nw;
    if (dirty) dirty[v] = 1;
    atomicAdd(nupd, 1ull);
  }
}

int64_t gradient_step(int np, const Pt* pts, const Tg* T, float alpha_b, float alpha_d, float* f, uint8_t* dirty,
                      SolverBufs& B, cudaStream_t st) {
  cudaMemsetAsync(B.count, 0, sizeof(int), st);
  cudaMemsetAsync(B.counters, 0, sizeof(unsigned long long), st);
  if (np == 0) return 0;
  k_contrib<<<(np + 255) / 256, 256, 0, st>>>(np, pts, T, alpha_b, alpha_d, B.contrib, B.count); note_launch();
  int nc = 0;
  cudaMemcpyAsync(&nc, B.count, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  int32_t* idx = merge_sort(nc, B.idxA, B.idxB, ContribLess{B.contrib}, st);
  k_apply_step<<<(nc + 255) / 256, 256, 0, st>>>(nc, idx, B.contrib, f, dirty, B.counters); note_launch();
  unsigned long long nupd = 0;
  cudaMemcpyAsync(&nupd, B.counters, sizeof(nupd), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return (int64_t)nupd;
}

void targets_as_points(int nt, const Tg* T, Pt* R, cudaStream_t st) {
  if (nt > 0) k_targets_as_points<<<(nt + 255) / 256, 256, 0, st>>>(nt, T, R); note_launch();
}

}  // namespace tsf
