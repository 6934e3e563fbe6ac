// k_pairs.cu -- persistence pairs of the critical cells.
//
// The critical cells left by the lower-star gradient are paired exactly as
// the plain reduction of the lexicographic filtration would pair them:
//   D0 (minimum, 1-saddle): integral lines from both ends of each critical
//     edge down to minima, then the elder rule over critical edges in
//     increasing order (union-find);
//   D2 (2-saddle, maximum): by duality, integral lines from the two
//     tetrahedra (or the outside) of each critical triangle up to maxima, then
//     the elder rule over critical triangles in decreasing order, the outside
//     of the domain being the oldest node;
//   D1 (1-saddle, 2-saddle): the column reduction of the critical triangles
//     left over, restricted to positive edges, where a gradient-paired edge is
//     eliminated with its triangle's reduced column.
// The union-find runs in rounds of deterministic reservations: an item
// commits when no earlier item touches the component that would die, which
// gives exactly the sequential elder-rule result whatever the schedule.
#include <atomic>
#include <utility>

#include "tsf_grid.cuh"
#include "tsf_group.cuh"
#include "tsf_kernels.cuh"
#include "tsf_star.cuh"

namespace tsf {

constexpr int kUFT = 1024;
// Schedule of the union-find rounds (process-wide; tsf_debug_set changes
// them for tests): items from which the rounds start over the whole GPU,
// active items below which one block finishes them, a cap on the rounds
// (0: the bound n + 2 that can never be reached) and the grid barrier's poll
// limit.
std::atomic<int64_t> g_uf_grid_min{1 << 16};
std::atomic<int64_t> g_uf_handoff{1 << 13};
std::atomic<int64_t> g_uf_round_cap{0};
std::atomic<int64_t> g_barrier_limit{1 << 24};
// ... and of the D1 reduction: columns from which its rounds start over the
// whole GPU, active columns below which one block finishes them
std::atomic<int64_t> g_d1_grid_min{1 << 16};
std::atomic<int64_t> g_d1_handoff{1 << 12};
// schedule of the D1 Morse boundaries' phase A: 0 the default (half a warp
// per column, 64 frontier + 128 stage entries for diagrams of at least 2^19
// critical triangles, else as 5), 1 and 2 one warp with 128 +
// 256 and 256 + 512, 3 one warp with 64 + 128 uncapped, 4 capped, 5 half a
// warp with 32 + 64, 6 a quarter of a warp with 16 + 32, 7 half a warp
// with 64 + 128 at any size
std::atomic<int64_t> g_d1_phase_a{0};
// blocks per SM the lower-star gradient kernels are compiled for: 0 the
// default (six), 1 no register cap, 2 five
std::atomic<int64_t> g_gradient_blocks{0};
// entries of a column the D1 reduction's short rounds keep in shared memory
// per warp while every warp is busy (at most 512, scaled up when fewer
// warps share the buffers; 0: every chained addition runs in the pool)
std::atomic<int64_t> g_chain_cap{512};
// D1 Morse boundaries: visits a thread chains per round along single-target
// updates (0: the default), rounds of the first phase before a column moves
// to a block (0: the default); both defaults depend on the diagram's size
std::atomic<int64_t> g_morse_chain{0};
std::atomic<int64_t> g_morse_rounds{0};
// D1 reduction: active columns up to which a round chains additions (0: the default)
std::atomic<int64_t> g_chain_max{0};

static std::atomic<int64_t>* knob(int what) {
  return what == 1   ? &g_uf_grid_min
         : what == 2 ? &g_uf_handoff
         : what == 3 ? &g_uf_round_cap
         : what == 4 ? &g_barrier_limit
         : what == 5 ? &g_d1_grid_min
         : what == 6 ? &g_d1_handoff
         : what == 7 ? &g_d1_phase_a
         : what == 8 ? &g_gradient_blocks
         : what == 9 ? &g_chain_cap
         : what == 10 ? &g_morse_chain
         : what == 11 ? &g_morse_rounds
         : what == 12 ? &g_chain_max
                     : nullptr;
}

int64_t get_knob(int what) {
  std::atomic<int64_t>* k = knob(what);
  return k ? k->load() : -1;
}

int64_t set_knob(int what, int64_t value) {
  std::atomic<int64_t>* k = knob(what);
  if (!k) return -1;
  return k->exchange(value);
}

// Control block of the whole-GPU union-find rounds (PairScratch::counter).
struct UfCtl {
  unsigned bar[2];  // grid barrier: arrivals, generation
  int n[2];         // lengths of listA, listB
  int which;        // list holding the active items
  int rounds;       // rounds done
  int pad[10];
};

// ---------------------------------------------------------------------------
// integral lines
// ---------------------------------------------------------------------------
// A descending line visits each vertex at most once (ranks decrease), so it
// has at most nv steps; an ascending dual line crosses into a higher vertex's
// star at most nv times and takes at most 24 steps inside one star.
__device__ __forceinline__ int32_t trace_down(uint32_t w, const uint8_t* __restrict__ vnext8,
                                              const uint32_t* __restrict__ cidx, const NbrDelta& nd, int64_t nv) {
  for (int64_t s = 0; s <= nv; ++s) {
    int k = vnext8[w];
    if (k == kVnextMin) return (int32_t)cidx[w];
    w = (uint32_t)((int32_t)w + nd.d[k]);
  }
  return -1;
}

// One thread per endpoint of each critical edge.
__global__ void k_d0_trace(int n1, int64_t nv, CritLists L, const uint8_t* __restrict__ vnext8,
                           const uint32_t* __restrict__ cidx, NbrDelta nd, int32_t* __restrict__ ends,
                           uint32_t* status) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * (int64_t)n1) return;
  uint32_t vn = L.c1_vn[t >> 1];
  uint32_t v = vn >> 4;
  if (t & 1) v = (uint32_t)((int32_t)v + nd.d[vn & 15u]);
  int32_t a = trace_down(v, vnext8, cidx, nd, nv);
  if (a < 0) atomicOr(status, kErrTrace);
  ends[t] = a < 0 ? 0 : a;
}

__device__ __forceinline__ Rec ld_rec(const Rec* rec, uint32_t v) {
  const uint4* p = reinterpret_cast<const uint4*>(rec + v);
  uint4 a = __ldg(p), b = __ldg(p + 1);
  Rec r;
  r.w[0] = a.x; r.w[1] = a.y; r.w[2] = a.z; r.w[3] = a.w;
  r.w[4] = b.x; r.w[5] = b.y; r.w[6] = b.z; r.w[7] = b.w;
  return r;
}

// Ascending integral line in the dual: from tetrahedron (w, tau) follow the
// record codes to a maximum (its index) or to the outside (returns n3).
__device__ int32_t trace_up(uint32_t w, int tau, const Rec* __restrict__ rec, const uint32_t* __restrict__ cidx,
                            const int32_t* nd, int n3, const UpStep* up, int64_t nv) {
  Rec r = ld_rec(rec, w);
  for (int64_t s = 0; s <= 25 * nv; ++s) {
    int code = rec_tet_code(r, tau);
    if (code == kCodeMax) return (int32_t)cidx[w];
    if (code == kCodeOut) return n3;
    if (code < 24) {
      tau = code;
      continue;
    }
    if (code >= 96) return -1;
    UpStep u = up[code - 24];
    tau = u.tau;
    w = (uint32_t)((int32_t)w + nd[u.c]);
    r = ld_rec(rec, w);
  }
  return -1;
}

// One thread per (critical triangle, side): the ascending dual line from the
// tetrahedron on that side to a maximum or the outside.
__global__ void k_d2_trace(Dims d, int n2, int n3, CritLists L, const uint32_t* __restrict__ rank,
                           const Rec* __restrict__ rec, const uint32_t* __restrict__ cidx, NbrDelta nd,
                           int32_t* __restrict__ ends, uint32_t* status) {
  __shared__ UpStep sup[72];
  __shared__ int32_t snd[14];
  if (threadIdx.x < 14) snd[threadIdx.x] = nd.d[threadIdx.x];
  if (threadIdx.x < 72) sup[threadIdx.x] = c_up.s[threadIdx.x];
  __syncthreads();
  int64_t tt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tt >= 2 * (int64_t)n2) return;
  int i = (int)(tt >> 1), k = (int)(tt & 1);
  const Geo& G = c_geo;
  uint32_t ve = L.c2_ve[i];
  uint32_t v = ve >> 6;
  int e = (int)(ve & 63u);
  int a = G.edge[e][0], b = G.edge[e][1];
  int x, y, z;
  vxyz(d, v, x, y, z);
  int t = G.edge_tri[e][k];
  int j = 0;
  while (G.tri[t][j] == a || G.tri[t][j] == b) ++j;
  int c = G.tri[t][j];
  int nx, ny, nz;
  int32_t res;
  if (!nbr_xyz(d, x, y, z, c, nx, ny, nz)) {
    res = n3;
  } else {
    uint32_t wc = vid(d, nx, ny, nz);
    if (rank[wc] < rank[v]) {
      res = trace_up(v, t, rec, cidx, snd, n3, sup, d.nv);
    } else {
      int i0 = nbr_index(G, -G.off[c][0], -G.off[c][1], -G.off[c][2]);
      int i1 = nbr_index(G, G.off[a][0] - G.off[c][0], G.off[a][1] - G.off[c][1], G.off[a][2] - G.off[c][2]);
      int i2 = nbr_index(G, G.off[b][0] - G.off[c][0], G.off[b][1] - G.off[c][1], G.off[b][2] - G.off[c][2]);
      int tau = (i0 >= 0 && i1 >= 0 && i2 >= 0) ? G.tri_of3[i0][i1][i2] : -1;
      res = tau < 0 ? -1 : trace_up(wc, tau, rec, cidx, snd, n3, sup, d.nv);
    }
  }
  if (res < 0) {
    atomicOr(status, kErrTrace);
    res = n3;
  }
  ends[tt] = res;
}

// ---------------------------------------------------------------------------
// elder-rule union-find by rounds of deterministic reservations (one block)
// ---------------------------------------------------------------------------
constexpr int kFindLimit = 1 << 26;

// For kernels spread over several SMs: every read of the union-find state
// goes to L2 (another SM may have linked a root since this SM cached it).
__device__ __forceinline__ int uf_root_cg(int32_t* parent, int x) {
  for (int s = 0; s < kFindLimit; ++s) {
    const int p = __ldcg(&parent[x]);
    if (p == x) return x;
    const int gp = __ldcg(&parent[p]);
    if (gp != p) parent[x] = gp;
    x = gp;
  }
  return x;
}

__device__ __forceinline__ int uf_root(int32_t* parent, int x) {
  for (int s = 0; s < kFindLimit; ++s) {
    int p = parent[x];
    if (p == x) return x;
    int gp = parent[p];
    if (gp != p) parent[x] = gp;
    x = gp;
  }
  return x;
}

__device__ __forceinline__ int block_exscan_int(int v, int& total) {
  __shared__ int sw[kUFT / 32 + 1];
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
    int s = sw[lane];
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

// n items (priority i, or n-1-i when `reverse`), nn nodes.  Younger node =
// larger index (reverse = false) or smaller index (reverse = true).
// kill[i] = node killed by item i, or -1 (item closes a cycle).
// `ctl` (may be null): resume after k_uf_rounds_grid, from its active list
// (ctl->which selects listA or listB, ctl->n[which] its length) and its
// union-find state.
__global__ void __launch_bounds__(kUFT) k_uf_rounds(int n, int nn, bool reverse, const int32_t* __restrict__ ends,
                                                    int32_t* parent, int32_t* reserve, int32_t* listA,
                                                    int32_t* listB, int32_t* roots, int32_t* kill,
                                                    const UfCtl* ctl, int cap, uint32_t* status) {
  __shared__ int s_n;
  int32_t* cur = listA;
  int32_t* nxt = listB;
  int round0 = 0;
  if (ctl) {
    // the whole-GPU rounds gave up (a barrier or the round cap): their lists
    // may be partly written, so nothing resumes from them
    if (*reinterpret_cast<const volatile uint32_t*>(status) & (kErrSpin | kErrRounds)) return;
    if (ctl->which) {
      cur = listB;
      nxt = listA;
    }
    if (threadIdx.x == 0) s_n = ctl->n[ctl->which];
    round0 = ctl->rounds;
  } else {
    for (int x = threadIdx.x; x < nn; x += kUFT) {
      parent[x] = x;
      reserve[x] = 0x7FFFFFFF;
    }
    for (int i = threadIdx.x; i < n; i += kUFT) {
      kill[i] = -1;
      listA[i] = i;
    }
    if (threadIdx.x == 0) s_n = n;
  }
  __syncthreads();
  for (int round = round0;; ++round) {
    int m = s_n;
    if (m == 0) break;
    if (round > n + 2 || (cap > 0 && round >= cap)) {
      if (threadIdx.x == 0) atomicOr(status, kErrRounds);
      break;
    }
    for (int k = threadIdx.x; k < m; k += kUFT) {
      int i = cur[k];
      int a = uf_root(parent, ends[2 * i]), b = uf_root(parent, ends[2 * i + 1]);
      roots[2 * i] = a;
      roots[2 * i + 1] = b;
      if (a != b) {
        int pr = reverse ? n - 1 - i : i;
        atomicMin(&reserve[a], pr);
        atomicMin(&reserve[b], pr);
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < m; k += kUFT) {
      int i = cur[k];
      int a = roots[2 * i], b = roots[2 * i + 1];
      if (a == b) continue;
      int young = reverse ? min(a, b) : max(a, b);
      int old = a + b - young;
      int pr = reverse ? n - 1 - i : i;
      if (reserve[young] == pr) {
        parent[young] = old;
        kill[i] = young;
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < m; k += kUFT) {
      int i = cur[k];
      int a = roots[2 * i], b = roots[2 * i + 1];
      if (a != b) {
        reserve[a] = 0x7FFFFFFF;
        reserve[b] = 0x7FFFFFFF;
      }
    }
    int cnt = 0;
    for (int base = 0; base < m; base += kUFT) {
      int k = base + threadIdx.x;
      int keep = 0, i = 0;
      if (k < m) {
        i = cur[k];
        keep = (roots[2 * i] != roots[2 * i + 1]) && kill[i] < 0;
      }
      int tot;
      int ex = block_exscan_int(keep, tot);
      if (keep) nxt[cnt + ex] = i;
      cnt += tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_n = cnt;
    __syncthreads();
    int32_t* t = cur;
    cur = nxt;
    nxt = t;
  }
}

__global__ void k_mark_d0(int n1, const int32_t* __restrict__ kill, uint8_t* __restrict__ killed) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n1) killed[i] = kill[i] >= 0 ? 1 : 0;
}
__global__ void k_d0mask_clear(int n1, CritLists L, uint32_t* __restrict__ d0mask) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n1) d0mask[L.c1_vn[i] >> 4] = 0u;
}
__global__ void k_d0mask_set(int n1, CritLists L, const int32_t* __restrict__ kill, uint32_t* __restrict__ d0mask) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n1 && kill[i] >= 0) atomicOr(&d0mask[L.c1_vn[i] >> 4], 1u << (L.c1_vn[i] & 15u));
}

// The same rounds over the whole GPU (cooperative launch, grid barriers
// between the phases of a round), while the active list holds at least
// `handoff` items; then it stops and k_uf_rounds resumes from ctl.  The
// list order within a round does not matter (reservations compare item
// priorities), so blocks append survivors with atomics.
__global__ void __launch_bounds__(kUFT) k_uf_rounds_grid(int n, int nn, bool reverse,
                                                         const int32_t* __restrict__ ends, int32_t* parent,
                                                         int32_t* reserve, int32_t* listA, int32_t* listB,
                                                         int32_t* roots, int32_t* kill, UfCtl* ctl, int handoff,
                                                         int cap, unsigned limit, uint32_t* status) {
  __shared__ int s_cnt, s_base;
  const unsigned nb = gridDim.x;
  const int gt = blockIdx.x * kUFT + threadIdx.x, gn = nb * kUFT;
  for (int x = gt; x < nn; x += gn) {
    parent[x] = x;
    reserve[x] = 0x7FFFFFFF;
  }
  for (int i = gt; i < n; i += gn) {
    kill[i] = -1;
    listA[i] = i;
  }
  if (gt == 0) {
    ctl->n[0] = n;
    ctl->n[1] = 0;
    ctl->which = 0;
    ctl->rounds = 0;
  }
  if (!grid_barrier(ctl->bar, nb, status, limit)) return;
  int which = 0;
  for (int round = 0;; ++round) {
    const int m = *reinterpret_cast<volatile int*>(&ctl->n[which]);
    if (m == 0 || m < handoff) break;
    if (round > n + 2 || (cap > 0 && round >= cap)) {
      if (gt == 0) atomicOr(status, kErrRounds);
      break;
    }
    const int32_t* cur = which ? listB : listA;
    int32_t* nxt = which ? listA : listB;
    for (int k = gt; k < m; k += gn) {
      const int i = __ldcg(&cur[k]);
      const int a = uf_root_cg(parent, ends[2 * i]), b = uf_root_cg(parent, ends[2 * i + 1]);
      roots[2 * i] = a;
      roots[2 * i + 1] = b;
      if (a != b) {
        const int pr = reverse ? n - 1 - i : i;
        atomicMin(&reserve[a], pr);
        atomicMin(&reserve[b], pr);
      }
    }
    if (gt == 0) ctl->n[which ^ 1] = 0;
    if (!grid_barrier(ctl->bar, nb, status, limit)) return;
    for (int k = gt; k < m; k += gn) {
      const int i = __ldcg(&cur[k]);
      const int a = __ldcg(&roots[2 * i]), b = __ldcg(&roots[2 * i + 1]);
      if (a == b) continue;
      const int young = reverse ? min(a, b) : max(a, b);
      const int old = a + b - young;
      const int pr = reverse ? n - 1 - i : i;
      if (__ldcg(&reserve[young]) == pr) {
        parent[young] = old;
        kill[i] = young;
      }
    }
    if (!grid_barrier(ctl->bar, nb, status, limit)) return;
    // clear the reservations and keep the items still joining two components
    for (int base = blockIdx.x * kUFT; base < m; base += gn) {
      const int k = base + threadIdx.x;
      int keep = 0, i = 0;
      if (k < m) {
        i = __ldcg(&cur[k]);
        const int a = __ldcg(&roots[2 * i]), b = __ldcg(&roots[2 * i + 1]);
        if (a != b) {
          reserve[a] = 0x7FFFFFFF;
          reserve[b] = 0x7FFFFFFF;
        }
        keep = (a != b) && __ldcg(&kill[i]) < 0;
      }
      int tot;
      const int ex = block_exscan_int(keep, tot);
      if (threadIdx.x == 0) {
        s_cnt = tot;
        s_base = tot ? atomicAdd(&ctl->n[which ^ 1], tot) : 0;
      }
      __syncthreads();
      if (keep) nxt[s_base + ex] = i;
      __syncthreads();
    }
    which ^= 1;
    if (gt == 0) {
      ctl->which = which;
      ctl->rounds = round + 1;
    }
    if (!grid_barrier(ctl->bar, nb, status, limit)) return;
  }
}

// Union-find rounds of n items: over the whole GPU while the active list
// is long, then on one block.
void uf_rounds(int n, int nn, bool reverse, PairScratch& S, int32_t* kill, uint32_t* status, cudaStream_t st) {
  int cap = (int)std::min<int64_t>(g_uf_round_cap.load(), 1 << 30);
  const int nb = n >= g_uf_grid_min.load() ? cooperative_blocks((const void*)k_uf_rounds_grid, kUFT) : 0;
  if (nb > 0) {
    UfCtl* ctl = reinterpret_cast<UfCtl*>(S.counter);
    cudaMemsetAsync(ctl, 0, sizeof(UfCtl), st);
    int handoff = (int)std::min<int64_t>(g_uf_handoff.load(), 1 << 30);
    unsigned limit = (unsigned)std::min<int64_t>(std::max<int64_t>(g_barrier_limit.load(), 1), 1u << 30);
    void* args[] = {&n,        &nn,   &reverse, &S.ends, &S.parent, &S.reserve, &S.listA, &S.listB, &S.roots,
                    &kill,     &ctl,  &handoff, &cap,    &limit,    &status};
    if (cooperative_launch((const void*)k_uf_rounds_grid, dim3(nb), dim3(kUFT), args, st) == cudaSuccess) {
      k_uf_rounds<<<1, kUFT, 0, st>>>(n, nn, reverse, S.ends, S.parent, S.reserve, S.listA, S.listB, S.roots, kill,
                                      ctl, cap, status); note_launch();
      return;
    }
    cudaGetLastError();  // not launched: the single block does every round
  }
  k_uf_rounds<<<1, kUFT, 0, st>>>(n, nn, reverse, S.ends, S.parent, S.reserve, S.listA, S.listB, S.roots, kill,
                                  nullptr, cap, status); note_launch();
}

void launch_d0(const Dims& d, const NbrDelta& nd, const CritLists& L, int n0, int n1, const uint8_t* vnext8,
               const uint32_t* cidx, PairScratch& S, PairOut& P, uint32_t* status, cudaStream_t st) {
  if (n1 > 0) {
    k_d0_trace<<<(unsigned)((2 * (int64_t)n1 + 255) / 256), 256, 0, st>>>(n1, d.nv, L, vnext8, cidx, nd, S.ends,
                                                                         status); note_launch();
    uf_rounds(n1, n0, false, S, P.d0_min, status, st);
    k_mark_d0<<<(n1 + 255) / 256, 256, 0, st>>>(n1, P.d0_min, P.d0_killed); note_launch();
    k_d0mask_clear<<<(n1 + 255) / 256, 256, 0, st>>>(n1, L, P.d0mask); note_launch();
    k_d0mask_set<<<(n1 + 255) / 256, 256, 0, st>>>(n1, L, P.d0_min, P.d0mask); note_launch();
  }
}

void launch_d2(const Dims& d, const NbrDelta& nd, const CritLists& L, int n2, int n3, const uint32_t* rank,
               const Rec* rec, const uint32_t* cidx, PairScratch& S, PairOut& P, uint32_t* status,
               cudaStream_t st) {
  if (n2 > 0) {
    k_d2_trace<<<(unsigned)((2 * (int64_t)n2 + 127) / 128), 128, 0, st>>>(d, n2, n3, L, rank, rec, cidx, nd, S.ends,
                                                                         status); note_launch();
    uf_rounds(n2, n3 + 1, true, S, P.d2_max, status, st);
  }
}

// ---------------------------------------------------------------------------
// D1: column reduction of the critical triangles not paired in D2
// ---------------------------------------------------------------------------
struct D1Ctx {
  Dims d;
  NbrDelta nd;
  const uint32_t* rank;
  const uint32_t* order;
  const Rec* rec;
  const D1Tab* tab;
  const uint32_t* c1base;
  CritLists L;
  const uint8_t* d0_killed;
  const uint32_t* d0mask;
  const float* f;
  int chain;  // visits one thread makes per round along single-target updates
};

__device__ __forceinline__ int nbr_of_pair(const Dims& d, uint32_t hi, uint32_t lo) {
  int hx, hy, hz, lx, ly, lz;
  vxyz(d, hi, hx, hy, hz);
  vxyz(d, lo, lx, ly, lz);
  return nbr_index(lx - hx, ly - hy, lz - hz);
}
__device__ __forceinline__ int nbr_of_pair(const Dims& d, uint32_t hi, uint32_t lo, const Geo& G) {
  int hx, hy, hz, lx, ly, lz;
  vxyz(d, hi, hx, hy, hz);
  vxyz(d, lo, lx, ly, lz);
  return nbr_index(G, lx - hx, ly - hy, lz - hz);
}

__device__ int crit_edge_index(const D1Ctx& c, uint32_t hi, const Rec& r, int k) {
  int cnt = __popc(rec_crit_edges(r));
  uint32_t base = c.c1base[hi];
  for (int j = 0; j < cnt; ++j)
    if ((int)(c.L.c1_vn[base + j] & 15u) == k) return (int)(base + j);
  return -1;
}

// 0: negative edge (not a row of the D1 matrix), 1: positive and critical,
// 2: positive and paired with a triangle in its lower star.
__device__ int edge_status(const D1Ctx& c, uint32_t p, uint32_t q, unsigned long long& key, int& ci) {
  uint32_t rp = c.rank[p], rq = c.rank[q];
  uint32_t hi = rp > rq ? p : q, lo = rp > rq ? q : p;
  key = ((unsigned long long)max(rp, rq) << 32) | min(rp, rq);
  int k = nbr_of_pair(c.d, hi, lo);
  Rec r = ld_rec(c.rec, hi);
  if (rec_vnext(r) == k) return 0;
  if ((rec_crit_edges(r) >> k) & 1u) {
    ci = crit_edge_index(c, hi, r, k);
    if (ci < 0) return 0;
    return c.d0_killed[ci] ? 0 : 1;
  }
  return 2;
}

struct Heap {
  unsigned long long* h;
  uint32_t off, cap, size;
};

__device__ bool heap_push(D1Work& W, Heap& H, unsigned long long key, uint32_t* status) {
  if (H.size == H.cap) {
    uint32_t ncap = H.cap * 2;
    uint32_t noff = atomicAdd(W.pool_head, ncap);
    if ((unsigned long long)noff + ncap > W.pool_cap) {
      atomicOr(status, kErrPool);
      return false;
    }
    unsigned long long* nh = W.pool + noff;
    for (uint32_t i = 0; i < H.size; ++i) nh[i] = H.h[i];
    H.h = nh;
    H.off = noff;
    H.cap = ncap;
  }
  uint32_t i = H.size++;
  H.h[i] = key;
  while (i > 0) {
    uint32_t p = (i - 1) >> 1;
    if (H.h[p] >= H.h[i]) break;
    unsigned long long t = H.h[p];
    H.h[p] = H.h[i];
    H.h[i] = t;
    i = p;
  }
  return true;
}

__device__ unsigned long long heap_pop(Heap& H) {
  unsigned long long top = H.h[0];
  unsigned long long last = H.h[--H.size];
  uint32_t i = 0;
  while (true) {
    uint32_t l = 2 * i + 1;
    if (l >= H.size) break;
    uint32_t r = l + 1;
    uint32_t m = (r < H.size && H.h[r] > H.h[l]) ? r : l;
    if (H.h[m] <= last) break;
    H.h[i] = H.h[m];
    i = m;
  }
  if (H.size > 0) H.h[i] = last;
  return top;
}

// largest entry present an odd number of times (Z/2), 0 if the column is empty
__device__ unsigned long long heap_low(Heap& H) {
  while (H.size > 0) {
    unsigned long long top = heap_pop(H);
    int c = 1;
    while (H.size > 0 && H.h[0] == top) {
      heap_pop(H);
      ++c;
    }
    if (c & 1) return top;
  }
  return 0ull;
}

__device__ __forceinline__ Heap heap_of(D1Work& W, int j) {
  Heap H;
  H.off = W.hoff[j];
  H.cap = W.hcap[j];
  H.size = W.hsize[j];
  H.h = W.pool + H.off;
  return H;
}
__device__ __forceinline__ void heap_store(D1Work& W, int j, const Heap& H) {
  W.hoff[j] = H.off;
  W.hcap[j] = H.cap;
  W.hsize[j] = H.size;
}

__device__ void push_if_positive(const D1Ctx& c, D1Work& W, Heap& H, uint32_t p, uint32_t q, uint32_t* status) {
  unsigned long long key;
  int ci;
  if (edge_status(c, p, q, key, ci) != 0) heap_push(W, H, key, status);
}

__global__ void k_d1_select(int n2, const int32_t* __restrict__ d2_max, uint32_t* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n2) flag[i] = d2_max[i] < 0 ? 1u : 0u;
}
__global__ void k_d1_gather(int n2, const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                            int32_t* __restrict__ cols, int32_t* __restrict__ d1_edge, int32_t* __restrict__ ncols) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n2) {
    d1_edge[i] = -1;
    if (flag[i]) cols[pos[i]] = i;
    if (i == n2 - 1) *ncols = (int32_t)(pos[i] + flag[i]);
  }
}

// Growable array in the pool (a column's heap or its Morse boundary).
struct Vec {
  unsigned long long* h;
  uint32_t off, cap, size;
};

__device__ bool vec_alloc(D1Work& W, Vec& v, uint32_t cap, uint32_t* status) {
  uint32_t off = atomicAdd(W.pool_head, cap);
  if ((unsigned long long)off + cap > W.pool_cap) {
    atomicOr(status, kErrPool);
    return false;
  }
  v.off = off;
  v.cap = cap;
  v.size = 0;
  v.h = W.pool + off;
  return true;
}

__device__ bool vec_push(D1Work& W, Vec& v, unsigned long long x, uint32_t* status) {
  if (v.size == v.cap) {
    Vec n;
    if (!vec_alloc(W, n, v.cap * 2, status)) return false;
    for (uint32_t i = 0; i < v.size; ++i) n.h[i] = v.h[i];
    n.size = v.size;
    v = n;
  }
  v.h[v.size++] = x;
  return true;
}

__device__ __forceinline__ Heap as_heap(const Vec& v) {
  Heap H;
  H.h = v.h;
  H.off = v.off;
  H.cap = v.cap;
  H.size = v.size;
  return H;
}

constexpr int kD1StepLimit = 1 << 24;

// Phase 1: Morse boundary of each candidate triangle t: its boundary (positive
// edges) with every gradient-paired edge eliminated by its triangle's reduced
// column, largest first, one lower star at a time.  Output: the critical
// edges left (C1 indices), in decreasing lexicographic order.
__global__ void k_d1_morse(D1Ctx c, D1Work W, uint32_t* status) {
  const int ncols = W.flags[1];
  __shared__ Geo sg;
  geo_to_shared(sg);
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols) return;
  if (W.redo && !W.redo[j]) return;
  W.hsize[j] = 0;
  W.hoff[j] = 0;
  Vec hv, out;
  if (!vec_alloc(W, hv, 32, status) || !vec_alloc(W, out, 8, status)) return;
  Heap H = as_heap(hv);
  uint32_t ve = c.L.c2_ve[W.cols[j]];
  uint32_t v0 = ve >> 6;
  int e0 = (int)(ve & 63u);
  uint32_t a0 = (uint32_t)((int32_t)v0 + c.nd.d[c_geo.edge[e0][0]]);
  uint32_t b0 = (uint32_t)((int32_t)v0 + c.nd.d[c_geo.edge[e0][1]]);
  push_if_positive(c, W, H, v0, a0, status);
  push_if_positive(c, W, H, v0, b0, status);
  push_if_positive(c, W, H, a0, b0, status);
  int nblocks = 0;
  for (int step = 0;; ++step) {
    if (step >= kD1StepLimit) {
      atomicOr(status, kErrRounds);
      return;
    }
    unsigned long long top = heap_low(H);
    if (top == 0) break;
    uint32_t rv = (uint32_t)(top >> 32);
    uint32_t v = c.order[rv];
    // every entry of v's lower star, with its parity, by neighbour index
    uint32_t m = 1u << nbr_of_pair(c.d, v, c.order[(uint32_t)(top & 0xFFFFFFFFull)]);
    while (H.size > 0 && (uint32_t)(H.h[0] >> 32) == rv) {
      unsigned long long e = heap_pop(H);
      m ^= 1u << nbr_of_pair(c.d, v, c.order[(uint32_t)(e & 0xFFFFFFFFull)]);
    }
    if (!m) continue;
    ++nblocks;
    Rec r = ld_rec(c.rec, v);
    uint32_t crit = rec_crit_edges(r);
    Star s;
    star_load(s, c.d, v, c.rank);
    int8_t y_of[14];
    uint64_t path_of[14];
    star_chains(s, y_of, path_of, sg);
    for (int p = s.nl - 1; p >= 1; --p) {
      int x = s.by_pos[p];
      if (!((m >> x) & 1u)) continue;
      m &= ~(1u << x);
      if ((crit >> x) & 1u) {
        int ci = crit_edge_index(c, v, r, x);
        if (ci >= 0 && !c.d0_killed[ci]) vec_push(W, out, (unsigned long long)ci, status);
        continue;
      }
      int y = y_of[x];
      if (y < 0) {
        atomicOr(status, kErrInconsistent);
        return;
      }
      if (y != s.by_pos[0]) m ^= 1u << y;  // w*y stays in this lower star (w*y negative if y is the lowest)
      for (uint64_t pm = path_of[x]; pm; pm &= pm - 1) {
        int le = __ffsll((long long)pm) - 1;
        uint32_t pa = (uint32_t)((int32_t)v + c.nd.d[c_geo.edge[le][0]]);
        uint32_t pb = (uint32_t)((int32_t)v + c.nd.d[c_geo.edge[le][1]]);
        push_if_positive(c, W, H, pa, pb, status);
      }
    }
  }
  W.hoff[j] = out.off;
  W.hsize[j] = out.size;
  atomicAdd(&W.stats[0], (unsigned long long)nblocks);
  atomicMax(&W.stats[1], (unsigned long long)nblocks);
}

// ---------------------------------------------------------------------------
// Phase 1, one group of threads per column.  The pending entries of a column
// are lower stars with a parity mask over their 14 edge directions.  All of
// a column's updates come from its own group, so they live in the group's
// shared memory: the frontier, sorted by descending key = value_key << 32 |
// vertex (the rank order), one entry per star.  Each round the group takes
// the NT highest entries, one per thread; every visit appends its updates of
// target stars to a stage; the stage is sorted, merged into the rest of the
// frontier and equal keys are combined (xor of masks, zero masks dropped).
// The projection is linear, so a star that receives entries after it was
// processed simply comes back, and the order only decides how often.
// ---------------------------------------------------------------------------
// Frontier entries are FEnt: key = value_key << 32 | vertex (0 never occurs,
// NaN is rejected), payload = the pending parity mask.  Entries saved in the
// pool (8-byte aligned) are two 64-bit words.
__device__ __forceinline__ void fent_save(unsigned long long* p, const FEnt& e) {
  p[0] = e.key;
  p[1] = e.mask;
}
__device__ __forceinline__ FEnt fent_restore(const unsigned long long* p) {
  FEnt e;
  e.key = p[0];
  e.mask = (uint32_t)p[1];
  e.pad = 0u;
  return e;
}

__device__ __forceinline__ unsigned long long star_key(uint32_t vkey, uint32_t v) {
  return ((unsigned long long)vkey << 32) | v;
}

// Target stars of the link edges left by a visit, with compile-time
// geometry: edge (a, b) goes to the lower star of whichever endpoint ranks
// higher (P: a, Q: b), as the direction towards the other endpoint.
template <int LE>
__device__ __forceinline__ void link_edge_target(uint64_t P, uint64_t Q, uint32_t (&tm)[14]) {
  constexpr int a = geo_edge(LE, 0), b = geo_edge(LE, 1);
  constexpr int dab = geo_dir(a, b), dba = geo_dir(b, a);
  tm[a] ^= (uint32_t)((P >> LE) & 1ull) << dab;
  tm[b] ^= (uint32_t)((Q >> LE) & 1ull) << dba;
}
template <int... LE>
__device__ __forceinline__ void link_targets(uint64_t P, uint64_t Q, uint32_t (&tm)[14],
                                             std::integer_sequence<int, LE...>) {
  (link_edge_target<LE>(P, Q, tm), ...);
}
template <int X>
__device__ __forceinline__ void closure_of(const D1Tab& t, uint32_t m, uint64_t& path, uint32_t& em) {
  if ((m >> X) & 1u) {
    path ^= tab_closure<X>(t);
    em ^= 1u << tab_end(t, X);
  }
}
template <int... X>
__device__ __forceinline__ void closures(const D1Tab& t, uint32_t m, uint64_t& path, uint32_t& em,
                                         std::integer_sequence<int, X...>) {
  (closure_of<X>(t, m, path, em), ...);
}

// One lower-star visit: apply the closures of the star's pending edges
// (linear over Z/2), keep the positive critical edges left as (v << 4 | x),
// and append the link edges left to the stage as updates of the target
// stars.  One dependent global load: the star's table row.  With `chain`
// set, a visit whose link edges all go to one target star hands that update
// back in *next instead of staging it, and the caller visits it at once (a
// star reached again later by another part of its mask is simply visited
// again: the projection is linear).
template <int SCAP>
__device__ __forceinline__ bool d1_visit(const D1Ctx& c, FEnt fe, const int32_t* snd, FEnt* stage, int* s_ntot,
                                         int* s_flag, unsigned long long* myouts, int& myout, int& updates, bool chain,
                                         FEnt* next, uint32_t* status) {
  uint32_t v = (uint32_t)fe.key;
  uint32_t m = fe.mask;
  if ((int64_t)v >= c.d.nv) {  // never for a valid entry: report and let the column be recomputed
    atomicOr(status, kErrInconsistent);
    atomicOr(s_flag, 1);
    return false;
  }
  D1Tab t;
  {
    const uint4* s4 = reinterpret_cast<const uint4*>(c.tab + v);
    uint4* d4 = reinterpret_cast<uint4*>(&t);
#pragma unroll
    for (int k = 0; k < 9; ++k) d4[k] = __ldg(s4 + k);
  }
  uint64_t path = 0;
  uint32_t em = 0;
  closures(t, m, path, em, std::make_integer_sequence<int, 14>{});
  em &= 0x3FFFu;
  if (em) {
    em &= ~__ldg(c.d0mask + v);  // negative critical edges are not rows
    for (; em; em &= em - 1) myouts[myout++] = ((unsigned long long)v << 4) | (unsigned)(__ffs(em) - 1);
  }
  uint32_t tmask[14];
#pragma unroll
  for (int k = 0; k < 14; ++k) tmask[k] = 0;
  link_targets(path & t.q[9], path & ~t.q[9], tmask, std::make_integer_sequence<int, 36>{});
  int cnt = 0, only = 0;
#pragma unroll
  for (int hn = 0; hn < 14; ++hn)
    if (tmask[hn]) {
      ++cnt;
      only = hn;
    }
  if (!cnt) return false;
  updates += cnt;
  if (chain && cnt == 1) {
    uint32_t hv = (uint32_t)((int32_t)v + snd[only]);
    next->key = star_key(t.nkey[only], hv);
    next->mask = tmask[only];
    next->pad = 0;
    return true;
  }
  int off = atomicAdd(s_ntot, cnt);
  if (off + cnt > SCAP) {
    atomicOr(s_flag, 1);
    return false;
  }
#pragma unroll
  for (int hn = 0; hn < 14; ++hn) {
    if (tmask[hn]) {
      uint32_t hv = (uint32_t)((int32_t)v + snd[hn]);
      FEnt e;
      e.key = star_key(t.nkey[hn], hv);
      e.mask = tmask[hn];
      e.pad = 0;
      stage[off++] = e;
      // the star is likely visited in a later round: bring its row to L2
      const char* row = reinterpret_cast<const char*>(c.tab + hv);
      asm volatile("prefetch.global.L2 [%0];" ::"l"(row));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(row + 128));
    }
  }
  return false;
}

// Sorts a stage of n <= SCAP entries (a[] holds SCAP entries, a power of
// two): in registers for up to two entries per thread (the usual case),
// else in shared memory (compact code: the unrolled networks for more
// entries per thread only crowd the instruction cache).
template <int GS, int SCAP>
__device__ void group_sort_stage(FEnt* a, int n) {
  static_assert(SCAP % GS == 0 && (SCAP & (SCAP - 1)) == 0, "a stage is a power of two");
  if (n <= GS) group_sort_reg<GS, 1>(a, n);
  else if (n <= 2 * GS && SCAP >= 2 * GS) group_sort_reg<GS, (SCAP >= 2 * GS ? 2 : 1)>(a, n);
  else group_sort_smem<GS>(a, n);
}

// New frontier from the untaken rest (front[nb..nf), descending) and the
// stage (ntot updates, any order): sort the stage, merge, combine equal keys.
// Returns the new frontier size.  All threads of the group call it.
template <int GS, int SCAP>
__device__ int group_combine(FEnt* front, int nb, int nf, FEnt* other, FEnt* stage, int ntot, int* scan_sm) {
  const int tid = gtid<GS>();
  int rest = nf - nb;
  group_sort_stage<GS, SCAP>(stage, ntot);
  int total = rest + ntot;
  for (int k = tid; k < total; k += GS) {  // merge path
    int lo = max(0, k - ntot), hi = min(k, rest);
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (front[nb + mid].key >= stage[k - mid - 1].key) lo = mid + 1;
      else hi = mid;
    }
    int i = lo, jb = k - lo;
    other[k] = (i < rest && (jb >= ntot || front[nb + i].key >= stage[jb].key)) ? front[nb + i] : stage[jb];
  }
  gsync<GS>();
  int kept = 0;
  for (int base = 0; base < total; base += GS) {
    int k = base + tid;
    int keep = 0;
    FEnt e;
    e.key = 0ull;
    e.mask = 0u;
    e.pad = 0u;
    if (k < total) {
      e = other[k];
      if (k == 0 || other[k - 1].key != e.key) {
        for (int q = k + 1; q < total && other[q].key == e.key; ++q) e.mask ^= other[q].mask;
        keep = e.mask != 0u;
      }
    }
    int t;
    int off = gscan<GS>(keep, t, scan_sm);
    if (keep) front[kept + off] = e;
    kept += t;
  }
  gsync<GS>();
  return kept;
}

// Visits one thread makes per round along a chain of single-target updates;
// room for the critical edges those visits keep; rounds of phase A before a
// column moves to a block.  The defaults depend on the diagram's size.  A
// large diagram (at least kLargeD1 critical triangles) keeps enough columns
// in flight in phase A to fill the GPU, so its columns stay there (no
// chaining, 128 rounds, 64 + 128 entries per column).  A small one gains
// from moving its long columns to 128-thread blocks early (chains of 2, 16
// rounds, 32 + 64 entries).  Measured, ms per iteration on the 256^3
// headline field (1.8 M critical triangles) / the 128^3 filament field
// (~0.25 M): large settings 64.7 / 2.89, small settings 67.8 / 1.89;
// 32 rounds with either tile lay in between on both (65.1-65.5 / 2.07-2.15).
constexpr int kOutCap = 28;
constexpr int kLargeD1 = 1 << 19;
constexpr int kChainLarge = 1, kRoundsLarge = 128;  // defaults of knobs 10 and 11, large diagrams
constexpr int kChainSmall = 2, kRoundsSmall = 16;   // ... small diagrams

// Round loop of one column.  Phase A (max_rounds > 0): every column, one
// group of GS threads (a half or a whole warp; NT / GS columns per block);
// a column still open after max_rounds, or whose frontier outgrows the
// group's buffers, saves its entries and is listed for phase B (NT = GS =
// 128, one block per listed column).  Groups of one block share nothing
// but the neighbour offsets and synchronise only among themselves.
template <int NT, int FCAP, int SCAP, int MINB = (NT == 32 ? 12 : 4), int GS = NT>
__global__ void __launch_bounds__(NT, MINB) k_d1_morse_group(D1Ctx c, D1Work W, int max_rounds, uint32_t* status) {
  static_assert(GS == NT || (NT == 32 && GS < 32), "several groups only within one warp");
  constexpr int G = NT / GS;
  const int ncols = W.flags[1];
  const int gi = (int)threadIdx.x / GS;
  extern __shared__ __align__(16) unsigned char smem[];
  FEnt* front = reinterpret_cast<FEnt*>(smem) + (size_t)gi * (2 * FCAP + SCAP);
  FEnt* other = front + FCAP;
  FEnt* stage = other + FCAP;
  __shared__ int32_t snd[16];
  __shared__ int scan_sm[16];  // GS/32 + 1 <= 16 (blocks only)
  __shared__ int sg_nf[G], sg_flag[G], sg_ntot[G], sg_otot[G];
  __shared__ Vec sg_out[G], sg_grow[G], sg_fr[G], sg_fr2[G];
  int& s_nf = sg_nf[gi];
  int& s_flag = sg_flag[gi];
  int& s_ntot = sg_ntot[gi];
  int& s_otot = sg_otot[gi];
  Vec& s_out = sg_out[gi];
  Vec& s_grow = sg_grow[gi];
  if (threadIdx.x < 14) snd[threadIdx.x] = c.nd.d[threadIdx.x];
  if (NT > 32) __syncthreads();
  else __syncwarp();  // snd is read by every group
  const bool phase_b = max_rounds <= 0;
  int j;
  if (phase_b) {
    if ((int)blockIdx.x >= *W.nbig) return;
    j = W.big[blockIdx.x];
  } else {
    j = (int)blockIdx.x * G + gi;
    if (j >= ncols) return;
  }
  const int tid = gtid<GS>();
  if (tid == 0) {
    s_flag = 0;
    s_nf = 0;
    s_ntot = 0;
    s_otot = 0;
    if (phase_b) {
      uint4 cs = W.cont[j];
      s_ntot = (int)cs.y;  // saved entries, combined below like a stage
      s_out.off = cs.z;
      s_out.size = cs.w;
      s_out.cap = W.cont_cap[j];
      s_out.h = W.pool + s_out.off;
    } else {
      if (!vec_alloc(W, s_out, 64, status)) s_flag = 1;
      // seed: the boundary of the critical triangle, each edge an entry of
      // the lower star of its higher endpoint
      uint32_t ve = c.L.c2_ve[W.cols[j]];
      uint32_t v0 = ve >> 6;
      int e0 = (int)(ve & 63u);
      uint32_t ea = (uint32_t)((int32_t)v0 + c.nd.d[c_geo.edge[e0][0]]);
      uint32_t eb = (uint32_t)((int32_t)v0 + c.nd.d[c_geo.edge[e0][1]]);
      uint32_t ends[3][2] = {{v0, ea}, {v0, eb}, {ea, eb}};
      for (int k = 0; k < 3; ++k) {
        uint32_t p = ends[k][0], q = ends[k][1];
        uint32_t rp = c.rank[p], rq = c.rank[q];
        uint32_t hi = rp > rq ? p : q, lo = rp > rq ? q : p;
        FEnt e;
        e.key = star_key(value_key(c.f[hi]), hi);
        e.mask = 1u << nbr_of_pair(c.d, hi, lo);
        e.pad = 0u;
        stage[s_ntot++] = e;
      }
    }
  }
  gsync<GS>();
  if (phase_b) {
    uint4 cs = W.cont[j];
    for (int i = tid; i < (int)cs.y; i += GS) stage[i] = fent_restore(W.pool + cs.x + 2 * (size_t)i);
  }
  gsync<GS>();
  {
    int n0 = group_combine<GS, SCAP>(front, 0, 0, other, stage, s_ntot, scan_sm);
    if (tid == 0) {
      s_nf = n0;
      s_ntot = 0;
    }
    gsync<GS>();
  }
  int visits = 0, updates = 0, rounds = 0;
  bool failed = s_flag != 0;
  bool handoff = false;
  while (!failed) {
    int nf = s_nf;
    if (nf == 0) break;
    if (!phase_b && rounds >= max_rounds) break;
    // every target is a lower neighbour of the visited vertex, so the
    // frontier's highest key drops each round: at most nv rounds
    if (rounds > c.d.nv) {
      if (tid == 0) atomicOr(status, kErrRounds);
      failed = true;
      break;
    }
    ++rounds;
    int nb = min(GS, nf);
    int myout = 0;
    unsigned long long myouts[kOutCap];
    if (tid < nb) {
      FEnt cur = front[tid];
      for (int k = 0;; ++k) {
        ++visits;
        FEnt nxt;
        bool more = k + 1 < c.chain && myout + 14 <= kOutCap;
        if (!d1_visit<SCAP>(c, cur, snd, stage, &s_ntot, &s_flag, myouts, myout, updates, more, &nxt, status))
          break;
        cur = nxt;
      }
    }
    int ooff = myout ? atomicAdd(&s_otot, myout) : 0;
    gsync<GS>();
    if (s_flag) {  // stage overflow: updates were dropped, recompute the column
      failed = true;
      break;
    }
    // outputs: append to the column's list in the pool (grown by the group)
    int otot = s_otot;
    if (otot > 0) {
      if (tid == 0) {
        s_grow.h = nullptr;
        if (s_out.size + otot > s_out.cap) {
          uint32_t cap = s_out.cap;
          while (cap < s_out.size + otot) cap *= 2;
          if (!vec_alloc(W, s_grow, cap, status)) {
            s_grow.h = nullptr;
            s_flag = 1;
          }
        }
      }
      gsync<GS>();
      if (s_flag) {
        failed = true;
        break;
      }
      if (s_grow.h) {
        for (uint32_t i = tid; i < s_out.size; i += GS) s_grow.h[i] = s_out.h[i];
        gsync<GS>();
        if (tid == 0) {
          s_grow.size = s_out.size;
          s_out = s_grow;
        }
        gsync<GS>();
      }
      for (int k = 0; k < myout; ++k) s_out.h[s_out.size + ooff + k] = myouts[k];
      gsync<GS>();
      if (tid == 0) {
        s_out.size += otot;
        s_otot = 0;
      }
    }
    int ntot = s_ntot;
    if (nf - nb + ntot > FCAP) {  // the new frontier would not fit
      handoff = !phase_b;
      failed = true;
      if (handoff) {  // phase A: the rest and the stage go to phase B as they are
        Vec& s_fr = sg_fr[gi];
        int rest = nf - nb;
        if (tid == 0 && !vec_alloc(W, s_fr, 2u * (uint32_t)(rest + ntot), status)) s_flag = 1;
        gsync<GS>();
        if (!s_flag) {
          for (int i = tid; i < rest; i += GS) fent_save(s_fr.h + 2 * i, front[nb + i]);
          for (int i = tid; i < ntot; i += GS) fent_save(s_fr.h + 2 * (rest + i), stage[i]);
          gsync<GS>();
          if (tid == 0) {
            W.cont[j] = make_uint4(s_fr.off, (uint32_t)(rest + ntot), s_out.off, s_out.size);
            W.cont_cap[j] = s_out.cap;
            W.big[atomicAdd(W.nbig, 1)] = j;
          }
        } else {
          handoff = false;
        }
      }
      break;
    }
    if (nf == nb && ntot <= GS) {
      // every entry is taken next round, so neither their order nor
      // combining equal keys matters (a star listed twice is visited twice
      // with parts of its mask: the projection is linear)
      for (int i = tid; i < ntot; i += GS) front[i] = stage[i];
      gsync<GS>();  // every thread has read s_ntot before it is reset
      if (tid == 0) {
        s_nf = ntot;
        s_ntot = 0;
      }
      gsync<GS>();
      continue;
    }
    gsync<GS>();
    int nn = group_combine<GS, SCAP>(front, nb, nf, other, stage, ntot, scan_sm);
    if (tid == 0) {
      s_nf = nn;
      s_ntot = 0;
    }
    gsync<GS>();
  }
  // visits and target updates of the whole group
  int vtot, utot;
  gscan<GS>(visits, vtot, scan_sm);
  gscan<GS>(updates, utot, scan_sm);
  if (handoff || (!failed && !phase_b && s_nf > 0)) {
    if (!handoff) {  // still open after max_rounds: save the frontier for phase B
      Vec& s_fr2 = sg_fr2[gi];
      if (tid == 0 && !vec_alloc(W, s_fr2, 2u * (uint32_t)s_nf, status)) s_flag = 1;
      gsync<GS>();
      if (s_flag) {
        if (tid == 0) {
          W.redo[j] = 1;
          W.hsize[j] = 0;
        }
        return;
      }
      for (int i = tid; i < s_nf; i += GS) fent_save(s_fr2.h + 2 * i, front[i]);
      gsync<GS>();
      if (tid == 0) {
        W.cont[j] = make_uint4(s_fr2.off, (uint32_t)s_nf, s_out.off, s_out.size);
        W.cont_cap[j] = s_out.cap;
        W.big[atomicAdd(W.nbig, 1)] = j;
      }
    }
    if (tid == 0) {
      W.redo[j] = 0;
      W.hsize[j] = 0;
      atomicAdd(&W.stats[0], (unsigned long long)vtot);
      atomicAdd(&W.stats[2], (unsigned long long)rounds);
      atomicAdd(&W.stats[4], (unsigned long long)utot);
    }
    return;
  }
  if (failed) {
    if (tid == 0) {
      W.redo[j] = 1;
      W.hsize[j] = 0;
    }
    return;
  }
  // finished: (v, x) -> C1 index, sort descending, keep the entries present
  // an odd number of times (Z/2)
  uint32_t nout = s_out.size;
  int n2 = 1;
  while (n2 < (int)nout) n2 <<= 1;
  unsigned long long* a = reinterpret_cast<unsigned long long*>(stage);
  if (n2 > 2 * SCAP) {  // too long for shared memory: sort in the pool
    if (tid == 0 && !vec_alloc(W, s_grow, (uint32_t)n2, status)) s_flag = 1;
    gsync<GS>();
    if (s_flag) {
      if (tid == 0) {
        W.redo[j] = 1;
        W.hsize[j] = 0;
      }
      return;
    }
    a = s_grow.h;
  }
  for (int i = tid; i < n2; i += GS) {
    unsigned long long ci = 0;
    if (i < (int)nout) {
      uint32_t v = (uint32_t)(s_out.h[i] >> 4);
      int x = (int)(s_out.h[i] & 15ull);
      int cnt = __popc(rec_crit_edges(ld_rec(c.rec, v)));
      uint32_t base = c.c1base[v];
      int found = -1;
      for (int k2 = 0; k2 < cnt; ++k2)
        if ((int)(c.L.c1_vn[base + k2] & 15u) == x) found = (int)(base + k2);
      if (found < 0) atomicOr(status, kErrInconsistent);
      ci = (unsigned long long)(found < 0 ? 0 : found);
    }
    a[i] = ci;
  }
  gsync<GS>();
  group_sort_desc<GS>(a, n2);
  int kept = 0;
  for (int base = 0; base < (int)nout; base += GS) {
    int k = base + tid;
    int keep = 0;
    unsigned long long x = 0;
    if (k < (int)nout) {
      x = a[k];
      if (k == 0 || a[k - 1] != x) {
        int e = k + 1;
        while (e < (int)nout && a[e] == x) ++e;
        keep = (e - k) & 1;
      }
    }
    int t;
    int off = gscan<GS>(keep, t, scan_sm);
    if (keep) s_out.h[kept + off] = x;
    kept += t;
  }
  gsync<GS>();
  if (tid == 0) {
    W.hoff[j] = s_out.off;
    W.hsize[j] = (uint32_t)kept;
    W.redo[j] = 0;
    atomicAdd(&W.stats[0], (unsigned long long)vtot);
    atomicMax(&W.stats[1], (unsigned long long)vtot);
    atomicAdd(&W.stats[2], (unsigned long long)rounds);
    atomicMax(&W.stats[3], (unsigned long long)rounds);
    atomicAdd(&W.stats[4], (unsigned long long)utot);
  }
}

// Phase A runs two columns per warp (half a warp each: a round visits ~9
// lower stars on average, so a whole warp left most lanes idle), keeps its
// shared memory small (4 KB per column) and its registers at 63 so that 28
// one-warp blocks, 56 columns, share an SM: the rounds are latency-bound.  A visit appends 1.1 updates on average, 14 at most; a
// column that outgrows the buffers continues in phase B.
constexpr int kThreadsB = 128;
constexpr int kFrontA = 64, kStageA = 128;
constexpr int kFrontH = 32, kStageH = 64;
constexpr int kFrontQ = 16, kStageQ = 32;
constexpr int kFrontB = 1024, kStageB = 1024;
static_assert(kFrontA + kStageA <= kStageB, "a phase A handoff fits phase B's stage");

static size_t d1_group_smem(int fcap, int scap) { return (2 * (size_t)fcap + scap) * sizeof(FEnt); }

// Phase 2 (one block): reduce the Morse boundaries, smallest column owning
// each low; every addition is of an earlier column.  Rounds of two phases:
// every listed column claims its low (atomicMin), then every listed column
// that does not own its low adds the owner's column (owners do not change in
// that phase) and is listed again.  A settled owner that a smaller column
// displaces is listed for the next round; columns not listed own their lows
// and stay as they are, so a round costs as much as its list.
// Number of entries of a strictly decreasing column greater than v.
// Loads of column entries: from L2 when other SMs may have written them in
// this kernel (CG), plain otherwise.
template <bool CG>
__device__ __forceinline__ unsigned long long d1_ld(const unsigned long long* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

template <bool CG = false>
__device__ __forceinline__ uint32_t d1_count_greater(unsigned long long v, const unsigned long long* arr,
                                                    uint32_t len) {
  uint32_t lo = 0, hi = len;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (d1_ld<CG>(arr + mid) > v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// One warp writes the sum over Z/2 of two strictly decreasing columns a (n)
// and b (nb) to d, decreasing, and returns its length.  An entry x of a that
// b lacks lands at x + (entries of b above it) - 2 (entries of a above it
// that b also has): everything above it, minus the cancelled pairs.  Same
// for b.  Positions outside [0, n + nb) set kErrInconsistent.
template <bool CG = false>
__device__ uint32_t d1_warp_add(const unsigned long long* a, uint32_t n, const unsigned long long* b, uint32_t nb,
                                unsigned long long* d, uint32_t* status) {
  const int lane = threadIdx.x & 31;
  const uint32_t cap = n + nb;
  uint32_t common = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const unsigned long long* p = pass == 0 ? a : b;
    const unsigned long long* q = pass == 0 ? b : a;
    const uint32_t np_ = pass == 0 ? n : nb, nq = pass == 0 ? nb : n;
    uint32_t before = 0;
    for (uint32_t x0 = 0; x0 < np_; x0 += 32) {
      const uint32_t x = x0 + lane;
      bool found = false;
      uint32_t c = 0;
      unsigned long long v = 0;
      if (x < np_) {
        v = d1_ld<CG>(p + x);
        c = d1_count_greater<CG>(v, q, nq);
        found = c < nq && d1_ld<CG>(q + c) == v;
      }
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, found);
      if (x < np_ && !found) {
        const uint32_t pos = x + c - 2u * (before + __popc(bal & ((1u << lane) - 1u)));
        if (pos < cap) d[pos] = v;
        else atomicOr(status, kErrInconsistent);
      }
      before += __popc(bal);
    }
    common = before;
  }
  return cap - 2u * common;
}

constexpr int kChainMax = 64;      // active columns up to which a round chains additions (default of knob 12)
constexpr int kChainLimit = 1024;  // ... at most
constexpr int kChainSteps = 1 << 16;  // chained additions of one column in one round, at most
constexpr uint32_t kLongAdd = 64;  // column additions at least this long run on a warp
constexpr int kLongCap = 1024;     // ... at most this many per round (the rest on one thread)

__device__ __forceinline__ void d1_list_push(int32_t* next, int* n_next, int32_t* mark, int j, int round) {
  if (atomicExch(&mark[j], round) != round) next[atomicAdd(n_next, 1)] = j;
}

// Chained additions of the short rounds in shared memory.  The block splits
// into G groups of kUFT / G threads (G = 32 while more than 8 columns chain,
// then 8, 4, 2, 1); a group keeps the column it reduces in shared memory
// (32-bit entries: C1 indices are below 2^31) for up to kSubSteps
// additions.  Each step loads only the owner's column (one coalesced read),
// adds it to the group's copy there and writes the column back to the pool
// when it stops.  Nobody else reads a column that does not own its low, so
// the pool copy may lag behind until then.  The owner of the next low is
// looked up while the group adds: the next low is the first entry of the
// two columns that the other lacks, past the cancelled common top.  Columns
// still chaining after kSubSteps additions go on in the next sub-round;
// with fewer columns left, groups grow and their buffers with them.  A sum
// longer than the group's buffers is added in the pool by its first warp
// instead (d1_warp_add).
constexpr int kCGroupsMax = kUFT / 32;                   // groups of one warp
constexpr uint32_t kCBufWords = 49152;                   // 32-bit buffer entries of the block
constexpr size_t kChainSmem = (size_t)kCBufWords * sizeof(uint32_t);
constexpr int kSubSteps = 64;                            // chained additions of one column per sub-round
constexpr uint32_t kCCap = kCBufWords / (3 * kCGroupsMax);  // entries per buffer with one warp per column (512)

// Barrier of group g (gs threads): the warp itself, or named barrier g + 1
// (groups of several warps: at most 8 of them).
__device__ __forceinline__ void cg_bar(int g, int gs) {
  if (gs == 32) __syncwarp();
  else asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(gs) : "memory");
}

// d = a (n) + b (nb) over Z/2 by group g (gs threads), all in shared memory,
// strictly decreasing.  Merge path: thread t walks positions [t*per,
// (t+1)*per) of the merged order (ties: a first, so a common entry is a[i]
// directly followed by b[j]); an entry is cancelled when the other column
// holds it, which each thread sees from its neighbour in the walk (b[j] from
// a[i-1], a[i] from b[j]).  A counting walk, a group scan (warp shuffles,
// then one warp over the warp totals in wsum: gs / 32 + 1 ints), then the
// writing walk.  Returns the length of d; the group sees d complete.
__device__ uint32_t group_merge_add(const uint32_t* a, uint32_t n, const uint32_t* b, uint32_t nb, uint32_t* d,
                                    int g, int gt, int gs, int* wsum) {
  const int lane = gt & 31, w = gt >> 5, nw = gs >> 5;
  const uint32_t N = n + nb, per = (N + (uint32_t)gs - 1) / (uint32_t)gs;
  const uint32_t k0 = min(N, (uint32_t)gt * per), k1 = min(N, k0 + per);
  // split: i = entries of a among the first k0 of the merged order
  uint32_t lo = k0 > nb ? k0 - nb : 0u, hi = min(k0, n);
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] >= b[k0 - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  const uint32_t i0 = lo, j0 = k0 - lo;
  uint32_t cnt = 0, base = 0, total = 0;
  for (int pass = 0; pass < 2; ++pass) {
    uint32_t i = i0, j = j0, out = 0;
    if (pass == 1) {
      uint32_t inc = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += t;
      }
      if (nw == 1) {
        total = __shfl_sync(0xFFFFFFFFu, inc, 31);
      } else {
        if (lane == 31) wsum[w] = (int)inc;
        cg_bar(g, gs);
        if (w == 0) {
          const uint32_t v = lane < nw ? (uint32_t)wsum[lane] : 0u;
          uint32_t vi = v;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, vi, o);
            if (lane >= o) vi += t;
          }
          if (lane < nw) wsum[lane] = (int)(vi - v);
          if (lane == 31) wsum[nw] = (int)vi;
        }
        cg_bar(g, gs);
        base = (uint32_t)wsum[w];
        total = (uint32_t)wsum[nw];
      }
      out = base + inc - cnt;
    }
    uint32_t ai = i < n ? a[i] : 0u, bj = j < nb ? b[j] : 0u, ap = i > 0 ? a[i - 1] : 0xFFFFFFFFu;
    for (uint32_t k = k0; k < k1; ++k) {
      bool cancel;
      uint32_t v;
      if (i < n && (j >= nb || ai >= bj)) {
        v = ai;
        cancel = j < nb && ai == bj;
        ap = ai;
        ++i;
        ai = i < n ? a[i] : 0u;
      } else {
        v = bj;
        cancel = i > 0 && ap == bj;
        ++j;
        bj = j < nb ? b[j] : 0u;
      }
      if (!cancel) {
        if (pass == 1) d[out] = v;
        ++out;
      }
    }
    if (pass == 0) cnt = out;
  }
  cg_bar(g, gs);  // d complete; wsum free again
  return total;
}

// Writes the group's copy of column j (n entries) to fresh pool space;
// false when the pool is full (the status word says so).
__device__ bool cg_write_back(D1Work& W, int j, const uint32_t* col, uint32_t n, int g, int gt, int gs, int* ctl,
                              uint32_t* status) {
  if (gt == 0) {
    const uint32_t off = atomicAdd(W.pool_head, n);
    const bool ok = (unsigned long long)off + n <= W.pool_cap;
    if (!ok) atomicOr(status, kErrPool);
    ctl[3] = ok ? (int)off : -1;
  }
  cg_bar(g, gs);
  const int off = ctl[3];
  if (off >= 0) {
    for (uint32_t i = gt; i < n; i += (uint32_t)gs) W.pool[(uint32_t)off + i] = col[i];
    if (gt == 0) {
      W.hoff[j] = (uint32_t)off;
      W.hsize[j] = n;
    }
  }
  cg_bar(g, gs);
  return off >= 0;
}

// ctl[0..2] = the owner of a low (as the group leader loaded its index and
// {index, pool offset, length} record), its column's offset and length.
__device__ __forceinline__ void cg_publish(const D1Work& W, int j, int o, const uint4& r, int* ctl, uint32_t* status) {
  // an owner writes its record before it is read, and its column lies in the pool
  if (o != j && o != 0x7FFFFFFF && o < j &&
      (r.x != (uint32_t)o || r.z == 0u || (unsigned long long)r.y + r.z > W.pool_cap)) {
    atomicOr(status, kErrInconsistent);
    o = j;
  }
  ctl[0] = o;
  ctl[1] = (int)r.z;
  ctl[2] = (int)r.y;
}

// Up to kSubSteps chained additions of column j by group g (gs threads);
// buf holds its three buffers of cap entries.  Returns true when the column
// is still chaining (it goes on in the next sub-round); adds = the additions
// made.
__device__ bool cg_chain(D1Work& W, int n1, int j, int round, uint32_t* buf, uint32_t cap, int g, int gt, int gs,
                         int* wsum, int* ctl, int32_t* nxt, int* s_nb, int32_t* mark, int& adds, uint32_t* status) {
  uint32_t* A = buf;
  uint32_t* B = buf + cap;
  uint32_t* D = buf + 2 * (size_t)cap;
  uint32_t n = W.hsize[j];
  bool in_smem = false, dirty = false, more = false;
  adds = 0;
  if (n == 0 || (unsigned long long)W.hoff[j] + n > W.pool_cap) {  // a listed column is never empty
    if (gt == 0) atomicOr(status, kErrInconsistent);
    return false;
  }
  if (n <= cap) {
    const unsigned long long* a = W.pool + W.hoff[j];
    for (uint32_t i = gt; i < n; i += (uint32_t)gs) A[i] = (uint32_t)a[i];
    in_smem = true;
  }
  cg_bar(g, gs);
  if (gt == 0) {
    const uint32_t low = in_smem ? A[0] : (uint32_t)W.pool[W.hoff[j]];
    if (low < (uint32_t)n1) {
      cg_publish(W, j, W.owner[low], W.orec[low], ctl, status);
    } else {
      atomicOr(status, kErrInconsistent);
      ctl[0] = j;
    }
  }
  cg_bar(g, gs);
  for (int step = 0;; ++step) {
    const int o = ctl[0];
    const uint32_t no = (uint32_t)ctl[1], ob = (uint32_t)ctl[2];
    if (o == j) break;
    if (o == 0x7FFFFFFF || o > j) {
      if (gt == 0) d1_list_push(nxt, s_nb, mark, j, round);
      break;
    }
    if (step >= kSubSteps) {
      more = true;
      break;
    }
    const uint32_t sum = n + no;
    uint32_t m;
    if (in_smem && sum <= cap) {
      const unsigned long long* b = W.pool + ob;
      for (uint32_t i = gt; i < no; i += (uint32_t)gs) B[i] = (uint32_t)b[i];
      cg_bar(g, gs);  // B loaded; every thread has read ctl
      // the leader finds the next low and loads its owner while the group adds
      int o_next = j;
      uint4 r_next = make_uint4(0u, 0u, 0u, 0u);
      uint32_t nl = 0;
      if (gt == 0) {
        uint32_t x = 1, y = 1;
        while (x < n && y < no && A[x] == B[y]) {
          ++x;
          ++y;
        }
        if (x < n || y < no) {  // else the sum is empty: stop (reported below)
          nl = (y >= no || (x < n && A[x] > B[y])) ? A[x] : B[y];
          if (nl < (uint32_t)n1) {
            o_next = W.owner[(int)nl];
            r_next = W.orec[(int)nl];
          }
        }
      }
      m = group_merge_add(A, n, B, no, D, g, gt, gs, wsum);
      if (gt == 0) {
        if (m > 0 && (D[0] != nl || A[0] != B[0] || nl >= (uint32_t)n1)) {  // the sum's low is the one looked up
          atomicOr(status, kErrInconsistent);
          o_next = j;
        }
        cg_publish(W, j, o_next, r_next, ctl, status);
      }
      cg_bar(g, gs);
      uint32_t* t = A;
      A = D;
      D = t;
      dirty = true;
    } else {
      if (in_smem && dirty && !cg_write_back(W, j, A, n, g, gt, gs, ctl, status)) return false;
      in_smem = false;
      dirty = false;
      if (gt < 32) {
        uint32_t off = 0;
        if (gt == 0) off = atomicAdd(W.pool_head, sum);
        off = __shfl_sync(0xFFFFFFFFu, off, 0);
        if ((unsigned long long)off + sum > W.pool_cap) {
          if (gt == 0) {
            atomicOr(status, kErrPool);
            ctl[3] = -1;
          }
        } else {
          const uint32_t mm = d1_warp_add(W.pool + W.hoff[j], n, W.pool + ob, no, W.pool + off, status);
          if (gt == 0) {
            W.hoff[j] = off;
            W.hsize[j] = mm;
            ctl[3] = (int)mm;
          }
        }
      }
      cg_bar(g, gs);
      if (ctl[3] < 0) return false;  // the pool is full: the status word says so
      m = (uint32_t)ctl[3];
      cg_bar(g, gs);  // every thread has read ctl[3]
      if (m > 0 && m <= cap) {  // back into shared memory
        const unsigned long long* a = W.pool + W.hoff[j];
        for (uint32_t i = gt; i < m; i += (uint32_t)gs) A[i] = (uint32_t)a[i];
        in_smem = true;
      }
      if (gt == 0 && m > 0) {
        const uint32_t low = (uint32_t)W.pool[W.hoff[j]];
        if (low < (uint32_t)n1) {
          cg_publish(W, j, W.owner[low], W.orec[low], ctl, status);
        } else {
          atomicOr(status, kErrInconsistent);
          ctl[0] = j;
        }
      }
      cg_bar(g, gs);
    }
    n = m;
    ++adds;
    if (gt == 0) {
      atomicAdd(&W.stats[6], (unsigned long long)m);
      atomicMax(&W.stats[7], (unsigned long long)m);
      if (m == 0) atomicOr(status, kErrEmptyColumn);
    }
    if (m == 0) break;
  }
  if (in_smem && dirty) cg_write_back(W, j, A, n, g, gt, gs, ctl, status);
  return more;
}

// `ctl` (may be null): resume after k_d1_reduce_grid from its lists, owners
// and marks.
__global__ void __launch_bounds__(kUFT) k_d1_reduce(D1Work W, int n1, int32_t* d1_edge, const D1Ctl* ctl,
                                                    uint32_t ccap, int chain_max, uint32_t* status) {
  const int ncols = W.flags[1];
  // free per-column scratch by now: two lists and a "listed in round" mark
  int32_t* listA = W.lowc;
  int32_t* listB = reinterpret_cast<int32_t*>(W.hcap);
  int32_t* mark = W.redo;
  __shared__ int s_na, s_nb, s_nlong;
  __shared__ int32_t s_long[kLongCap];
  __shared__ int32_t s_sub[2][kChainLimit], s_subn[2][kChainLimit];
  __shared__ int s_cg[kCGroupsMax][4];
  __shared__ int s_wsum[2 * kCGroupsMax];
  __shared__ int s_nsub;
  int32_t* cur = listA;
  int32_t* nxt = listB;
  int round0 = 0;
  if (ctl) {
    // the whole-GPU rounds gave up (a barrier, the round bound or the pool):
    // their lists may be partly written, so nothing resumes from them
    if (*reinterpret_cast<const volatile uint32_t*>(status) & (kErrSpin | kErrRounds | kErrPool)) return;
    if (ctl->which) {
      cur = listB;
      nxt = listA;
    }
    if (threadIdx.x == 0) s_na = ctl->n[ctl->which];
    round0 = ctl->rounds;
  } else {
    // an earlier stage failed (its results are discarded): nothing to reduce
    if (*reinterpret_cast<const volatile uint32_t*>(status) & (kErrSpin | kErrRounds | kErrPool | kErrTrace)) return;
    for (int k = threadIdx.x; k < n1; k += kUFT) W.owner[k] = 0x7FFFFFFF;
    if (threadIdx.x == 0) s_na = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < ncols; j += kUFT) {
      mark[j] = -1;
      if (W.hsize[j] > 0) listA[atomicAdd(&s_na, 1)] = j;
    }
  }
  __syncthreads();
  const long long c_start = clock64();
  long long c_round = c_start;
  for (int round = round0;; ++round) {
    int na = s_na;
    if (na == 0) break;
    if (round > ncols + 2) {
      if (threadIdx.x == 0) atomicOr(status, kErrRounds);
      break;
    }
    if (threadIdx.x == 0) {
      s_nb = 0;
      s_nlong = 0;
      c_round = clock64();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < na; i += kUFT) {
      int j = cur[i];
      int old = atomicMin(&W.owner[(int)W.pool[W.hoff[j]]], j);
      if (old > j && old != 0x7FFFFFFF) d1_list_push(nxt, &s_nb, mark, old, round);  // displaced owner
    }
    __syncthreads();
    if (na <= chain_max) {
      // short list: chained additions by groups of threads, in sub-rounds
      // (in shared memory while a sum fits the group's buffers).  During this
      // phase every owner owns its low and does not change (a column that
      // does not own its low holds no owner entry), so after adding its
      // owner a column may go on adding the owner of its new low while that
      // owner is an earlier column: each step is still a left-to-right
      // addition.  It stops when it owns its low, or the low's owner is
      // later or absent (it claims the low next round).
      extern __shared__ __align__(16) uint32_t chain_buf[];
      // owner records of this round's new owners, before any column reads one
      for (int i = threadIdx.x; i < na; i += kUFT) {
        const int j = cur[i];
        const int low = (int)W.pool[W.hoff[j]];
        if (W.owner[low] == j) W.orec[low] = make_uint4((uint32_t)j, W.hoff[j], W.hsize[j], 0u);
      }
      for (int i = threadIdx.x; i < na; i += kUFT) {
        s_sub[0][i] = cur[i];
        s_subn[0][i] = 0;
      }
      if (threadIdx.x == 0) s_nsub = na;
      __syncthreads();
      for (int sub = 0, which = 0;; ++sub, which ^= 1) {
        const int ns = s_nsub;
        if (ns == 0) break;
        __syncthreads();  // every thread has read s_nsub
        if (sub >= kChainSteps / kSubSteps) {  // bounded: the rest claim their lows next round
          for (int i = threadIdx.x; i < ns; i += kUFT) d1_list_push(nxt, &s_nb, mark, s_sub[which][i], round);
          break;
        }
        if (threadIdx.x == 0) s_nsub = 0;
        __syncthreads();
        // groups: one warp per column while more than 8 columns are left,
        // then the next power of two of the columns left
        const int G = ns > 8 ? kCGroupsMax : ns > 4 ? 8 : ns > 2 ? 4 : ns;
        const int gs = kUFT / G, g = threadIdx.x / gs, gt = threadIdx.x % gs;
        const uint32_t gbuf = kCBufWords / (3u * (uint32_t)G);
        const uint32_t cap = min(gbuf, ccap * (uint32_t)(kCGroupsMax / G));
        for (int q = g; q < ns; q += G) {
          int adds = 0;
          const int j = s_sub[which][q];
          const bool more = cg_chain(W, n1, j, round, chain_buf + (size_t)g * 3 * gbuf, cap, g, gt, gs,
                                     s_wsum + g * ((gs >> 5) + 1), s_cg[g], nxt, &s_nb, mark, adds, status);
          if (gt == 0) {
            const int total = s_subn[which][q] + adds;
            atomicAdd(&W.stats[11], (unsigned long long)adds);
            if (more) {
              const int k = atomicAdd(&s_nsub, 1);
              s_sub[which ^ 1][k] = j;
              s_subn[which ^ 1][k] = total;
            } else {
              atomicMax(&W.stats[12], (unsigned long long)total);
            }
          }
        }
        __syncthreads();
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        s_na = s_nb;
        W.stats[5] = (unsigned long long)(round + 1);
        W.stats[13] += 1;  // short rounds and their cycles
        W.stats[14] += (unsigned long long)(clock64() - c_round);
      }
      int32_t* t = cur;
      cur = nxt;
      nxt = t;
      __syncthreads();
      continue;
    }
    for (int i = threadIdx.x; i < na; i += kUFT) {
      int j = cur[i];
      uint32_t n = W.hsize[j];
      const unsigned long long* a = W.pool + W.hoff[j];
      int o = W.owner[(int)a[0]];
      if (o == j) {  // owns its low: its record for the short rounds
        W.orec[(int)a[0]] = make_uint4((uint32_t)j, W.hoff[j], n, 0u);
        continue;
      }
      uint32_t no = W.hsize[o];
      if (n + no >= kLongAdd) {  // long: one warp adds it below
        const int q = atomicAdd(&s_nlong, 1);
        if (q < kLongCap) {
          s_long[q] = j;
          continue;
        }
      }
      const unsigned long long* b = W.pool + W.hoff[o];
      uint32_t cap = n + no;
      uint32_t off = atomicAdd(W.pool_head, cap);
      if ((unsigned long long)off + cap > W.pool_cap) {
        atomicOr(status, kErrPool);
        continue;
      }
      unsigned long long* d = W.pool + off;
      uint32_t x = 0, y = 0, m = 0;
      while (x < n && y < no) {  // both decreasing: symmetric difference
        if (a[x] > b[y]) d[m++] = a[x++];
        else if (b[y] > a[x]) d[m++] = b[y++];
        else {
          ++x;
          ++y;
        }
      }
      while (x < n) d[m++] = a[x++];
      while (y < no) d[m++] = b[y++];
      W.hoff[j] = off;
      W.hsize[j] = m;
      atomicAdd(&W.stats[6], (unsigned long long)m);  // entries written by merges
      atomicMax(&W.stats[7], (unsigned long long)m);  // longest merged column
      if (m == 0) atomicOr(status, kErrEmptyColumn);
      else d1_list_push(nxt, &s_nb, mark, j, round);
    }
    __syncthreads();
    {  // the long additions, one warp each
      const int nlong = min(s_nlong, kLongCap), lane = threadIdx.x & 31;
      for (int q = threadIdx.x >> 5; q < nlong; q += kUFT / 32) {
        const int j = s_long[q];
        const uint32_t n = W.hsize[j];
        const unsigned long long* a = W.pool + W.hoff[j];
        const int o = W.owner[(int)a[0]];
        const uint32_t no = W.hsize[o];
        const unsigned long long* b = W.pool + W.hoff[o];
        const uint32_t cap = n + no;
        uint32_t off = 0;
        if (lane == 0) off = atomicAdd(W.pool_head, cap);
        off = __shfl_sync(0xFFFFFFFFu, off, 0);
        if ((unsigned long long)off + cap > W.pool_cap) {
          if (lane == 0) atomicOr(status, kErrPool);
          continue;
        }
        const uint32_t m = d1_warp_add(a, n, b, no, W.pool + off, status);
        if (lane == 0) {
          W.hoff[j] = off;
          W.hsize[j] = m;
          atomicAdd(&W.stats[6], (unsigned long long)m);
          atomicMax(&W.stats[7], (unsigned long long)m);
          if (m == 0) atomicOr(status, kErrEmptyColumn);
          else d1_list_push(nxt, &s_nb, mark, j, round);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_na = s_nb;
      W.stats[5] = (unsigned long long)(round + 1);  // rounds so far
      if (na >= 4096) {  // rounds with many active columns and their cycles
        W.stats[8] += 1;
        W.stats[9] += (unsigned long long)(clock64() - c_round);
      }
    }
    int32_t* t = cur;
    cur = nxt;
    nxt = t;
    __syncthreads();
  }
  if (threadIdx.x == 0) W.stats[10] += (unsigned long long)(clock64() - c_start);
  for (int j = threadIdx.x; j < ncols; j += kUFT)
    d1_edge[W.cols[j]] = W.hsize[j] > 0 ? (int)W.pool[W.hoff[j]] : -1;
}

// Candidate columns in increasing triangle order; their number stays on the
// device (W.flags[1]), the later D1 launches are sized by n2.
void launch_d1_prepare(int n2, D1Work& W, PairOut& P, cudaStream_t st) {
  if (n2 == 0) {
    cudaMemsetAsync(W.flags + 1, 0, sizeof(int32_t), st);
    return;
  }
  uint32_t* flag = reinterpret_cast<uint32_t*>(W.lowc);  // scratch (n2 entries available)
  uint32_t* pos = reinterpret_cast<uint32_t*>(W.hsize);
  uint32_t* sums = reinterpret_cast<uint32_t*>(W.hcap);
  k_d1_select<<<(n2 + 255) / 256, 256, 0, st>>>(n2, P.d2_max, flag); note_launch();
  exclusive_scan_u32(flag, pos, n2, sums, st);
  k_d1_gather<<<(n2 + 255) / 256, 256, 0, st>>>(n2, flag, pos, W.cols, P.d1_edge, W.flags + 1); note_launch();
}

void launch_d1_morse(const Dims& d, const NbrDelta& nd, const CritLists& L, int n1, int n2, const uint32_t* rank,
                     const uint32_t* order, const float* f, const Rec* rec, const D1Tab* tab, const uint32_t* c1base,
                     D1Work& W, PairOut& P, uint32_t* status, cudaStream_t st) {
  if (n2 == 0) return;
  D1Ctx c;
  c.d = d;
  c.nd = nd;
  c.rank = rank;
  c.order = order;
  c.rec = rec;
  c.tab = tab;
  c.c1base = c1base;
  c.L = L;
  c.d0_killed = P.d0_killed;
  c.d0mask = P.d0mask;
  c.f = f;
  {
    const int64_t ch = g_morse_chain.load();
    c.chain = ch > 0 ? (int)std::min<int64_t>(ch, 8) : (n2 >= kLargeD1 ? kChainLarge : kChainSmall);
  }
  const int64_t mr = g_morse_rounds.load();
  const int roundsA =
      mr > 0 ? (int)std::min<int64_t>(mr, 1 << 20) : (n2 >= kLargeD1 ? kRoundsLarge : kRoundsSmall);
  cudaMemsetAsync(W.pool_head, 0, 4, st);
  cudaMemsetAsync(W.stats, 0, kD1Stats * sizeof(unsigned long long), st);
  cudaMemsetAsync(W.nbig, 0, sizeof(int32_t), st);
  size_t sb = d1_group_smem(kFrontB, kStageB);
  int dev = 0;
  cudaGetDevice(&dev);
  static std::atomic<bool> attr[64] = {};  // fields may be driven from several host threads
  if (dev >= 0 && dev < 64 && !attr[dev].load(std::memory_order_acquire)) {
    cudaFuncSetAttribute(k_d1_morse_group<32, kFrontA, kStageA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)d1_group_smem(kFrontA, kStageA));
    cudaFuncSetAttribute(k_d1_morse_group<32, kFrontA * 2, kStageA * 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)d1_group_smem(kFrontA * 2, kStageA * 2));
    cudaFuncSetAttribute(k_d1_morse_group<32, kFrontA * 4, kStageA * 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)d1_group_smem(kFrontA * 4, kStageA * 4));
    cudaFuncSetAttribute(k_d1_morse_group<32, kFrontA, kStageA, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)d1_group_smem(kFrontA, kStageA));
    cudaFuncSetAttribute(k_d1_morse_group<32, kFrontA, kStageA, 32, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(2 * d1_group_smem(kFrontA, kStageA)));
    cudaFuncSetAttribute(k_d1_morse_group<32, kFrontH, kStageH, 32, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(2 * d1_group_smem(kFrontH, kStageH)));
    cudaFuncSetAttribute(k_d1_morse_group<32, kFrontQ, kStageQ, 32, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(4 * d1_group_smem(kFrontQ, kStageQ)));
    cudaFuncSetAttribute(k_d1_morse_group<kThreadsB, kFrontB, kStageB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sb);
    attr[dev].store(true, std::memory_order_release);
  }
  // phase A buffers: the default, or 2x / 4x larger (more shared memory per
  // warp, fewer warps per SM; a column that outgrows them continues in
  // phase B)
  // knob 7 = 0: the larger tile for large diagrams, the smaller one otherwise
  int64_t phase_a = g_d1_phase_a.load();
  if (phase_a == 0 && n2 < kLargeD1) phase_a = 5;
  switch (phase_a) {
    case 1:
      k_d1_morse_group<32, kFrontA * 2, kStageA * 2><<<n2, 32, d1_group_smem(kFrontA * 2, kStageA * 2), st>>>(
          c, W, roundsA, status);
      break;
    case 2:
      k_d1_morse_group<32, kFrontA * 4, kStageA * 4><<<n2, 32, d1_group_smem(kFrontA * 4, kStageA * 4), st>>>(
          c, W, roundsA, status);
      break;
    case 3:  // one warp per column without the register cap
      k_d1_morse_group<32, kFrontA, kStageA><<<n2, 32, d1_group_smem(kFrontA, kStageA), st>>>(c, W, roundsA,
                                                                                             status);
      break;
    case 4:  // one warp per column, registers capped (63) so that 32 warps fit an SM
      k_d1_morse_group<32, kFrontA, kStageA, 32><<<n2, 32, d1_group_smem(kFrontA, kStageA), st>>>(c, W, roundsA,
                                                                                                  status);
      break;
    case 5:  // half a warp per column with the smaller tile
      k_d1_morse_group<32, kFrontH, kStageH, 32, 16><<<(n2 + 1) / 2, 32, 2 * d1_group_smem(kFrontH, kStageH), st>>>(
          c, W, roundsA, status);
      break;
    case 6:  // a quarter of a warp per column with the smallest tile
      k_d1_morse_group<32, kFrontQ, kStageQ, 32, 8><<<(n2 + 3) / 4, 32, 4 * d1_group_smem(kFrontQ, kStageQ), st>>>(
          c, W, roundsA, status);
      break;
    default:  // (0, 7) half a warp per column (two columns per warp), registers capped for 32 warps per SM
      k_d1_morse_group<32, kFrontA, kStageA, 32, 16><<<(n2 + 1) / 2, 32, 2 * d1_group_smem(kFrontA, kStageA), st>>>(
          c, W, roundsA, status);
  }
  note_launch();
  k_d1_morse_group<kThreadsB, kFrontB, kStageB><<<n2, kThreadsB, sb, st>>>(c, W, 0, status); note_launch();
  k_d1_morse<<<(n2 + 63) / 64, 64, 0, st>>>(c, W, status); note_launch();
}

// The same rounds over the whole GPU (cooperative launch, grid barriers
// between the phases) while at least `handoff` columns are active; then
// k_d1_reduce resumes from ctl on one block.  Any schedule of these rounds
// gives a left-to-right reduction with the same pivots; list order, pool
// offsets and which SM adds what do not change the pairs.  Every read of
// state that another SM may have written in this kernel goes to L2.
__global__ void __launch_bounds__(kUFT) k_d1_reduce_grid(D1Work W, int n1, D1Ctl* ctl, int handoff, unsigned limit,
                                                         uint32_t* status) {
  const int ncols = W.flags[1];
  int32_t* listA = W.lowc;
  int32_t* listB = reinterpret_cast<int32_t*>(W.hcap);
  int32_t* mark = W.redo;
  __shared__ int s_nlong;
  __shared__ int32_t s_long[kLongCap];
  const unsigned nb = gridDim.x;
  const int gt = blockIdx.x * kUFT + threadIdx.x, gn = nb * kUFT;
  const long long c_start = clock64();
  // an earlier stage failed (its results are discarded): every block returns
  // before the first barrier, and the resuming block sees the same bits
  if (*reinterpret_cast<const volatile uint32_t*>(status) & (kErrSpin | kErrRounds | kErrPool | kErrTrace)) return;
  for (int k = gt; k < n1; k += gn) W.owner[k] = 0x7FFFFFFF;
  for (int j = gt; j < ncols; j += gn) {
    mark[j] = -1;
    if (W.hsize[j] > 0) listA[atomicAdd(&ctl->n[0], 1)] = j;
  }
  if (!grid_barrier(ctl->bar, nb, status, limit)) return;
  int which = 0;
  for (int round = 0;; ++round) {
    const int na = *reinterpret_cast<volatile int*>(&ctl->n[which]);
    if (na == 0 || na < handoff) break;
    if (round > ncols + 2) {
      if (gt == 0) atomicOr(status, kErrRounds);
      break;
    }
    const long long c_round = clock64();
    const int32_t* cur = which ? listB : listA;
    int32_t* nxt = which ? listA : listB;
    int* n_next = &ctl->n[which ^ 1];
    if (threadIdx.x == 0) s_nlong = 0;
    for (int i = gt; i < na; i += gn) {
      const int j = __ldcg(&cur[i]);
      const int old = atomicMin(&W.owner[(int)__ldcg(&W.pool[__ldcg(&W.hoff[j])])], j);
      if (old > j && old != 0x7FFFFFFF) d1_list_push(nxt, n_next, mark, old, round);  // displaced owner
    }
    if (!grid_barrier(ctl->bar, nb, status, limit)) return;
    for (int i = gt; i < na; i += gn) {
      const int j = __ldcg(&cur[i]);
      const uint32_t n = __ldcg(&W.hsize[j]);
      const unsigned long long* a = W.pool + __ldcg(&W.hoff[j]);
      const int o = __ldcg(&W.owner[(int)__ldcg(a)]);
      if (o == j) {  // owns its low: its record for the short rounds
        W.orec[(int)__ldcg(a)] = make_uint4((uint32_t)j, __ldcg(&W.hoff[j]), n, 0u);
        continue;
      }
      const uint32_t no = __ldcg(&W.hsize[o]);
      if (n + no >= kLongAdd) {  // long: one warp of this block adds it below
        const int q = atomicAdd(&s_nlong, 1);
        if (q < kLongCap) {
          s_long[q] = j;
          continue;
        }
      }
      const unsigned long long* b = W.pool + __ldcg(&W.hoff[o]);
      const uint32_t cap = n + no;
      const uint32_t off = atomicAdd(W.pool_head, cap);
      if ((unsigned long long)off + cap > W.pool_cap) {
        atomicOr(status, kErrPool);
        continue;
      }
      unsigned long long* d = W.pool + off;
      uint32_t x = 0, y = 0, m = 0;
      unsigned long long ax = x < n ? __ldcg(a) : 0, by = y < no ? __ldcg(b) : 0;
      while (x < n && y < no) {  // both decreasing: symmetric difference
        if (ax > by) {
          d[m++] = ax;
          ax = ++x < n ? __ldcg(a + x) : 0;
        } else if (by > ax) {
          d[m++] = by;
          by = ++y < no ? __ldcg(b + y) : 0;
        } else {
          ax = ++x < n ? __ldcg(a + x) : 0;
          by = ++y < no ? __ldcg(b + y) : 0;
        }
      }
      for (; x < n; ++x) d[m++] = __ldcg(a + x);
      for (; y < no; ++y) d[m++] = __ldcg(b + y);
      W.hoff[j] = off;
      W.hsize[j] = m;
      atomicAdd(&W.stats[6], (unsigned long long)m);
      atomicMax(&W.stats[7], (unsigned long long)m);
      if (m == 0) atomicOr(status, kErrEmptyColumn);
      else d1_list_push(nxt, n_next, mark, j, round);
    }
    __syncthreads();
    {  // this block's long additions, one warp each
      const int nlong = min(s_nlong, kLongCap), lane = threadIdx.x & 31;
      for (int q = threadIdx.x >> 5; q < nlong; q += kUFT / 32) {
        const int j = s_long[q];
        const uint32_t n = __ldcg(&W.hsize[j]);
        const unsigned long long* a = W.pool + __ldcg(&W.hoff[j]);
        const int o = __ldcg(&W.owner[(int)__ldcg(a)]);
        const uint32_t no = __ldcg(&W.hsize[o]);
        const unsigned long long* b = W.pool + __ldcg(&W.hoff[o]);
        const uint32_t cap = n + no;
        uint32_t off = 0;
        if (lane == 0) off = atomicAdd(W.pool_head, cap);
        off = __shfl_sync(0xFFFFFFFFu, off, 0);
        if ((unsigned long long)off + cap > W.pool_cap) {
          if (lane == 0) atomicOr(status, kErrPool);
          continue;
        }
        const uint32_t m = d1_warp_add<true>(a, n, b, no, W.pool + off, status);
        if (lane == 0) {
          W.hoff[j] = off;
          W.hsize[j] = m;
          atomicAdd(&W.stats[6], (unsigned long long)m);
          atomicMax(&W.stats[7], (unsigned long long)m);
          if (m == 0) atomicOr(status, kErrEmptyColumn);
          else d1_list_push(nxt, n_next, mark, j, round);
        }
      }
    }
    which ^= 1;
    if (gt == 0) {
      ctl->n[which ^ 1] = 0;  // the list the next round fills
      ctl->which = which;
      ctl->rounds = round + 1;
      W.stats[5] = (unsigned long long)(round + 1);
      W.stats[8] += 1;
      W.stats[9] += (unsigned long long)(clock64() - c_round);
    }
    if (!grid_barrier(ctl->bar, nb, status, limit)) return;
  }
  if (gt == 0) W.stats[10] += (unsigned long long)(clock64() - c_start);
}

static_assert(sizeof(UfCtl) <= 64 && sizeof(D1Ctl) <= 64, "control blocks share PairScratch::counter (64 bytes)");

void launch_d1_reduce(int n1, int n2, D1Work& W, PairOut& P, uint32_t* status, D1Ctl* ctl, cudaStream_t st) {
  if (n2 == 0) return;
  int dev = 0;
  cudaGetDevice(&dev);
  static std::atomic<bool> attr[64] = {};
  if (dev >= 0 && dev < 64 && !attr[dev].load(std::memory_order_acquire)) {
    cudaFuncSetAttribute(k_d1_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kChainSmem);
    attr[dev].store(true, std::memory_order_release);
  }
  const uint32_t ccap = (uint32_t)std::min<int64_t>(std::max<int64_t>(g_chain_cap.load(), 0), kCCap);
  const int64_t cm = g_chain_max.load();
  const int chain_max = cm > 0 ? (int)std::min<int64_t>(cm, kChainLimit) : kChainMax;
  const int nb = n2 >= g_d1_grid_min.load() ? cooperative_blocks((const void*)k_d1_reduce_grid, kUFT) : 0;
  if (nb > 0) {
    cudaMemsetAsync(ctl, 0, sizeof(D1Ctl), st);
    int handoff = (int)std::min<int64_t>(g_d1_handoff.load(), 1 << 30);
    unsigned limit = (unsigned)std::min<int64_t>(std::max<int64_t>(g_barrier_limit.load(), 1), 1u << 30);
    void* args[] = {&W, &n1, &ctl, &handoff, &limit, &status};
    if (cooperative_launch((const void*)k_d1_reduce_grid, dim3(nb), dim3(kUFT), args, st) == cudaSuccess) {
      k_d1_reduce<<<1, kUFT, kChainSmem, st>>>(W, n1, P.d1_edge, ctl, ccap, chain_max, status); note_launch();
      return;
    }
    cudaGetLastError();  // not launched: the single block does every round
  }
  k_d1_reduce<<<1, kUFT, kChainSmem, st>>>(W, n1, P.d1_edge, nullptr, ccap, chain_max, status); note_launch();
}

}  // namespace tsf
