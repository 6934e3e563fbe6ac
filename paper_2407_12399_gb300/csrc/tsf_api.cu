// tsf_api.cu -- the C ABI (include/tsf.h): buffers, stage order and status
// mapping.  Every computation happens in the kernels; this file only
// allocates, launches and reads back counts.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include <atomic>

#include "../../include/tsf.h"
#include "tsf_kernels.cuh"
#include "tsf_solver.cuh"

using namespace tsf;

namespace tsf {
static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace tsf

namespace {

template <class T>
cudaError_t dev_alloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  return cudaMalloc((void**)p, n * sizeof(T));
}
template <class T>
void dev_free(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

struct Fail {
  int code;
};
inline void ck(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) throw Fail{TSF_ENOMEM};
  if (e != cudaSuccess) throw Fail{TSF_ECUDA};
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct tsf_field {
  int device = 0;  // the device current when the field was created
  Dims d{};
  NbrDelta nd{};
  cudaStream_t st = nullptr;
  // vertex-sized
  float* f = nullptr;
  uint32_t *order = nullptr, *rank = nullptr, *sort_scratch = nullptr;
  // value keys in order (skey[i] = value_key of order[i]), the buffers the
  // incremental order update writes, and its scratch
  uint32_t *skey = nullptr, *order2 = nullptr, *skey2 = nullptr, *ubits = nullptr, *ucnt = nullptr;
  unsigned long long* ordB = nullptr;
  bool order_valid = false;  // order/skey/rank are those of the current values
  Rec* rec = nullptr;
  D1Tab* tab = nullptr;
  uint8_t* vnext8 = nullptr;
  // fast persistence update (Section 4.2): vertices the last step updated,
  // the lower stars to recompute (listed once each by generation marks)
  uint32_t *upd = nullptr, *gmark = nullptr, *glist = nullptr;
  double* lgrad = nullptr;  // dL/df of the topological loss (allocated on first use)
  float* lstage = nullptr;  // host values staged on the device for it
  uint32_t ggen = 0;
  uint32_t *cidx = nullptr, *c1base = nullptr, *c2base = nullptr;
  int4 *tile_counts = nullptr, *totals = nullptr;
  uint32_t* status = nullptr;
  unsigned long long* counter = nullptr;
  // critical cells and their pairs
  CritLists L{};
  int n0 = 0, n1 = 0, n2 = 0, n3 = 0;
  int cap_c0 = 0, cap_c1 = 0, cap_c2 = 0, cap_c3 = 0;
  PairScratch PS{};
  int cap_items = 0, cap_nodes = 0;
  PairOut PO{};
  D1Work W{};
  int cap_cols = 0;
  uint32_t pool_cap = 0;
  // solver
  SolverBufs B{};
  int cap_pts = 0, cap_t = 0, cap_idx = 0, cap_idxcd = 0;
  Pt* pts = nullptr;
  Pt* prev = nullptr;
  int np = 0, nprev = 0;
  Tg* T = nullptr;
  int nt = 0;
  bool have_targets = false, diagram_current = false, records_valid = false, upd_valid = false;
  int iter = 0;
  double loss = 0, loss0 = 0;
  unsigned long long counts[4] = {0, 0, 0, 0};
  int64_t n_updated = 0, n_gradient = 0;
  unsigned long long d1_stats[15] = {};
  int d1_cols = 0;
  int32_t* h_flags = nullptr;  // pinned
  double ms_diag = 0, ms_assign = 0, ms_step = 0;
  int64_t assign_rounds = 0, assign_phases = 0, assign_checks = 0;
  // profiling: event pairs recorded around stages, resolved after each call
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, size_t>> ev_pending;  // (stage, index of the pair in ev_pool)
  int ev_open[TSF_NSTAGES] = {};
  double prof_ms[TSF_NSTAGES] = {};
  int64_t prof_calls[TSF_NSTAGES] = {};
};

namespace {

enum Stage { kSort, kGrad, kCrit, kD0, kD2, kD1, kPoints, kAssign, kLoss, kStep, kD1Morse, kD1Reduce };

void stage_begin(tsf_field* F, int s) {
  if (!F->prof) return;
  size_t k = F->ev_pending.size();
  while (F->ev_pool.size() < 2 * (k + 1)) {
    cudaEvent_t e;
    ck(cudaEventCreate(&e));
    F->ev_pool.push_back(e);
  }
  F->ev_pending.push_back({s, k});
  F->ev_open[s] = (int)k;
  ck(cudaEventRecord(F->ev_pool[2 * k], F->st));
}
void stage_end(tsf_field* F, int s) {
  if (!F->prof) return;
  ck(cudaEventRecord(F->ev_pool[2 * (size_t)F->ev_open[s] + 1], F->st));
}
// called once the stream is idle (end of a public call)
void profile_resolve(tsf_field* F) {
  if (F->ev_pending.empty()) return;
  cudaStreamSynchronize(F->st);
  for (auto& pe : F->ev_pending) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, F->ev_pool[2 * pe.second], F->ev_pool[2 * pe.second + 1]) == cudaSuccess) {
      F->prof_ms[pe.first] += ms;
      F->prof_calls[pe.first] += 1;
    }
  }
  F->ev_pending.clear();
}

void grow_crit(tsf_field* F, int n0, int n1, int n2, int n3) {
  auto need = [](int have, int want) { return want > have ? std::max(want + want / 2, 1024) : have; };
  int c0 = need(F->cap_c0, n0), c1 = need(F->cap_c1, n1), c2 = need(F->cap_c2, n2), c3 = need(F->cap_c3, n3);
  if (c0 != F->cap_c0) {
    dev_free(F->L.c0);
    ck(dev_alloc(&F->L.c0, c0));
    F->cap_c0 = c0;
  }
  if (c1 != F->cap_c1) {
    dev_free(F->L.c1_key);
    dev_free(F->L.c1_vn);
    dev_free(F->PO.d0_min);
    dev_free(F->PO.d0_killed);
    dev_free(F->W.owner);
    dev_free(F->W.orec);
    ck(dev_alloc(&F->L.c1_key, c1));
    ck(dev_alloc(&F->L.c1_vn, c1));
    ck(dev_alloc(&F->PO.d0_min, c1));
    ck(dev_alloc(&F->PO.d0_killed, c1));
    ck(dev_alloc(&F->W.owner, c1));
    ck(dev_alloc(&F->W.orec, c1));
    F->cap_c1 = c1;
  }
  if (c2 != F->cap_c2) {
    dev_free(F->L.c2_ve);
    dev_free(F->PO.d2_max);
    dev_free(F->PO.d1_edge);
    dev_free(F->W.cols);
    dev_free(F->W.low);
    dev_free(F->W.hoff);
    dev_free(F->W.hcap);
    dev_free(F->W.hsize);
    dev_free(F->W.lowc);
    dev_free(F->W.redo);
  dev_free(F->W.cont);
  dev_free(F->W.cont_cap);
  dev_free(F->W.big);
  dev_free(F->W.nbig);
    dev_free(F->W.cont);
    dev_free(F->W.cont_cap);
    dev_free(F->W.big);
    ck(dev_alloc(&F->L.c2_ve, c2));
    ck(dev_alloc(&F->PO.d2_max, c2));
    ck(dev_alloc(&F->PO.d1_edge, c2));
    ck(dev_alloc(&F->W.cols, c2));
    ck(dev_alloc(&F->W.low, c2));
    ck(dev_alloc(&F->W.hoff, c2));
    ck(dev_alloc(&F->W.hcap, c2));
    ck(dev_alloc(&F->W.hsize, c2));
    ck(dev_alloc(&F->W.lowc, c2));
    ck(dev_alloc(&F->W.redo, c2));
    ck(dev_alloc(&F->W.cont, c2));
    ck(dev_alloc(&F->W.cont_cap, c2));
    ck(dev_alloc(&F->W.big, c2));
    if (!F->W.nbig) ck(dev_alloc(&F->W.nbig, 1));
    F->cap_c2 = c2;
  }
  if (c3 != F->cap_c3) {
    dev_free(F->L.c3);
    ck(dev_alloc(&F->L.c3, c3));
    F->cap_c3 = c3;
  }
  F->L.cap0 = F->cap_c0;
  F->L.cap1 = F->cap_c1;
  F->L.cap2 = F->cap_c2;
  F->L.cap3 = F->cap_c3;
  int items = std::max(F->cap_c1, F->cap_c2);
  int nodes = std::max(F->cap_c0, F->cap_c3 + 1);
  if (items > F->cap_items || nodes > F->cap_nodes) {
    int ci = std::max(items, F->cap_items), cn = std::max(nodes, F->cap_nodes);
    dev_free(F->PS.ends);
    dev_free(F->PS.roots);
    dev_free(F->PS.listA);
    dev_free(F->PS.listB);
    dev_free(F->PS.parent);
    dev_free(F->PS.reserve);
    ck(dev_alloc(&F->PS.ends, 2 * (size_t)ci));
    ck(dev_alloc(&F->PS.roots, 2 * (size_t)ci));
    ck(dev_alloc(&F->PS.listA, ci));
    ck(dev_alloc(&F->PS.listB, ci));
    ck(dev_alloc(&F->PS.parent, cn));
    ck(dev_alloc(&F->PS.reserve, cn));
    F->cap_items = ci;
    F->cap_nodes = cn;
  }
}

void grow_solver(tsf_field* F, int np, int nt) {
  bool again = np > F->cap_pts || nt > F->cap_t;
  if (!again) return;
  int cp = std::max(np + np / 2 + 64, F->cap_pts);
  int ctt = std::max(nt + nt / 2 + 64, F->cap_t);
  int ci = std::max(2 * cp, ctt) + 64;
  SolverBufs& B = F->B;
  // points (current/previous) keep their contents across a resize
  Pt *np_ = nullptr, *pp_ = nullptr;
  ck(dev_alloc(&np_, cp));
  ck(dev_alloc(&pp_, cp));
  if (F->pts && F->np) ck(cudaMemcpyAsync(np_, F->pts, sizeof(Pt) * F->np, cudaMemcpyDeviceToDevice, F->st));
  if (F->prev && F->nprev) ck(cudaMemcpyAsync(pp_, F->prev, sizeof(Pt) * F->nprev, cudaMemcpyDeviceToDevice, F->st));
  ck(cudaStreamSynchronize(F->st));
  dev_free(F->pts);
  dev_free(F->prev);
  F->pts = np_;
  F->prev = pp_;
  Tg* nt_ = nullptr;
  ck(dev_alloc(&nt_, ctt));
  if (F->T && F->nt) ck(cudaMemcpyAsync(nt_, F->T, sizeof(Tg) * F->nt, cudaMemcpyDeviceToDevice, F->st));
  ck(cudaStreamSynchronize(F->st));
  dev_free(F->T);
  F->T = nt_;
  dev_free(B.tmp_pts);
  dev_free(B.keyord);
  B.keyord_for = nullptr;
  dev_free(B.idxA);
  dev_free(B.idxB);
  dev_free(B.idxC);
  dev_free(B.idxD);
  dev_free(B.u32a);
  dev_free(B.u32b);
  dev_free(B.u32c);
  dev_free(B.taken);
  dev_free(B.plist);
  dev_free(B.tlist);
  dev_free(B.nkept);
  dev_free(B.is_col);
  dev_free(B.colpos);
  dev_free(B.col_point);
  dev_free(B.diag_t);
  dev_free(B.terms);
  dev_free(B.contrib);
  ck(dev_alloc(&B.tmp_pts, cp));
  ck(dev_alloc(&B.keyord, cp));
  dev_free(B.rsort);
  B.cap_rsort = 2 * (int64_t)cp;
  ck(dev_alloc(&B.rsort, (size_t)radix_sort64_words(B.cap_rsort)));
  ck(dev_alloc(&B.idxA, ci));
  ck(dev_alloc(&B.idxB, ci));
  int cicd = std::max(ci, B.cap_cand + 64);
  ck(dev_alloc(&B.idxC, cicd));
  ck(dev_alloc(&B.idxD, cicd));
  F->cap_idxcd = cicd;
  ck(dev_alloc(&B.u32a, ci));
  ck(dev_alloc(&B.u32b, ci));
  ck(dev_alloc(&B.u32c, ci));
  ck(dev_alloc(&B.taken, ctt));
  ck(dev_alloc(&B.plist, cp));
  ck(dev_alloc(&B.tlist, ctt));
  ck(dev_alloc(&B.nkept, ctt));
  ck(dev_alloc(&B.is_col, cp));
  ck(dev_alloc(&B.colpos, cp));
  ck(dev_alloc(&B.col_point, cp));
  ck(dev_alloc(&B.diag_t, ctt));
  ck(dev_alloc(&B.terms, (size_t)cp + ctt));
  ck(dev_alloc(&B.contrib, 2 * (size_t)cp));
  {
    AsgDev& A = B.A;
    dev_free(A.counts);
    dev_free(A.kept);
    dev_free(A.kept_off);
    dev_free(A.col_point);
    dev_free(A.H.u);
    dev_free(A.H.v);
    dev_free(A.H.minv);
    dev_free(A.H.list);
    dev_free(A.H.pm);
    dev_free(A.H.way);
    dev_free(A.H.used);
    dev_free(A.H.key);
    dev_free(A.H.aw);
    dev_free(A.H.bw);
    dev_free(A.aux);
    size_t w = (size_t)cp + ctt + 8;
    A.cap_kept = (int)std::min<int64_t>((int64_t)ctt * 2048, std::max<int64_t>((int64_t)16 * cp, 1 << 18));
    ck(dev_alloc(&A.counts, 16));
    ck(dev_alloc(&A.kept, (size_t)A.cap_kept));
    ck(dev_alloc(&A.kept_off, ctt));
    ck(dev_alloc(&A.col_point, w));
    ck(dev_alloc(&A.H.u, w));
    ck(dev_alloc(&A.H.v, w));
    ck(dev_alloc(&A.H.minv, w));
    ck(dev_alloc(&A.H.list, w));
    ck(dev_alloc(&A.H.pm, w));
    ck(dev_alloc(&A.H.way, w));
    ck(dev_alloc(&A.H.used, w));
    ck(dev_alloc(&A.H.key, w));
    ck(dev_alloc(&A.H.aw, w));
    ck(dev_alloc(&A.H.bw, w));
    ck(dev_alloc(&A.aux, 4 * w));
    A.plist = B.plist;
    A.tlist = B.tlist;
    A.nkept = B.nkept;
    A.is_col = B.is_col;
    A.colpos = B.colpos;
    A.diag_t = B.diag_t;
    A.col_to_row = nullptr;
  }
  if (!B.count) ck(dev_alloc(&B.count, 4));
  if (!B.dsum) ck(dev_alloc(&B.dsum, 1));
  if (!B.counters) ck(dev_alloc(&B.counters, 4));
  if (!B.actl) ck(cudaMalloc(&B.actl, 256));
  B.cap_k = ctt;
  F->cap_pts = cp;
  F->cap_t = ctt;
  F->cap_idx = ci;
}

void grow_assign(tsf_field* F, int cand, int cols) {
  SolverBufs& B = F->B;
  if (cand > B.cap_cand) {
    int c = cand + cand / 2 + 1024;
    dev_free(B.cands);
    dev_free(B.kept);
    ck(dev_alloc(&B.cands, c));
    ck(dev_alloc(&B.kept, c));
    B.cap_cand = c;
    if (c + 64 > F->cap_idxcd) {  // candidate sorts use idxC/idxD
      int ci = c + 64;
      dev_free(B.idxC);
      dev_free(B.idxD);
      ck(dev_alloc(&B.idxC, ci));
      ck(dev_alloc(&B.idxD, ci));
      F->cap_idxcd = ci;
    }
  }
  if (cols > B.cap_cols) {
    int c = cols + cols / 2 + 1024;
    HungWork& H = B.H;
    dev_free(H.u);
    dev_free(H.v);
    dev_free(H.minv);
    dev_free(H.list);
    dev_free(H.pm);
    dev_free(H.way);
    dev_free(H.used);
    dev_free(H.key);
    dev_free(H.aw);
    dev_free(H.bw);
    dev_free(B.aux);
    dev_free(B.col_to_row);
    ck(dev_alloc(&H.u, c + 1));
    ck(dev_alloc(&H.v, c + 1));
    ck(dev_alloc(&H.minv, c + 1));
    ck(dev_alloc(&H.list, c + 1));
    ck(dev_alloc(&H.pm, c + 1));
    ck(dev_alloc(&H.way, c + 1));
    ck(dev_alloc(&H.used, c + 1));
    ck(dev_alloc(&H.key, c + 1));
    ck(dev_alloc(&H.aw, c + 1));
    ck(dev_alloc(&H.bw, c + 1));
    ck(dev_alloc(&B.aux, 4 * ((size_t)c + 1)));
    ck(dev_alloc(&B.col_to_row, c + 1));
    B.cap_cols = c;
  }
}

uint32_t read_status(tsf_field* F) {
  uint32_t s = 0;
  ck(cudaMemcpyAsync(&s, F->status, 4, cudaMemcpyDeviceToHost, F->st));
  ck(cudaStreamSynchronize(F->st));
  return s;
}

static_assert(TSF_ENAN == -2 && TSF_ETIMEOUT == -5 && TSF_EINTERNAL == -8, "status_code() values");

// Stages 1-4 of the diagram: vertex order, lower-star gradient, critical
// cells, pairs, points (in F->pts, diagram order).
int compute_diagram(tsf_field* F, bool incremental) {
  cudaStream_t st = F->st;
  double t0 = now_ms();
  ck(cudaMemsetAsync(F->status, 0, 4, st));
  stage_begin(F, kSort);
  if (incremental && F->order_valid && F->upd_valid && F->n_updated <= kIncOrderMax) {
    if (F->n_updated > 0) {
      vertex_order_incremental(F->f, F->d.nv, F->upd, (int)F->n_updated, F->order, F->skey, F->order2, F->skey2,
                               F->rank, F->ubits, F->ucnt, F->ordB, F->status, st);
      std::swap(F->order, F->order2);
      std::swap(F->skey, F->skey2);
    }
  } else {
    vertex_order(F->f, F->d.nv, F->order, F->rank, F->skey, F->sort_scratch, F->status, st);
  }
  F->order_valid = true;
  stage_end(F, kSort);
  // The status word is read where the host waits anyway (the critical-cell
  // counts, the end of D1); every kernel in between stays in bounds on any
  // permutation, so a NaN found late only invalidates the results.
  bool inc = incremental && F->records_valid && F->upd_valid;
  unsigned long long ngrad = (unsigned long long)F->d.nv;
  stage_begin(F, kGrad);
  if (inc) {
    if (++F->ggen == 0) {  // the marks wrapped around: start over
      ck(cudaMemsetAsync(F->gmark, 0, sizeof(uint32_t) * (size_t)F->d.nv, st));
      F->ggen = 1;
    }
    launch_gradient_incremental(F->d, F->rank, F->f, F->upd, F->n_updated, F->gmark, F->ggen, F->glist, F->counter,
                                F->rec, F->vnext8, F->tab, F->status, st);
    ck(cudaMemcpyAsync(&ngrad, F->counter, 8, cudaMemcpyDeviceToHost, st));
  } else {
    launch_gradient(F->d, F->rank, F->f, F->rec, F->vnext8, F->tab, F->status, st);
  }
  stage_end(F, kGrad);
  F->records_valid = true;
  stage_begin(F, kCrit);
  launch_crit_count(F->d, F->order, F->rec, F->tile_counts, F->totals, st);
  int4 tot;
  uint32_t s = 0;
  ck(cudaMemcpyAsync(&tot, F->totals, sizeof(int4), cudaMemcpyDeviceToHost, st));
  ck(cudaMemcpyAsync(&s, F->status, sizeof(s), cudaMemcpyDeviceToHost, st));
  ck(cudaStreamSynchronize(st));
  if (s & kErrNaN) {
    F->order_valid = false;
    F->records_valid = false;
    return TSF_ENAN;
  }
  if (status_code(s) != TSF_OK) return status_code(s);
  F->n_gradient = (int64_t)ngrad;
  F->n0 = tot.x;
  F->n1 = tot.y;
  F->n2 = tot.z;
  F->n3 = tot.w;
  grow_crit(F, F->n0, F->n1, F->n2, F->n3);
  launch_crit_write(F->d, F->order, F->rank, F->rec, F->tile_counts, F->L, F->cidx, F->c1base, F->c2base, F->status,
                    st);
  stage_end(F, kCrit);
  stage_begin(F, kD0);
  launch_d0(F->d, F->nd, F->L, F->n0, F->n1, F->vnext8, F->cidx, F->PS, F->PO, F->status, st);
  stage_end(F, kD0);
  stage_begin(F, kD2);
  launch_d2(F->d, F->nd, F->L, F->n2, F->n3, F->rank, F->rec, F->cidx, F->PS, F->PO, F->status, st);
  stage_end(F, kD2);
  // D1, growing the column pool until it suffices (D0 and D2 report through
  // the same status word, read after the first attempt)
  for (int attempt = 0;; ++attempt) {
    uint32_t want = (uint32_t)std::min<int64_t>(std::max<int64_t>((int64_t)64 * std::max(F->n2, 1), 1 << 20) << attempt,
                                                 (int64_t)1 << 31);
    if (want > F->pool_cap) {
      dev_free(F->W.pool);
      ck(dev_alloc(&F->W.pool, want));
      F->pool_cap = want;
    }
    F->W.pool_cap = F->pool_cap;
    if (!F->W.pool_head) ck(dev_alloc(&F->W.pool_head, 1));
    if (!F->W.flags) ck(dev_alloc(&F->W.flags, 4));
    if (!F->W.stats) ck(dev_alloc(&F->W.stats, kD1Stats));
    if (attempt > 0) ck(cudaMemsetAsync(F->status, 0, 4, st));
    stage_begin(F, kD1);
    launch_d1_prepare(F->n2, F->W, F->PO, st);
    stage_end(F, kD1);
    stage_begin(F, kD1Morse);
    launch_d1_morse(F->d, F->nd, F->L, F->n1, F->n2, F->rank, F->order, F->f, F->rec, F->tab, F->c1base, F->W,
                    F->PO, F->status, st);
    stage_end(F, kD1Morse);
    stage_begin(F, kD1Reduce);
    launch_d1_reduce(F->n1, F->n2, F->W, F->PO, F->status, reinterpret_cast<D1Ctl*>(F->PS.counter), st);
    stage_end(F, kD1Reduce);
    int32_t ncols = 0;
    for (auto& x : F->d1_stats) x = 0;
    ck(cudaMemcpyAsync(&s, F->status, sizeof(s), cudaMemcpyDeviceToHost, st));
    if (F->n2 > 0) {
      ck(cudaMemcpyAsync(&ncols, F->W.flags + 1, sizeof(ncols), cudaMemcpyDeviceToHost, st));
      ck(cudaMemcpyAsync(F->d1_stats, F->W.stats, sizeof(F->d1_stats), cudaMemcpyDeviceToHost, st));
    }
    ck(cudaStreamSynchronize(st));
    F->d1_cols = ncols;
    if ((s & kErrPool) && !(s & ~kErrPool) && attempt < 6) continue;
    break;
  }
  if (status_code(s) != TSF_OK) return status_code(s);
  // points
  int want_pts = F->n0 + F->n2 + 1;
  grow_solver(F, want_pts, F->nt);
  stage_begin(F, kPoints);
  int np = build_diagram(F->d, F->nd, F->L, F->n1, F->n2, F->n3, F->PO, F->order, F->f, F->B, F->pts, F->cap_pts, st);
  stage_end(F, kPoints);
  if (np < 0) return TSF_EINTERNAL;
  F->np = np;
  F->diagram_current = true;
  ck(cudaGetLastError());
  F->ms_diag = now_ms() - t0;
  return TSF_OK;
}

int run_assign(tsf_field* F, const Pt* ref, int nr, double prec = 0.0) {
  double t0 = now_ms();
  AssignStats as{};
  for (int attempt = 0; attempt < 8; ++attempt) {
    as.status_valid = false;
    ck(cudaMemsetAsync(F->status, 0, 4, F->st));
    stage_begin(F, kAssign);
    int r = assign(F->np, F->pts, nr, ref, F->nt, F->T, prec, F->B, F->status, &as, F->st);
    stage_end(F, kAssign);
    if (r == 0) break;
    if (r == -2) grow_assign(F, std::max(2 * F->B.cap_cand, 4096), 0);
    else if (r == -3) grow_assign(F, 0, std::max(2 * F->B.cap_cols, 4096));
    else if (r == -4) return TSF_ECUDA;  // a cooperative launch was refused
    else return TSF_EINTERNAL;
    // the failed pass may have written partial assignments: restart from the still step
  }
  uint32_t s = as.status_valid ? as.status : read_status(F);
  if (status_code(s) != TSF_OK) return status_code(s);
  F->ms_assign = now_ms() - t0;
  F->assign_rounds = as.rounds;
  F->assign_phases = as.phases;
  F->assign_checks = as.checks;
  return TSF_OK;
}

void fill_stats(tsf_field* F, const tsf_params* p, tsf_stats* out, int done) {
  if (!out) return;
  std::memset(out, 0, sizeof(*out));
  out->iters = F->iter;
  out->done = done;
  out->loss0 = F->loss0;
  out->loss = F->loss;
  out->n_points = F->np;
  out->n_pairs[0] = F->n0 > 0 ? F->n0 - 1 : 0;
  out->n_pairs[1] = F->n2 - F->n3;
  out->n_pairs[2] = F->n3;
  out->n_critical[0] = F->n0;
  out->n_critical[1] = F->n1;
  out->n_critical[2] = F->n2;
  out->n_critical[3] = F->n3;
  out->n_uncancelled = (int64_t)F->counts[0];
  out->n_still = (int64_t)F->counts[1];
  out->n_nonstill_matched = (int64_t)F->counts[2];
  out->n_updated_vertices = F->n_updated;
  out->n_gradient_vertices = F->n_gradient;
  out->d1_columns = F->d1_cols;
  out->d1_blocks_total = (int64_t)F->d1_stats[0];
  out->d1_blocks_max = (int64_t)F->d1_stats[1];
  out->d1_rounds_total = (int64_t)F->d1_stats[2];
  out->d1_rounds_max = (int64_t)F->d1_stats[3];
  out->d1_star_updates = (int64_t)F->d1_stats[4];
  out->d1_reduce_rounds = (int64_t)F->d1_stats[5];
  out->d1_reduce_merged = (int64_t)F->d1_stats[6];
  out->d1_reduce_longest = (int64_t)F->d1_stats[7];
  out->d1_reduce_big_rounds = (int64_t)F->d1_stats[8];
  out->d1_reduce_big_cycles = (int64_t)F->d1_stats[9];
  out->d1_reduce_cycles = (int64_t)F->d1_stats[10];
  out->d1_chain_adds = (int64_t)F->d1_stats[11];
  out->d1_chain_longest = (int64_t)F->d1_stats[12];
  out->d1_chain_rounds = (int64_t)F->d1_stats[13];
  out->d1_chain_cycles = (int64_t)F->d1_stats[14];
  out->ms_diagram = F->ms_diag;
  out->ms_assign = F->ms_assign;
  out->assign_rounds = F->assign_rounds;
  out->assign_phases = F->assign_phases;
  out->assign_checks = F->assign_checks;
  out->ms_step = F->ms_step;
  (void)p;
}

int eval(tsf_field* F, float cancel_eps) {
  stage_begin(F, kLoss);
  loss_and_counts(F->np, F->pts, F->nt, F->T, cancel_eps, F->B, &F->loss, F->counts, F->st);
  stage_end(F, kLoss);
  return TSF_OK;
}

int is_done(tsf_field* F, const tsf_params* p) {
  if (F->counts[0] == 0) return 1;
  if (p->stop_s > 0.0f && F->loss <= (double)p->stop_s * F->loss0) return 1;
  return F->iter >= p->max_iters ? 1 : 0;
}

int start_solver(tsf_field* F) {
  // j = 0: the targets play the previous diagram, each assigned to itself
  grow_solver(F, F->np, F->nt);
  targets_as_points(F->nt, F->T, F->prev, F->st);
  F->B.keyord_for = nullptr;  // prev now holds the targets
  F->nprev = F->nt;
  int r = run_assign(F, F->prev, F->nt);
  if (r) return r;
  F->iter = 0;
  eval(F, 0.0f);
  F->loss0 = F->loss;
  F->have_targets = true;
  return TSF_OK;
}

int check_params(const tsf_params* p) {
  if (!p) return TSF_EINVAL;
  if (!(p->alpha_b >= 0.0f) || !(p->alpha_d >= 0.0f) || !(p->cancel_eps >= 0.0f) || p->max_iters < 0 ||
      !(p->assignment_precision >= 0.0f) || !(p->assignment_precision <= 3.4e38f))
    return TSF_EINVAL;
  return TSF_OK;
}

int step(tsf_field* F, const tsf_params* p, tsf_stats* stats) {
  cudaStream_t st = F->st;
  double t0 = now_ms();
  bool fast = p->fast_gradient_update != 0;
  stage_begin(F, kStep);
  F->n_updated =
      gradient_step(F->np, F->pts, F->T, p->alpha_b, p->alpha_d, F->f, fast ? F->upd : nullptr, F->B, F->status, st);
  stage_end(F, kStep);
  F->upd_valid = fast;
  F->ms_step = now_ms() - t0;
  // previous diagram (with its assignment) becomes the still-pair reference
  std::swap(F->pts, F->prev);
  F->nprev = F->np;
  int r = compute_diagram(F, fast);
  if (r) return r;
  // without the Section 4.3 reuse no point of the previous diagram is
  // consulted: every point is matched by the exact solver
  r = run_assign(F, F->prev, p->fast_assignment_update ? F->nprev : 0, (double)p->assignment_precision);
  if (r) return r;
  F->iter += 1;
  eval(F, p->cancel_eps);
  int done = is_done(F, p);
  fill_stats(F, p, stats, done);
  return TSF_OK;
}

template <class Fn>
int guarded(Fn&& fn) {
  try {
    return fn();
  } catch (const Fail& f) {
    return f.code;
  } catch (...) {
    return TSF_EINTERNAL;
  }
}

// Makes the field's device current for one call (the current device is per
// host thread) and restores the caller's afterwards.
struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(const tsf_field* F) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev >= 0 && prev != F->device) cudaSetDevice(F->device);
  }
  ~DeviceScope() {
    int now = -1;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
  }
};

template <class Fn>
int guarded_dev(tsf_field* F, Fn&& fn) {
  DeviceScope ds(F);
  return guarded(fn);
}

template <class Fn>
int guarded_f(tsf_field* F, Fn&& fn) {
  DeviceScope ds(F);
  int r = guarded(fn);
  profile_resolve(F);
  return r;
}

}  // namespace

extern "C" {

const char* tsf_status_string(int s) {
  switch (s) {
    case TSF_OK: return "ok";
    case TSF_EINVAL: return "invalid argument";
    case TSF_ENAN: return "field holds a NaN or infinite value";
    case TSF_ENOMEM: return "device allocation failed";
    case TSF_ECUDA: return "CUDA error";
    case TSF_ETIMEOUT: return "a device loop hit its bound";
    case TSF_ENOTARGET: return "no target diagram set";
    case TSF_ECAPACITY: return "output buffer too small";
    case TSF_EINTERNAL: return "internal consistency check failed";
    default: return "unknown status";
  }
}

int tsf_destroy_field(tsf_field* F) {
  if (!F) return TSF_OK;
  DeviceScope ds(F);
  cudaStreamSynchronize(F->st);
  dev_free(F->f);
  dev_free(F->order);
  dev_free(F->rank);
  dev_free(F->sort_scratch);
  dev_free(F->rec);
  dev_free(F->tab);
  dev_free(F->vnext8);
  dev_free(F->skey);
  dev_free(F->order2);
  dev_free(F->skey2);
  dev_free(F->ubits);
  dev_free(F->ucnt);
  dev_free(F->ordB);
  dev_free(F->lgrad);
  dev_free(F->lstage);
  dev_free(F->upd);
  dev_free(F->gmark);
  dev_free(F->glist);
  dev_free(F->cidx);
  dev_free(F->c1base);
  dev_free(F->c2base);
  dev_free(F->tile_counts);
  dev_free(F->totals);
  dev_free(F->status);
  dev_free(F->counter);
  dev_free(F->L.c0);
  dev_free(F->L.c1_key);
  dev_free(F->L.c1_vn);
  dev_free(F->L.c2_ve);
  dev_free(F->L.c3);
  dev_free(F->PS.ends);
  dev_free(F->PS.roots);
  dev_free(F->PS.listA);
  dev_free(F->PS.listB);
  dev_free(F->PS.parent);
  dev_free(F->PS.reserve);
  dev_free(F->PS.counter);
  dev_free(F->PO.d0_min);
  dev_free(F->PO.d0_killed);
  dev_free(F->PO.d0mask);
  dev_free(F->PO.d2_max);
  dev_free(F->PO.d1_edge);
  dev_free(F->W.cols);
  dev_free(F->W.low);
  dev_free(F->W.hoff);
  dev_free(F->W.hcap);
  dev_free(F->W.hsize);
  dev_free(F->W.lowc);
  dev_free(F->W.owner);
  dev_free(F->W.orec);
  dev_free(F->W.pool);
  dev_free(F->W.pool_head);
  dev_free(F->W.flags);
  dev_free(F->W.stats);
  dev_free(F->W.redo);
  dev_free(F->W.cont);
  dev_free(F->W.cont_cap);
  dev_free(F->W.big);
  dev_free(F->W.nbig);
  SolverBufs& B = F->B;
  dev_free(F->pts);
  dev_free(F->prev);
  dev_free(F->T);
  dev_free(B.tmp_pts);
  dev_free(B.keyord);
  dev_free(B.rsort);
  B.keyord_for = nullptr;
  dev_free(B.idxA);
  dev_free(B.idxB);
  dev_free(B.idxC);
  dev_free(B.idxD);
  dev_free(B.count);
  dev_free(B.u32a);
  dev_free(B.u32b);
  dev_free(B.u32c);
  dev_free(B.taken);
  dev_free(B.plist);
  dev_free(B.tlist);
  dev_free(B.cands);
  dev_free(B.kept);
  dev_free(B.nkept);
  dev_free(B.is_col);
  dev_free(B.colpos);
  dev_free(B.col_point);
  dev_free(B.col_to_row);
  dev_free(B.diag_t);
  dev_free(B.H.u);
  dev_free(B.H.v);
  dev_free(B.H.minv);
  dev_free(B.H.list);
  dev_free(B.H.pm);
  dev_free(B.H.way);
  dev_free(B.H.used);
  dev_free(B.H.key);
  if (B.actl) cudaFree(B.actl);
  dev_free(B.H.aw);
  dev_free(B.H.bw);
  dev_free(B.aux);
  dev_free(B.terms);
  dev_free(B.dsum);
  dev_free(B.counters);
  dev_free(B.contrib);
  dev_free(B.A.counts);
  dev_free(B.A.kept);
  dev_free(B.A.kept_off);
  dev_free(B.A.col_point);
  dev_free(B.A.H.u);
  dev_free(B.A.H.v);
  dev_free(B.A.H.minv);
  dev_free(B.A.H.list);
  dev_free(B.A.H.pm);
  dev_free(B.A.H.way);
  dev_free(B.A.H.used);
  dev_free(B.A.H.key);
  dev_free(B.A.H.aw);
  dev_free(B.A.H.bw);
  dev_free(B.A.aux);
  if (F->h_flags) cudaFreeHost(F->h_flags);
  for (auto e : F->ev_pool) cudaEventDestroy(e);
  delete F;
  return TSF_OK;
}

int tsf_create_field(int lx, int ly, int lz, const float* values, int values_on_device, void* cuda_stream,
                     tsf_field** out) {
  if (!out || !values || lx < 2 || ly < 2 || lz < 2) return TSF_EINVAL;
  int64_t nv = (int64_t)lx * ly * lz;
  if (nv >= ((int64_t)1 << 26)) return TSF_EINVAL;  // vertex ids are packed in 26 bits
  *out = nullptr;
  tsf_field* F = new (std::nothrow) tsf_field();
  if (!F) return TSF_ENOMEM;
  if (cudaGetDevice(&F->device) != cudaSuccess) {
    delete F;
    return TSF_ECUDA;
  }
  int r = guarded([&]() {
    F->d.lx = lx;
    F->d.ly = ly;
    F->d.lz = lz;
    F->d.nv = nv;
    F->B.ids30 = nv <= ((int64_t)1 << 30);
    F->st = (cudaStream_t)cuda_stream;
    for (int i = 0; i < 14; ++i)
      F->nd.d[i] = kGeo.off[i][0] + lx * (kGeo.off[i][1] + ly * kGeo.off[i][2]);
    ck(dev_alloc(&F->f, nv));
    ck(dev_alloc(&F->order, nv));
    ck(dev_alloc(&F->rank, nv));
    ck(dev_alloc(&F->sort_scratch, sort_scratch_words(nv)));
    ck(dev_alloc(&F->skey, nv));
    ck(dev_alloc(&F->order2, nv));
    ck(dev_alloc(&F->skey2, nv));
    ck(dev_alloc(&F->ubits, (size_t)(nv / 32 + 1)));
    ck(dev_alloc(&F->ucnt, (size_t)order_count_words(nv)));
    ck(dev_alloc(&F->ordB, kIncOrderMax));
    ck(dev_alloc(&F->rec, nv));
    ck(dev_alloc(&F->tab, nv));
    ck(dev_alloc(&F->vnext8, nv));
    ck(dev_alloc(&F->upd, nv));
    ck(dev_alloc(&F->gmark, nv));
    ck(dev_alloc(&F->glist, nv));
    ck(cudaMemsetAsync(F->gmark, 0, sizeof(uint32_t) * (size_t)nv, F->st));
    ck(dev_alloc(&F->cidx, nv));
    ck(dev_alloc(&F->c1base, nv));
    ck(dev_alloc(&F->c2base, nv));
    ck(dev_alloc(&F->PO.d0mask, nv));
    ck(dev_alloc(&F->tile_counts, crit_tiles(nv)));
    ck(dev_alloc(&F->totals, 1));
    ck(dev_alloc(&F->status, 1));
    ck(dev_alloc(&F->counter, 1));
    ck(dev_alloc(&F->PS.counter, 16));
    ck(cudaMallocHost((void**)&F->h_flags, 16));
    ck(cudaMemcpyAsync(F->f, values, sizeof(float) * nv,
                       values_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, F->st));
    ck(cudaStreamSynchronize(F->st));
    return TSF_OK;
  });
  if (r != TSF_OK) {
    tsf_destroy_field(F);
    return r;
  }
  *out = F;
  return TSF_OK;
}

}  // extern "C"

namespace tsf {
// Full diagram of a field's current values, for timing (the batch
// autotuner); refused once a target diagram is set, since it replaces the
// diagram the solver's assignment refers to.
int full_diagram_for_tuning(tsf_field* F) {
  if (!F) return TSF_EINVAL;
  if (F->have_targets) return TSF_EINVAL;
  return guarded_f(F, [&]() { return compute_diagram(F, false); });
}
}  // namespace tsf

extern "C" {

int tsf_compute_diagram(tsf_field* F, tsf_pair* out, int64_t cap, int64_t* n_out, int out_on_device) {
  if (!F || !n_out || cap < 0 || (cap > 0 && !out)) return TSF_EINVAL;
  return guarded_f(F, [&]() {
    if (!F->diagram_current) {
      int r = compute_diagram(F, false);
      if (r) return r;
    }
    *n_out = F->np;
    if (F->np > cap) return TSF_ECAPACITY;
    std::vector<Pt> h(F->np);
    ck(cudaMemcpyAsync(h.data(), F->pts, sizeof(Pt) * F->np, cudaMemcpyDeviceToHost, F->st));
    ck(cudaStreamSynchronize(F->st));
    std::vector<tsf_pair> o(F->np);
    for (int i = 0; i < F->np; ++i) {
      o[i].dim = h[i].dim;
      o[i].essential = h[i].ess;
      o[i].v_birth = h[i].vb;
      o[i].v_death = h[i].vd;
      o[i].cell_birth = h[i].cb;
      o[i].cell_death = h[i].cd;
      o[i].birth = h[i].b;
      o[i].death = h[i].d;
    }
    if (F->np)
      ck(cudaMemcpyAsync(out, o.data(), sizeof(tsf_pair) * F->np,
                         out_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, F->st));
    ck(cudaStreamSynchronize(F->st));
    return TSF_OK;
  });
}

int tsf_set_signal_threshold(tsf_field* F, float fraction) {
  if (!F || !(fraction >= 0.0f)) return TSF_EINVAL;
  return guarded_f(F, [&]() {
    int r = compute_diagram(F, false);
    if (r) return r;
    grow_solver(F, F->np, F->np);
    F->nt = make_targets(F->np, F->pts, F->order, F->f, F->d.nv, fraction, F->B, F->T, F->st);
    return start_solver(F);
  });
}

int tsf_set_signal_pairs(tsf_field* F, const tsf_pair* pairs, int64_t n) {
  if (!F || n < 0 || (n > 0 && !pairs)) return TSF_EINVAL;
  return guarded_f(F, [&]() {
    int r = compute_diagram(F, false);
    if (r) return r;
    std::vector<Tg> t((size_t)n);
    bool has_ess = false;
    for (int64_t i = 0; i < n; ++i) {
      t[i].b = pairs[i].birth;
      t[i].d = pairs[i].death;
      t[i].vb = pairs[i].v_birth;
      t[i].vd = pairs[i].v_death;
      t[i].dim = pairs[i].dim;
      t[i].ess = pairs[i].essential ? 1 : 0;
      t[i].src = (uint64_t)i;
      if (pairs[i].dim < 0 || pairs[i].dim > 2) return TSF_EINVAL;
      has_ess |= t[i].ess != 0;
    }
    if (!has_ess) {
      std::vector<Pt> h(F->np);
      ck(cudaMemcpyAsync(h.data(), F->pts, sizeof(Pt) * F->np, cudaMemcpyDeviceToHost, F->st));
      ck(cudaStreamSynchronize(F->st));
      for (auto& p : h)
        if (p.ess) {
          Tg e;
          e.b = p.b;
          e.d = p.d;
          e.vb = p.vb;
          e.vd = p.vd;
          e.dim = p.dim;
          e.ess = 1;
          e.src = (uint64_t)n;
          t.push_back(e);
        }
    }
    auto vk = [](float x) {
      uint32_t u;
      std::memcpy(&u, &x, 4);
      if (u == 0x80000000u) u = 0;
      return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    };
    std::sort(t.begin(), t.end(), [&](const Tg& x, const Tg& y) {
      if (vk(x.b) != vk(y.b)) return vk(x.b) < vk(y.b);
      if (vk(x.d) != vk(y.d)) return vk(x.d) < vk(y.d);
      if (x.vb != y.vb) return x.vb < y.vb;
      if (x.vd != y.vd) return x.vd < y.vd;
      if (x.dim != y.dim) return x.dim < y.dim;
      if (x.ess != y.ess) return x.ess < y.ess;
      return x.src < y.src;
    });
    grow_solver(F, F->np, (int)t.size());
    F->nt = (int)t.size();
    if (F->nt) ck(cudaMemcpyAsync(F->T, t.data(), sizeof(Tg) * t.size(), cudaMemcpyHostToDevice, F->st));
    ck(cudaStreamSynchronize(F->st));
    return start_solver(F);
  });
}

int tsf_solver_step(tsf_field* F, const tsf_params* p, tsf_stats* stats) {
  if (!F) return TSF_EINVAL;
  if (check_params(p)) return TSF_EINVAL;
  if (!F->have_targets) return TSF_ENOTARGET;
  return guarded_f(F, [&]() { return step(F, p, stats); });
}

int tsf_simplify(tsf_field* F, const tsf_params* p, float* out_values, int out_on_device, tsf_stats* stats) {
  if (!F) return TSF_EINVAL;
  if (check_params(p)) return TSF_EINVAL;
  if (!F->have_targets) return TSF_ENOTARGET;
  return guarded_f(F, [&]() {
    eval(F, p->cancel_eps);
    int done = is_done(F, p);
    fill_stats(F, p, stats, done);
    while (!done) {
      int r = step(F, p, stats);
      if (r) return r;
      done = is_done(F, p);
    }
    if (out_values)
      ck(cudaMemcpyAsync(out_values, F->f, sizeof(float) * F->d.nv,
                         out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, F->st));
    ck(cudaStreamSynchronize(F->st));
    return TSF_OK;
  });
}

int tsf_loss_and_gradient(tsf_field* F, const float* values, int values_on_device, double* loss, double* grad,
                          int grad_on_device) {
  if (!F || !values || !loss) return TSF_EINVAL;
  if (!F->have_targets) return TSF_ENOTARGET;
  return guarded_f(F, [&]() {
    // the new values replace the field's; the vertices they change are
    // listed, so the diagram follows them incrementally (Section 4.2) where
    // the previous order and records are those of the current values
    const float* in = values;
    if (!values_on_device) {
      if (!F->lstage) ck(dev_alloc(&F->lstage, (size_t)F->d.nv));
      ck(cudaMemcpyAsync(F->lstage, values, sizeof(float) * F->d.nv, cudaMemcpyHostToDevice, F->st));
      in = F->lstage;
    }
    replace_values(F->d.nv, in, F->f, F->upd, F->counter, F->st);
    unsigned long long nchanged = 0;
    ck(cudaMemcpyAsync(&nchanged, F->counter, sizeof(nchanged), cudaMemcpyDeviceToHost, F->st));
    ck(cudaStreamSynchronize(F->st));
    F->n_updated = (int64_t)nchanged;
    F->upd_valid = true;
    std::swap(F->pts, F->prev);  // the previous diagram is not consulted
    F->nprev = F->np;
    int r = compute_diagram(F, true);
    if (r) return r;
    r = run_assign(F, F->prev, 0);
    if (r) return r;
    eval(F, 0.0f);
    *loss = F->loss;
    if (grad) {
      if (!F->lgrad) ck(dev_alloc(&F->lgrad, (size_t)F->d.nv));
      loss_gradient(F->np, F->pts, F->T, F->B, F->lgrad, F->d.nv, F->st);
      ck(cudaMemcpyAsync(grad, F->lgrad, sizeof(double) * F->d.nv,
                         grad_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, F->st));
    }
    ck(cudaStreamSynchronize(F->st));
    ck(cudaGetLastError());
    return TSF_OK;
  });
}

int tsf_set_start_field(tsf_field* F, const float* values, int values_on_device) {
  if (!F || !values) return TSF_EINVAL;
  if (!F->have_targets) return TSF_ENOTARGET;
  return guarded_f(F, [&]() {
    // the start field replaces the values; the targets and loss_0 stay those
    // of f_0, and the solver restarts at iteration 0 from the new diagram
    const float* in = values;
    if (!values_on_device) {
      if (!F->lstage) ck(dev_alloc(&F->lstage, (size_t)F->d.nv));
      ck(cudaMemcpyAsync(F->lstage, values, sizeof(float) * F->d.nv, cudaMemcpyHostToDevice, F->st));
      in = F->lstage;
    }
    replace_values(F->d.nv, in, F->f, F->upd, F->counter, F->st);
    unsigned long long nchanged = 0;
    ck(cudaMemcpyAsync(&nchanged, F->counter, sizeof(nchanged), cudaMemcpyDeviceToHost, F->st));
    ck(cudaStreamSynchronize(F->st));
    F->n_updated = (int64_t)nchanged;
    F->upd_valid = true;
    // the current diagram (with its assignment) is the still-pair reference
    // of the start field's diagram, as after a solver step (Section 4.3)
    std::swap(F->pts, F->prev);
    F->nprev = F->np;
    int r = compute_diagram(F, true);
    if (r) return r;
    r = run_assign(F, F->prev, F->nprev);
    if (r) return r;
    F->iter = 0;
    eval(F, 0.0f);
    ck(cudaStreamSynchronize(F->st));
    return TSF_OK;
  });
}

int tsf_get_field(tsf_field* F, float* out, int out_on_device) {
  if (!F || !out) return TSF_EINVAL;
  return guarded_dev(F, [&]() {
    ck(cudaMemcpyAsync(out, F->f, sizeof(float) * F->d.nv,
                       out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, F->st));
    ck(cudaStreamSynchronize(F->st));
    return TSF_OK;
  });
}

int tsf_set_field(tsf_field* F, const float* values, int values_on_device) {
  if (!F || !values) return TSF_EINVAL;
  return guarded_dev(F, [&]() {
    ck(cudaMemcpyAsync(F->f, values, sizeof(float) * F->d.nv,
                       values_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, F->st));
    ck(cudaStreamSynchronize(F->st));
    F->diagram_current = false;
    F->records_valid = false;
    F->upd_valid = false;
    F->order_valid = false;
    F->have_targets = false;
    return TSF_OK;
  });
}

int tsf_get_assignment(tsf_field* F, int32_t* target, int32_t* still, int64_t cap, int64_t* n_out) {
  if (!F || !n_out) return TSF_EINVAL;
  return guarded_dev(F, [&]() {
    *n_out = F->np;
    if (F->np > cap) return TSF_ECAPACITY;
    std::vector<Pt> h(F->np);
    ck(cudaMemcpyAsync(h.data(), F->pts, sizeof(Pt) * F->np, cudaMemcpyDeviceToHost, F->st));
    ck(cudaStreamSynchronize(F->st));
    for (int i = 0; i < F->np; ++i) {
      if (target) target[i] = h[i].tgt;
      if (still) still[i] = h[i].still;
    }
    return TSF_OK;
  });
}

int tsf_get_targets(tsf_field* F, tsf_pair* out, int64_t cap, int64_t* n_out) {
  if (!F || !n_out) return TSF_EINVAL;
  return guarded_dev(F, [&]() {
    *n_out = F->nt;
    if (F->nt > cap) return TSF_ECAPACITY;
    std::vector<Tg> h(F->nt);
    if (F->nt) ck(cudaMemcpyAsync(h.data(), F->T, sizeof(Tg) * F->nt, cudaMemcpyDeviceToHost, F->st));
    ck(cudaStreamSynchronize(F->st));
    for (int i = 0; i < F->nt; ++i) {
      out[i].dim = h[i].dim;
      out[i].essential = h[i].ess;
      out[i].v_birth = h[i].vb;
      out[i].v_death = h[i].vd;
      out[i].cell_birth = h[i].src;
      out[i].cell_death = 0;
      out[i].birth = h[i].b;
      out[i].death = h[i].d;
    }
    return TSF_OK;
  });
}

int tsf_zero_pairs(tsf_field* F, uint64_t* out, int64_t cap_pairs, int64_t* n_out) {
  if (!F || !n_out || cap_pairs < 0) return TSF_EINVAL;
  return guarded_dev(F, [&]() {
    ck(cudaMemsetAsync(F->status, 0, 4, F->st));
    vertex_order(F->f, F->d.nv, F->order, F->rank, F->skey, F->sort_scratch, F->status, F->st);
    uint32_t s = read_status(F);
    F->order_valid = !(s & kErrNaN);
    if (s & kErrNaN) return TSF_ENAN;
    unsigned long long* dout = nullptr;
    int64_t cap = std::max<int64_t>(cap_pairs, 1);
    ck(dev_alloc(&dout, 2 * (size_t)cap));
    ck(cudaMemsetAsync(F->counter, 0, 8, F->st));
    launch_zero_pairs(F->d, F->rank, dout, cap, F->counter, F->status, F->st);
    unsigned long long n = 0;
    ck(cudaMemcpyAsync(&n, F->counter, 8, cudaMemcpyDeviceToHost, F->st));
    ck(cudaStreamSynchronize(F->st));
    *n_out = (int64_t)n;
    int rc = TSF_OK;
    if ((int64_t)n > cap_pairs) rc = TSF_ECAPACITY;
    else if (n) ck(cudaMemcpyAsync(out, dout, 16 * n, cudaMemcpyDeviceToHost, F->st));
    ck(cudaStreamSynchronize(F->st));
    dev_free(dout);
    s = read_status(F);
    if (status_code(s) != TSF_OK) return status_code(s);
    F->diagram_current = false;
    return rc;
  });
}

int tsf_profile_enable(tsf_field* F, int enable) {
  if (!F) return TSF_EINVAL;
  return guarded_dev(F, [&]() {
    profile_resolve(F);
    F->prof = enable != 0;
    for (int i = 0; i < TSF_NSTAGES; ++i) {
      F->prof_ms[i] = 0;
      F->prof_calls[i] = 0;
    }
    return TSF_OK;
  });
}

int tsf_profile_read(tsf_field* F, double* ms, int64_t* calls, int cap) {
  if (!F || cap < TSF_NSTAGES) return TSF_EINVAL;
  for (int i = 0; i < TSF_NSTAGES; ++i) {
    if (ms) ms[i] = F->prof_ms[i];
    if (calls) calls[i] = F->prof_calls[i];
  }
  return TSF_OK;
}

const char* tsf_stage_name(int s) {
  static const char* names[TSF_NSTAGES] = {"vertex_order", "gradient",      "critical_cells", "pairs_d0",
                                           "pairs_d2",     "pairs_d1_prep", "diagram_points", "assignment",
                                           "loss",         "gradient_step", "pairs_d1_morse", "pairs_d1_reduce"};
  return (s >= 0 && s < TSF_NSTAGES) ? names[s] : "unknown";
}

int64_t tsf_kernel_launches(void) { return (int64_t)tsf::launches(); }

int64_t tsf_debug_set(int what, int64_t value) { return tsf::set_knob(what, value); }

}  // extern "C"
