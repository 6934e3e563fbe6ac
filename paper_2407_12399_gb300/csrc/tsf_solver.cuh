// tsf_solver.cuh -- diagram points, targets and the solver's scratch buffers.
#pragma once
#include "tsf_kernels.cuh"

namespace tsf {

// A point of the persistence diagram (Section 2.2), with its assignment.
struct Pt {
  float b, d;        // f(v_b), f(v_d)
  uint32_t vb, vd;   // birth / death vertices
  uint64_t cb, cd;   // birth / death cells (cd = ~0 for the essential class)
  int32_t dim, ess;
  int32_t tgt;       // index into the target list, -1 = diagonal
  int32_t still;     // 1 if (dim, v_b, v_d) was in the previous diagram
};

// A point of the target diagram (Section 3).
struct Tg {
  float b, d;
  uint32_t vb, vd;
  uint64_t src;      // birth cell of the D(f0) pair it came from, or input index
  int32_t dim, ess;
};

struct Cand {
  double w;  // c(p,t) - diag(p)
  int32_t p; // index in the group's point list
  int32_t t; // index in the group's target list
};

struct Contrib {
  uint32_t v;
  uint32_t key;  // monotone key of c (summation order)
  float c;
  uint32_t pad;
};

struct HungWork {
  double* u;
  double* v;
  double* minv;
  int32_t* list;  // columns reached by the current row's search
  unsigned long long* key;  // auction: round-tagged winner of a column
  double* aw;               // auction: cost of each row's assigned option
  double* bw;               // auction: cost of each row's bid option
  int32_t* pm;
  int32_t* way;
  uint8_t* used;
};

// Device-side buffers of the reduced assignment.
struct AsgDev {
  int32_t* plist;      // non-still points, grouped: group g at [pbase[g], pbase[g]+np[g])
  int32_t* tlist;      // free targets, grouped the same way
  int32_t* counts;     // [0..3] np per group, [4..7] k per group, [8] overflow flag, [9] kept head
  Cand* kept;          // candidate lists, per target at kept_off[t], nkept[t] entries
  uint32_t* kept_off;  // per position in tlist
  uint32_t* nkept;
  uint32_t* is_col;    // per position in plist
  uint32_t* colpos;
  int32_t* col_point;
  int32_t* col_to_row;
  double* diag_t;
  HungWork H;          // arrays of np + nt + 8 entries, split per group
  int32_t* aux;        // auction: 4 x (np + nt + 8) ints, split per group
  int cap_kept;
};

struct SolverBufs {
  Pt* tmp_pts;
  int32_t *idxA, *idxB, *idxC, *idxD;
  int* count;
  uint32_t *u32a, *u32b, *u32c;
  uint8_t* taken;
  int32_t *plist, *tlist;
  Cand* cands;
  Cand* kept;
  uint32_t* nkept;
  uint32_t* is_col;
  uint32_t* colpos;
  int32_t* col_point;
  int32_t* aux;  // auction scratch of the group-by-group path: 4 x (cap_cols + 1)
  void* actl;    // control blocks (barrier, counters) of the grid auction, one per group
  int32_t* col_to_row;
  double* diag_t;
  HungWork H;
  double* terms;
  double* dsum;
  unsigned long long* counters;
  Contrib* contrib;
  int cap_k, cap_cand, cap_cols;
  int64_t cap_kept;
  AsgDev A;
  // key order (KeyLess) of the points of the last assignment: the next
  // iteration's reference diagram is that array, unchanged
  int32_t* keyord;
  const Pt* keyord_for;
  int keyord_n;
  // radix sorts of 64-bit keys: key halves, identity, sort scratch
  uint32_t* rsort;
  int64_t cap_rsort;  // items
  bool ids30;         // vertex ids fit 30 bits (the still-pair key packs two)
};

// Words of scratch a 64-bit-key radix sort of n items needs.
int64_t radix_sort64_words(int64_t n);

struct AssignStats {
  int k[4];
  uint32_t status;    // the status word, read with the group counts (fast path)
  bool status_valid;
  int32_t rounds;     // auction rounds (all groups)
  int32_t phases;     // auction eps phases (all groups)
  int32_t checks;     // auction release passes (all groups)
};

int build_diagram(const Dims& d, const NbrDelta& nd, const CritLists& L, int n1, int n2, int n3, const PairOut& P,
                  const uint32_t* order, const float* f, SolverBufs& B, Pt* out, int cap, cudaStream_t st);
int make_targets(int np, const Pt* pts, const uint32_t* order, const float* f, int64_t nv, float fraction,
                 SolverBufs& B, Tg* T, cudaStream_t st);
void targets_as_points(int nt, const Tg* T, Pt* R, cudaStream_t st);
// f[v] = in[v] where they differ, the changed vertices listed in upd, their
// number in *count.
void replace_values(int64_t nv, const float* in, float* f, uint32_t* upd, unsigned long long* count,
                    cudaStream_t st);
// dL/df (fp64, nv entries) of the topological loss for the current points
// and their matching.
void loss_gradient(int np, const Pt* pts, const Tg* T, SolverBufs& B, double* grad, int64_t nv, cudaStream_t st);
int assign(int np, Pt* pts, int nr, const Pt* ref, int nt, const Tg* T, double prec, SolverBufs& B, uint32_t* status,
           AssignStats* as, cudaStream_t st);
void loss_and_counts(int np, const Pt* pts, int nt, const Tg* T, float cancel_eps, SolverBufs& B, double* h_loss,
                     unsigned long long* h_counts, cudaStream_t st);
// One gradient step (Eq. 3); returns the number of vertices whose value
// changed and, with upd non-null, lists them there.
int64_t gradient_step(int np, const Pt* pts, const Tg* T, float alpha_b, float alpha_d, float* f, uint32_t* upd,
                      SolverBufs& B, uint32_t* status, cudaStream_t st);

}  // namespace tsf
