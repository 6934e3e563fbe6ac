// tsf_kernels.cuh -- buffers shared between kernel translation units, and the
// host-side launch functions each unit exports to the C-ABI layer.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "tsf_internal.cuh"

namespace tsf {

enum : uint32_t { kErrNaN = 1u << 7 };

// C-ABI status of a device status word: NaN/Inf input, then any bound that
// was hit (trace steps, rounds, spin-waits), then internal inconsistencies.
// The values are those of TSF_ENAN, TSF_ETIMEOUT and TSF_EINTERNAL.
inline int status_code(uint32_t s) {
  if (s & kErrNaN) return -2;
  if (s & (kErrTrace | kErrRounds | kErrSpin)) return -5;
  if (s & (kErrInconsistent | kErrEmptyColumn | kErrCapacity | kErrPool)) return -8;
  return 0;
}

// Stable sort of n (key, value) pairs by the u32 key (four 8-bit onesweep
// passes); keys_out may be null; scratch holds sort_scratch_words(n) words.
void sort_u32_pairs(const uint32_t* keys, const uint32_t* vals, int64_t n, uint32_t* keys_out, uint32_t* vals_out,
                    uint32_t* scratch, uint32_t* status, cudaStream_t st);

// Test and tuning knobs of the pairing kernels (tsf_debug_set); returns the
// previous value, -1 for an unknown knob.
int64_t set_knob(int what, int64_t value);
int64_t get_knob(int what);

// Number of kernels this library has launched (process-wide).
void note_launch();
long long launches();

// Critical cells, each list in lexicographic order (Section 2.2).
struct CritLists {
  uint32_t* c0;       // minima: vertex id
  uint64_t* c1_key;   // critical edges: (rank_hi << 32) | rank_lo
  uint32_t* c1_vn;    // critical edges: (v << 4) | neighbour index of the lower end
  uint32_t* c2_ve;    // critical triangles: (v << 6) | link edge index
  uint32_t* c3;       // maxima: (v << 5) | link triangle index
  int cap0, cap1, cap2, cap3;
};

// Neighbour offsets as vertex-id deltas for one grid.
struct NbrDelta {
  int32_t d[14];
};

// Persistence pairs of the critical cells.
struct PairOut {
  int32_t* d0_min;     // per critical edge: index of the minimum it kills, -1
  int32_t* d2_max;     // per critical triangle: index of the maximum it kills, -1
  int32_t* d1_edge;    // per critical triangle: critical edge paired (D1), -1
  uint8_t* d0_killed;  // per critical edge: 1 if it is a D0 death (negative)
  uint32_t* d0mask;    // per vertex: bit a set if the critical edge v*a is a D0 death
};

// ---- k_sort.cu -----------------------------------------------------------
int64_t sort_scratch_words(int64_t n);
// Full vertex order: order[] (vertex ids by (value, id)), rank[] its inverse
// and, with skey non-null, skey[i] = value_key of order[i].
void vertex_order(const float* f, int64_t n, uint32_t* order, uint32_t* rank, uint32_t* skey, uint32_t* scratch,
                  uint32_t* status, cudaStream_t st);

// ---- k_order.cu ----------------------------------------------------------
// Largest number of updated vertices the incremental order update takes.
constexpr int kIncOrderMax = 8192;
// New order2/skey2/rank from the old order/skey/rank and the nu vertices upd[]
// whose values changed.  Scratch: ubits (n/32 + 1 words), ucnt
// (order_count_words(n) words), B (kIncOrderMax double words).
void vertex_order_incremental(const float* f, int64_t n, const uint32_t* upd, int nu, const uint32_t* order,
                              const uint32_t* skey, uint32_t* order2, uint32_t* skey2, uint32_t* rank,
                              uint32_t* ubits, uint32_t* ucnt, unsigned long long* B, uint32_t* status,
                              cudaStream_t st);
int64_t order_count_words(int64_t n);
void exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* sums, cudaStream_t st);

// ---- k_gradient.cu -------------------------------------------------------
void launch_gradient(const Dims& d, const uint32_t* rank, const float* f, Rec* rec, uint8_t* vnext8, D1Tab* tab,
                     uint32_t* status, cudaStream_t st);
// Recomputes the lower stars of the nu updated vertices upd[] and of their
// neighbours; *count receives how many (listed in list[], nv entries).
void launch_gradient_incremental(const Dims& d, const uint32_t* rank, const float* f, const uint32_t* upd, int64_t nu,
                                 uint32_t* mark, uint32_t gen, uint32_t* list, unsigned long long* count, Rec* rec,
                                 uint8_t* vnext8, D1Tab* tab, uint32_t* status, cudaStream_t st);
int crit_tiles(int64_t nv);
void launch_crit_count(const Dims& d, const uint32_t* order, const Rec* rec, int4* tile_counts, int4* totals,
                       cudaStream_t st);
void launch_crit_write(const Dims& d, const uint32_t* order, const uint32_t* rank, const Rec* rec,
                       const int4* tile_off, const CritLists& L, uint32_t* cidx, uint32_t* c1base, uint32_t* c2base,
                       uint32_t* status, cudaStream_t st);
void launch_zero_pairs(const Dims& d, const uint32_t* rank, unsigned long long* out, int64_t cap,
                       unsigned long long* count, uint32_t* status, cudaStream_t st);

// ---- k_pairs.cu ----------------------------------------------------------
struct PairScratch {
  int32_t* ends;      // 2 per item: component endpoints
  int32_t* parent;    // union-find parents over nodes
  int32_t* reserve;   // per node reservation
  int32_t* listA;     // active item lists
  int32_t* listB;
  int32_t* roots;     // 2 per item
  int32_t* counter;   // device counters (>= 4 ints)
};
void launch_d0(const Dims& d, const NbrDelta& nd, const CritLists& L, int n0, int n1, const uint8_t* vnext8,
               const uint32_t* cidx, PairScratch& S, PairOut& P, uint32_t* status, cudaStream_t st);
void launch_d2(const Dims& d, const NbrDelta& nd, const CritLists& L, int n2, int n3, const uint32_t* rank,
               const Rec* rec, const uint32_t* cidx, PairScratch& S, PairOut& P, uint32_t* status,
               cudaStream_t st);

// Control block of the whole-GPU D1 reduction rounds.
struct D1Ctl {
  unsigned bar[2];  // grid barrier: arrivals, generation
  int n[2];         // lengths of the two column lists
  int which;        // list holding the active columns
  int rounds;       // rounds done
  int pad[10];
};

// Counters of the D1 stages (D1Work::stats): [0] lower stars visited, [1]
// by the largest column, [2] rounds over all columns, [3] of the longest,
// [4] target-star updates, [5] reduction rounds, [6] entries merged, [7]
// longest sum, [8] whole-GPU rounds, [9] their cycles, [10] all cycles of
// the reduction, [11] chained additions of the short rounds, [12] the
// longest chain of one column in one round, [13] short rounds, [14] their
// cycles.
constexpr int kD1Stats = 16;

struct D1Work {
  int32_t* cols;          // candidate triangle index per column
  unsigned long long* low;  // current low per column (0 = to be recomputed)
  uint32_t* hoff;         // heap offset in the pool
  uint32_t* hcap;         // heap capacity
  uint32_t* hsize;        // heap size
  int32_t* lowc;          // critical edge index of the low
  int32_t* owner;         // per critical edge: smallest column holding it as low
  uint4* orec;            // ... and that column's {index, pool offset, length} while it owns it
  unsigned long long* pool;
  uint32_t pool_cap;
  uint32_t* pool_head;
  int32_t* flags;         // [0] changed, [1] number of candidate columns
  unsigned long long* stats;  // [0] lower stars visited, [1] max per column
  int32_t* redo;          // columns whose warp frontier overflowed
  uint4* cont;            // open columns after phase A: frontier off/size, output off/size
  uint32_t* cont_cap;     // ... output capacity
  int32_t* big;           // list of open columns
  int32_t* nbig;
};
// D1: candidate columns (their number in W.flags[1]), Morse boundaries,
// reduction; grids are sized by n2, the kernels read the column count.
void launch_d1_prepare(int n2, D1Work& W, PairOut& P, cudaStream_t st);
void launch_d1_morse(const Dims& d, const NbrDelta& nd, const CritLists& L, int n1, int n2, const uint32_t* rank,
                     const uint32_t* order, const float* f, const Rec* rec, const D1Tab* tab, const uint32_t* c1base,
                     D1Work& W, PairOut& P, uint32_t* status, cudaStream_t st);
void launch_d1_reduce(int n1, int n2, D1Work& W, PairOut& P, uint32_t* status, D1Ctl* ctl, cudaStream_t st);

}  // namespace tsf
