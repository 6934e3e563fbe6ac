/*
 * tsf.h -- C ABI of the GB300 topological simplification solver.
 *
 * The library implements the solver of "A Practical Solver for Scalar Data
 * Topological Simplification" (Algorithm 1 with the accelerations of
 * Sections 4.1-4.3) for a 3D fp32 scalar field on the Freudenthal
 * triangulation of a regular grid, every stage as a CUDA kernel on one GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid and values.  A field has lx * ly * lz vertices (each >= 2); vertex
 * (x, y, z) has id x + lx * (y + ly * z) and its value is values[id] (C order
 * of a (lz, ly, lx) array).  Values must be finite; -0.0 equals +0.0; equal
 * values are ordered by vertex id (Section 2.1).
 *
 * Cells.  A simplex is identified by (dim << 60) | (base << 6) | type, where
 * the simplex is the chain base, base+A, base+A+B, base+(1,1,1) of cube
 * corners (axis masks x = 1, y = 2, z = 4): an edge has type A, a triangle or
 * tetrahedron type 8*A + B, a vertex type 0.  The essential class has
 * cell_death = UINT64_MAX.
 *
 * Memory.  The library owns every device buffer of a field.  Pointers passed
 * in are owned by the caller; a flag next to each pointer says whether it is
 * a device pointer (1) or a host pointer (0).  All work is enqueued on the
 * CUDA stream given at creation (NULL = the legacy default stream), and every
 * call has finished on that stream when it returns.
 *
 * Errors.  Every function returns TSF_OK (0) or a negative code; no C++
 * exception crosses the boundary.  tsf_status_string() names a code.  A
 * device-side bound that was hit (a loop or wait limit) surfaces as
 * TSF_ETIMEOUT; the field stays usable.
 */
#ifndef TSF_H
#define TSF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TSF_OK 0
#define TSF_EINVAL (-1)      /* bad argument: null pointer, grid < 2 per axis, bad parameter */
#define TSF_ENAN (-2)        /* a value is NaN or infinite */
#define TSF_ENOMEM (-3)      /* device allocation failed */
#define TSF_ECUDA (-4)       /* a CUDA call failed */
#define TSF_ETIMEOUT (-5)    /* a device loop hit its bound; results of the call are invalid */
#define TSF_ENOTARGET (-6)   /* a solver call before a target diagram was set */
#define TSF_ECAPACITY (-7)   /* an output buffer is too small; *n_out holds the size needed */
#define TSF_EINTERNAL (-8)   /* an internal consistency check failed */

typedef struct tsf_field tsf_field;

/* One point of a persistence diagram (Section 2.2): the pair (sigma_b,
 * sigma_d) of the lexicographic filtration, its birth/death vertices (the
 * highest vertex of each simplex) and their values.  dim is the homology
 * dimension (0: minimum-1-saddle, 1: 1-saddle-2-saddle, 2: 2-saddle-maximum);
 * essential = 1 marks the class that never dies, reported at
 * (f(v_min), f(v_max)) (Section 2.2). */
typedef struct {
  int32_t dim;
  int32_t essential;
  uint32_t v_birth, v_death;
  uint64_t cell_birth, cell_death;
  float birth, death;
} tsf_pair; /* 40 bytes */

/* Solver parameters.
 * alpha_b, alpha_d: step sizes of the birth and death gradients (Section 4.1;
 *   0.5 is the paper's default, Section 5; alpha_d = 0 cuts handles and
 *   alpha_b = 0 fills them, Section 5.3).
 * stop_s: Algorithm 1 stops once loss_j <= stop_s * loss_0 (<= 0: off; the
 *   paper uses 0.01).
 * cancel_eps: the solver also stops once no diagonal-matched point has
 *   persistence > cancel_eps (every non-signal pair cancelled).
 * max_iters: j_max of Algorithm 1 (the paper uses 1000).
 * fast_gradient_update: 1 recomputes the gradient only around vertices the
 *   last step changed (Section 4.2); 0 recomputes it everywhere.  Results are
 *   identical either way.
 * fast_assignment_update: 1 lets still pairs keep their previous assignment
 *   and matches only the others (Section 4.3); 0 matches every point of the
 *   new diagram with the solver.  The j = 0 assignment is the identity
 *   either way.
 * assignment_precision: 0 solves each reduced assignment exactly (shortest
 *   augmenting paths); p > 0 uses the Auction algorithm, as the paper's
 *   implementation does (Section 5, p = 0.01), whose reduced Wasserstein
 *   distance sqrt(W2^2) is within a factor (1 + p) of the minimum: much
 *   faster when many targets compete for the same points.  Deterministic
 *   either way.  Must be finite, >= 0. */
typedef struct {
  float alpha_b, alpha_d;
  float stop_s;
  float cancel_eps;
  int32_t max_iters;
  int32_t fast_gradient_update;
  int32_t fast_assignment_update;
  float assignment_precision;
} tsf_params;

/* Per-iteration statistics. */
typedef struct {
  int32_t iters;              /* j */
  int32_t done;               /* 1 when the stop rule holds */
  double loss0, loss;         /* W2^2 between D(f_0) / D(f_j) and the target (Eq. 2) */
  int64_t n_points;           /* points of D(f_j), essential class included */
  int64_t n_pairs[3];         /* finite points per dimension */
  int64_t n_critical[4];      /* critical vertices, edges, triangles, tetrahedra */
  int64_t n_uncancelled;      /* diagonal-matched points with persistence > cancel_eps */
  int64_t n_still;            /* points still since the previous iteration (Section 4.3) */
  int64_t n_nonstill_matched; /* non-still points matched to a target */
  int64_t n_updated_vertices; /* vertices whose value the last step changed */
  int64_t n_gradient_vertices;/* lower stars recomputed by the last diagram */
  int64_t d1_columns;         /* saddle-saddle columns (negative critical triangles) */
  int64_t d1_blocks_total;    /* lower stars visited to build their Morse boundaries */
  int64_t d1_blocks_max;      /* ... by the largest column */
  int64_t d1_rounds_total;    /* rounds (32 lower stars at most each) over all columns */
  int64_t d1_rounds_max;      /* ... of the longest column */
  int64_t d1_star_updates;    /* parity-mask updates of target lower stars by those visits */
  double ms_diagram, ms_assign, ms_step; /* host wall time of the three stages */
  int64_t assign_rounds;      /* auction rounds of the last assignment (0 when exact) */
  int64_t assign_phases;      /* ... its eps phases */
  int64_t assign_checks;      /* ... its passes releasing rows off eps-complementary slackness */
  int64_t d1_reduce_rounds;   /* rounds of the saddle-saddle column reduction */
  int64_t d1_reduce_merged;   /* entries written by its column additions */
  int64_t d1_reduce_longest;  /* longest column an addition produced */
  int64_t d1_reduce_big_rounds; /* its rounds with at least 4096 active columns */
  int64_t d1_reduce_big_cycles; /* SM clock cycles spent in those rounds */
  int64_t d1_reduce_cycles;     /* SM clock cycles of the whole reduction */
  int64_t d1_chain_adds;        /* additions chained in its short rounds (at most 64 active columns) */
  int64_t d1_chain_longest;     /* ... by one column in one round, at most */
  int64_t d1_chain_rounds;      /* its short rounds */
  int64_t d1_chain_cycles;      /* SM clock cycles spent in those rounds */
} tsf_stats;

/* Creates a field from lx*ly*lz values (host or device memory, copied),
 * on the device current at this call; every later call on the field runs
 * on that device and leaves the caller's current device as it was.
 * cuda_stream: a cudaStream_t, or NULL.  Errors: TSF_EINVAL, TSF_ENAN,
 * TSF_ENOMEM, TSF_ECUDA.  On success *out owns all device memory. */
int tsf_create_field(int lx, int ly, int lz, const float* values, int values_on_device, void* cuda_stream,
                     tsf_field** out);

/* Frees the field and its device memory.  NULL is accepted. */
int tsf_destroy_field(tsf_field* field);

/* Persistence diagram D(f) of the field's current values (Section 2.2; the
 * pairs of the lexicographic filtration whose birth and death vertices
 * differ, plus the essential class), in diagram order: increasing birth, then
 * death (Section 2.4), then birth vertex, death vertex and birth cell.
 * out: cap entries (host or device per out_on_device), may be NULL when cap
 * is 0.  *n_out receives the number of points; TSF_ECAPACITY if cap is too
 * small (nothing written). */
int tsf_compute_diagram(tsf_field* field, tsf_pair* out, int64_t cap, int64_t* n_out, int out_on_device);

/* Target diagram (Section 3) = D(f_0) without the non-signal pairs, where a
 * pair is signal when its persistence fl(death - birth) >= fl(fraction *
 * fl(max f_0 - min f_0)); the essential class is always kept.  f_0 is the
 * field's current values.  Resets the solver to iteration 0 and assigns
 * every signal point to itself (Section 4.3).  Errors: TSF_EINVAL if
 * fraction < 0. */
int tsf_set_signal_threshold(tsf_field* field, float fraction_of_range);

/* Explicit target diagram: n host-memory points (dim, essential, v_birth,
 * v_death, birth, death are used; cells are ignored).  The essential class of
 * D(f_0) is added when no entry is essential.  Iteration 0 assigns each point
 * of D(f_0) to the target with the same (dim, essential, v_birth, v_death),
 * and the rest by the exact reduced assignment. */
int tsf_set_signal_pairs(tsf_field* field, const tsf_pair* pairs, int64_t n);

/* One solver iteration j -> j+1 (Algorithm 1): gradient step with phi*_j
 * (Section 4.1), diagram of f_{j+1} (Sections 2.2, 4.2), assignment
 * phi*_{j+1} (Section 4.3, exact).  stats may be NULL.  Errors:
 * TSF_ENOTARGET before a target was set, TSF_EINVAL for bad parameters. */
int tsf_solver_step(tsf_field* field, const tsf_params* params, tsf_stats* stats);

/* Iterates tsf_solver_step until the stop rule holds, then copies the field
 * to out_values (lx*ly*lz floats, host or device; may be NULL). */
int tsf_simplify(tsf_field* field, const tsf_params* params, float* out_values, int out_on_device, tsf_stats* stats);

/* Copies the current values to out (lx*ly*lz floats, host or device). */
int tsf_get_field(tsf_field* field, float* out, int out_on_device);

/* Topological loss of a field against the target diagram (Eq. 2 with q = 2:
 * squared distances of the points matched to targets to those targets, of
 * the others to the diagonal, plus unmatched targets to the diagonal) and
 * its gradient with respect to the field values.  values: lx*ly*lz floats
 * (host or device), which become the field's values (the diagram follows
 * the vertices they change, Section 4.2); every point of the diagram is
 * matched by the exact solver (no still-pair reuse).  *loss (host) receives
 * L in fp64; grad (may be NULL), lx*ly*lz doubles (host or device),
 * receives dL/df for that diagram and matching: 2 (b - t_b) at v_b and
 * 2 (d - t_d) at v_d for a point matched to target t (the essential class
 * included), b - d and d - b for a point matched to the diagonal, added per
 * vertex in diagram order (Section 4.1's gradient without the step size).
 * It is the derivative of L wherever a small change of the values changes
 * neither the pairing nor the matching.
 * Errors: TSF_EINVAL, TSF_ENOTARGET before a target was set, TSF_ENAN. */
int tsf_loss_and_gradient(tsf_field* field, const float* values, int values_on_device, double* loss,
                          double* grad, int grad_on_device);

/* A batch of independent fields solved together.  The paper solves one
 * field at a time (Algorithm 1); a batch runs many such solves at once:
 * every field gets its own non-blocking CUDA stream and one host thread of
 * a small pool drives it, so the kernels of different fields run
 * concurrently.  Each field's iteration is exactly tsf_solver_step /
 * tsf_simplify on it, so a field's result does not depend on its batch.
 *
 * tsf_batch_create: n fields, field i of lx[i]*ly[i]*lz[i] values copied
 *   from values[i] (host or device); the batch owns fields and streams, all
 *   on the device current at this call (its worker threads select it too).
 *   Errors: TSF_EINVAL, TSF_ENOMEM, TSF_ECUDA, TSF_ENAN.
 * tsf_batch_field: the i-th field (owned by the batch; use it with the
 *   single-field calls, but not while a batch call runs).
 * tsf_batch_set_signal_thresholds: tsf_set_signal_threshold(field i,
 *   fractions[i]) for every field, concurrently.
 * tsf_batch_step: one tsf_solver_step of every field; stats (may be NULL)
 *   has n entries.  tsf_batch_simplify: tsf_simplify of every field (no
 *   copy-out; read fields with tsf_get_field).  Both return the first
 *   non-zero status of the fields, after all of them finished. */
typedef struct tsf_batch tsf_batch;
int tsf_batch_create(int n, const int* lx, const int* ly, const int* lz, const float* const* values,
                     int values_on_device, tsf_batch** out);
int tsf_batch_destroy(tsf_batch* batch);
int tsf_batch_size(const tsf_batch* batch);
int tsf_batch_field(tsf_batch* batch, int i, tsf_field** out);
int tsf_batch_set_signal_thresholds(tsf_batch* batch, const float* fractions);
int tsf_batch_step(tsf_batch* batch, const tsf_params* params, tsf_stats* stats);
int tsf_batch_simplify(tsf_batch* batch, const tsf_params* params, tsf_stats* stats);
/* Autotuner of the batch (not in the paper): times the full persistence
 * diagram of every field (all fields concurrently, each candidate twice,
 * the second pass counted) for each candidate schedule of the D1 Morse
 * boundaries' first phase — 0: half a warp per column with 64 + 128
 * frontier and stage entries, 1: half a warp with 32 + 64, 2: a quarter of
 * a warp with 16 + 32, 3: one warp with 64 + 128 (tsf_debug_set knob 7
 * values 7, 5, 6, 4) — and keeps the fastest.  The choice applies
 * process-wide; results never depend on it.  *choice receives it (0..3),
 * ms[c] (cap entries, may be NULL when cap is 0) the time of candidate c in
 * milliseconds.  Call it before the signal thresholds are set (it replaces
 * each field's current diagram): TSF_EINVAL if a field has a target
 * diagram. */
int tsf_batch_autotune(tsf_batch* batch, int* choice, double* ms, int cap);

/* Overwrites the current values (restart from a saved field; the still-pair
 * history is reset, so the next assignment starts cold). */
int tsf_set_field(tsf_field* field, const float* values, int values_on_device);

/* Warm start (not in the paper): replaces the current values by a start
 * field g0 (lx*ly*lz floats, host or device) and keeps the target diagram
 * and loss_0 of the field the targets were set from.  The diagram of g0 is
 * computed (Sections 2.2, 4.2) and matched as after a solver step: points
 * with the (dim, v_b, v_d) of a point of the current diagram keep its
 * assignment, the rest go to the exact reduced assignment (Section 4.3);
 * the solver restarts at iteration 0 from g0, so tsf_simplify's stop rule
 * L <= stop_s * loss_0 refers to the original field's loss.  Errors:
 * TSF_EINVAL, TSF_ENOTARGET before a target was set, TSF_ENAN. */
int tsf_set_start_field(tsf_field* field, const float* values, int values_on_device);

/* The current assignment, in the order of the last diagram: target[i] is the
 * index of point i's target in the target list (tsf_get_targets), or -1 for
 * the diagonal; still[i] is 1 for still points.  Host memory, cap entries
 * each (either may be NULL). */
int tsf_get_assignment(tsf_field* field, int32_t* target, int32_t* still, int64_t cap, int64_t* n_out);

/* The target diagram, in target order (diagram order of the targets), host memory. */
int tsf_get_targets(tsf_field* field, tsf_pair* out, int64_t cap, int64_t* n_out);

/* Every zero-persistence pair (Section 2.2: v_b == v_d) of the current
 * values, as cell ids: out[2k] = birth cell, out[2k+1] = death cell (host
 * memory, unordered).  These are the pairs of the lower-star discrete
 * gradient (Section 4.2); intended for verification on small grids. */
int tsf_zero_pairs(tsf_field* field, uint64_t* out, int64_t cap_pairs, int64_t* n_out);

/* Diagnostics.  With profiling on, every stage of the solver is bracketed by
 * CUDA events on the field's stream and its device time accumulated (this
 * adds a stream synchronisation per stage).  Stages, in pipeline order:
 * 0 vertex order (sort + ranks), 1 lower-star gradient, 2 critical cells,
 * 3 D0 pairs, 4 D2 pairs, 5 D1 candidate columns, 6 diagram points,
 * 7 assignment, 8 loss, 9 gradient step, 10 D1 Morse boundaries, 11 D1
 * column reduction.  tsf_profile_read fills ms[] and calls[] (cap >=
 * TSF_NSTAGES entries each) with the totals since profiling was enabled;
 * enabling again resets them. */
#define TSF_NSTAGES 12
int tsf_profile_enable(tsf_field* field, int enable);
int tsf_profile_read(tsf_field* field, double* ms, int64_t* calls, int cap);
const char* tsf_stage_name(int stage);

/* Number of kernels this library has launched in this process. */
int64_t tsf_kernel_launches(void);

/* Test and tuning knobs of the pairing (process-wide, not in the paper;
 * results never depend on them, only the schedule and the bounds):
 *   1: items from which the union-find rounds run over the whole GPU
 *      (default 65536; below, one block runs them);
 *   2: active items below which one block finishes the rounds (default 8192);
 *   3: cap on the union-find rounds (default 0 = none; a cap that is hit
 *      makes the call fail with TSF_ETIMEOUT);
 *   4: polls a block waits at a grid barrier of the whole-GPU rounds (union-
 *      find and D1 reduction) before it gives up (default 2^24; giving up
 *      makes the call fail with TSF_ETIMEOUT);
 *   5: D1 columns from which the reduction rounds run over the whole GPU
 *      (default 65536);
 *   6: active D1 columns below which one block finishes them (default 4096);
 *   7: schedule of the D1 Morse boundaries' first phase: 0 the default
 *      (half a warp per column, registers capped for 32 warps per SM; 64 +
 *      128 frontier and stage entries for diagrams of at least 2^19
 *      critical triangles, else 32 + 64), 1 and 2 one warp per column with
 *      128 + 256 and 256 + 512 entries, 3 one warp with 64 + 128 without
 *      the register cap, 4 the same with it, 5 half a warp with 32 + 64, 6
 *      a quarter of a warp with 16 + 32, 7 half a warp with 64 + 128 at any
 *      size (columns that outgrow their buffers continue in the second
 *      phase);
 *   8: register budget of the lower-star gradient kernels, as blocks of
 *      128 threads per SM: 0 the default (6), 1 no cap, 2 five;
 *   9: entries of a column that the D1 reduction's short rounds (at most 64
 *      active columns) keep in shared memory while they chain additions,
 *      with one warp per column (default and maximum 512; the larger groups
 *      of the last columns scale it with their size; longer sums, or all
 *      with 0, are added in the column pool);
 *  10: lower-star visits a thread of the D1 Morse boundaries chains in one
 *      round along updates with a single target star (0: the default, 1
 *      for diagrams of at least 2^19 critical triangles, else 2; at most 8);
 *  11: rounds of the D1 Morse boundaries' first phase before a column
 *      moves to a block of the second (0: the default, 128 for diagrams of
 *      at least 2^19 critical triangles, else 16);
 *  12: active columns up to which a round of the D1 reduction chains
 *      additions in shared memory (0: the default, 64; at most 1024).
 * Returns the previous value, or -1 for an unknown knob.  Set them only
 * while no call of this library is running. */
int64_t tsf_debug_set(int what, int64_t value);

/* After a step that changed at most this many vertex values, the next
 * diagram merges the changed vertices into the previous vertex order instead
 * of sorting all values again (the result is the same order). */
#define TSF_INCREMENTAL_ORDER_MAX 8192

/* Zero-persistence pairs without device allocation.  The paper has no
 * counterpart: this is a service for callers that cannot call cudaMalloc,
 * e.g. code running inside a framework that owns all device memory through
 * its own pool, or a latency-critical loop where cudaMalloc's implicit
 * device-wide synchronisation is not acceptable.  Same result as
 * tsf_zero_pairs for the same values (as a set; the order is unspecified).
 *
 * values: device pointer to lx*ly*lz floats (layout as tsf_create_field);
 * out: device pointer to cap_pairs pairs (out[2k] = birth cell, out[2k+1] =
 * death cell), may be NULL when cap_pairs is 0; *n_out (host) receives the
 * number of pairs, TSF_ECAPACITY when it exceeds cap_pairs.  lx*ly*lz above
 * TSF_STATIC_MAX_VERTICES is rejected with TSF_EINVAL.
 *
 * All intermediate data lives in one fixed device array of about 6.6 MB
 * (sized for TSF_STATIC_MAX_VERTICES vertices) that every GPU loading this
 * library holds until the process exits.  Every call shares that array and
 * finds the previous call's contents in it; calls that overlap on the GPU
 * (other streams, other threads) race and must be serialised by the caller.
 * The first call on each device looks up the array's device address with
 * that device current.  Every call ends by copying the pair count and the
 * status word to the host and synchronising cuda_stream, so a call cannot
 * be recorded into a CUDA graph.  Errors as tsf_zero_pairs: TSF_EINVAL,
 * TSF_ENAN (a NaN or infinite value), TSF_ETIMEOUT (a bounded device wait
 * of the sort gave up), TSF_ECAPACITY, TSF_ECUDA, TSF_EINTERNAL. */
#define TSF_STATIC_MAX_VERTICES 262144
int tsf_zero_pairs_static(int lx, int ly, int lz, const float* values, uint64_t* out, int64_t cap_pairs,
                          int64_t* n_out, void* cuda_stream);

/* Learned warm start.  The paper has no learned component: this network
 * proposes a starting field g0 for a field f, and the solver (Algorithm 1)
 * then refines g0 against f's own target diagram, judging the result.
 *
 * Network: a 3-level 3D U-Net on an (lz, ly, lx) grid (each side a multiple
 * of 4, at least 8), channels 16/32/64; per level two 3x3x3 convolutions
 * with zero padding, bias and ReLU; 2x2x2 average pooling down, nearest x2
 * upsampling up, the skip features concatenated after the upsampled ones; a
 * 1x1 head to one channel.  Inputs: f and a constant channel holding the
 * threshold fraction tau; output g0 = f + head.  Weights and activations
 * are stored in bfloat16 and every sum is accumulated in fp32; the
 * convolutions run on the tensor cores.  Training minimises mean((g0 -
 * g)^2) over the voxels by Adam (beta1 0.9, beta2 0.999, eps 1e-8) on an
 * fp32 master copy of the parameters.
 *
 * Parameters: TSF_UNET_NPARAMS floats, layer by layer in the order e1a e1b
 * e2a e2b e3a e3b d2a d2b d1a d1b head; per convolution the weights
 * (cout, cin, 3, 3, 3) indexed (dz, dy, dx) as a cross-correlation, then the
 * cout biases; the head's 16 weights, then its bias.  Channels: e1a 2->16,
 * e1b 16->16, e2a 16->32, e2b 32->32, e3a 32->64, e3b 64->64, d2a 96->32
 * (upsampled e3b, then e2b), d2b 32->32, d1a 48->16 (upsampled d2b, then
 * e1b), d1b 16->16.
 *
 * tsf_unet_create: a network from host parameters, on the device current at
 *   this call; work is enqueued on cuda_stream (NULL = legacy default) and
 *   every call has finished when it returns.  Errors: TSF_EINVAL (n !=
 *   TSF_UNET_NPARAMS), TSF_ENOMEM.
 * tsf_unet_get_params: the current fp32 parameters (host, n floats).
 * tsf_unet_forward: g0 for the field f (lx*ly*lz floats, layout as
 *   tsf_create_field); f and g0 both host or both device (on_device).
 * tsf_unet_gradients: loss mean((g0 - g)^2) (*loss, fp64, may be NULL) and
 *   its gradient with respect to every parameter (grad: host, n floats, may
 *   be NULL) for the pair (f, g), without an update.
 * tsf_unet_train_step: the same, then one Adam step with learning rate lr.
 * tsf_unet_debug: every layer's stored activation as fp32 (host acts, in the
 *   order x e1a e1b e2a e2b e3a e3b d2a d2b d1a d1b g0, each (C, z, y, x) at
 *   its level: full grid for x e1a e1b d1a d1b g0, half for e2a e2b d2a d2b,
 *   quarter for e3a e3b) and, when g is not NULL, every convolution's
 *   gradient with respect to its pre-activation output (host gz, order d1b
 *   d1a d2b d2a e3b e3a e2b e2a e1b e1a); TSF_ECAPACITY if a buffer is too
 *   small.  For verification; f and g are host memory.
 * Grid errors: TSF_EINVAL.  A bounded device wait that gave up:
 *   TSF_ETIMEOUT. */
typedef struct tsf_unet tsf_unet;
#define TSF_UNET_NPARAMS 353713
int64_t tsf_unet_num_params(void);
int tsf_unet_create(const float* params, int64_t n, void* cuda_stream, tsf_unet** out);
int tsf_unet_destroy(tsf_unet* net);
int tsf_unet_get_params(tsf_unet* net, float* out, int64_t n);
int tsf_unet_forward(tsf_unet* net, int lx, int ly, int lz, const float* f, float tau, float* g0, int on_device);
int tsf_unet_gradients(tsf_unet* net, int lx, int ly, int lz, const float* f, const float* g, int on_device, float tau,
                       float* grad, double* loss);
int tsf_unet_train_step(tsf_unet* net, int lx, int ly, int lz, const float* f, const float* g, int on_device,
                        float tau, float lr, double* loss);
int tsf_unet_debug(tsf_unet* net, int lx, int ly, int lz, const float* f, const float* g, float tau, float* acts,
                   int64_t acts_cap, float* gz, int64_t gz_cap);

/* Human-readable name of a status code. */
const char* tsf_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* TSF_H */
