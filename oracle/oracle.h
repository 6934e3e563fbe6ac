/*
 * oracle.h -- plain, slow CPU oracle for the topological simplification solver.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code with the CUDA path.
 *
 * What it computes (paper: "A Practical Solver for Scalar Data Topological
 * Simplification"):
 *   - the lexicographic filtration of the Freudenthal triangulation of a
 *     regular grid (Section 2.1, Section 2.2) and its persistence pairs, by
 *     the textbook column reduction of the Z/2 boundary matrix (twist/clearing);
 *   - the persistence diagram: pairs whose birth and death vertices differ,
 *     plus the essential class at (f(v_min), f(v_max)) (Section 2.2);
 *   - the solver of Algorithm 1 with the direct gradient step (Section 4.1)
 *     and the still-pair reuse of the assignment (Section 4.3); the assignment
 *     itself is an exact minimum-cost matching by default (this project's
 *     reading), or the paper's approximate auction at a given relative
 *     precision.
 *
 * Cell ids: (dim << 60) | (base_vertex << 6) | type, where the simplex is the
 * chain base, base+A, base+A+B, base+(1,1,1) with axis masks A, B (x=1, y=2,
 * z=4): edges type = A, triangles type = 8*A + B, tetrahedra type = 8*A + B.
 */
#ifndef TSF_ORACLE_H
#define TSF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_diagram or_diagram;
typedef struct or_solver or_solver;

/* Full persistence of one field. status: 0 ok, -1 bad dims, -2 NaN/Inf, -3 no memory. */
or_diagram* or_diagram_compute(int lx, int ly, int lz, const float* f, int* status);
/* which: 0 = diagram pairs (v_b != v_d, plus essential), 1 = zero-persistence
 * pairs (v_b == v_d), 2 = number of simplices in the filtration. */
int64_t or_diagram_count(const or_diagram* d, int which);
void or_diagram_get(const or_diagram* d, int which, int32_t* dim, int32_t* essential,
                    uint32_t* vb, uint32_t* vd, uint64_t* cb, uint64_t* cd);
/* Every simplex, in filtration order. */
void or_diagram_filtration(const or_diagram* d, uint64_t* cells);
/* Vertex ranks (position of each vertex in the (value, id) order). */
void or_diagram_ranks(const or_diagram* d, uint32_t* rank);
void or_diagram_free(or_diagram* d);

/* Solver.  Signal = pairs of D(f0) with persistence >= tau * range(f0)
 * (fp32 arithmetic), plus the essential pair. */
or_solver* or_solver_create(int lx, int ly, int lz, const float* f0, float tau, int* status);
/* Explicit target diagram: n entries (dim, essential, vb, vd, birth, death).
 * The essential pair of D(f0) is added if no essential entry is given. */
or_solver* or_solver_create_targets(int lx, int ly, int lz, const float* f0, int64_t n,
                                    const int32_t* dim, const int32_t* essential,
                                    const uint32_t* vb, const uint32_t* vd,
                                    const float* birth, const float* death, int* status);
/* One iteration j -> j+1: gradient step with phi*_j, diagram of f_{j+1},
 * assignment phi*_{j+1}.  Returns 1 when the stop rule holds afterwards, 0 if
 * not, negative on error.  Stop rule: no diagonal-matched point with
 * persistence > cancel_eps, or (stop_s > 0 and loss_j <= stop_s * loss_0),
 * or j >= max_iters. */
int or_solver_iterate(or_solver* s, float alpha_b, float alpha_d, float stop_s, float cancel_eps,
                      int max_iters);
int or_solver_done(or_solver* s, float stop_s, float cancel_eps, int max_iters);
/* Section 4.3 fast assignment update on (default) or off for the following
 * iterations: off, every point of the new diagram is matched by the exact
 * solver instead of still points inheriting their previous assignment.  The
 * j = 0 assignment is the identity in both modes. */
void or_solver_set_fast_assignment(or_solver* s, int on);
/* Assignment of the following iterations: prec = 0 (default) the exact
 * reduced assignment; prec > 0 the Auction algorithm at that relative
 * precision (Section 5), its reduced Wasserstein distance sqrt(W2^2) within
 * a factor (1 + prec) of the optimum.  An iteration returns -4 if an
 * auction did not finish. */
void or_solver_set_assignment_precision(or_solver* s, double prec);
/* Topological loss of `values` (nv floats) against the target diagram:
 * diagram, full exact matching, *loss = Eq. 2 with q = 2, grad[nv] = dL/df
 * in fp64 (contributions added in diagram order, birth before death; the
 * essential class contributes at both its vertices).  The solver's state
 * becomes this field.  Returns 0, or a negative status. */
int or_solver_loss_grad(or_solver* s, const float* values, double* loss, double* grad);
/* Warm start: continue from the start field `values` with the same targets
 * and loss_0; its diagram is matched as after a step (Section 4.3), the
 * iteration count restarts at 0.  Returns 0, or negative on error. */
int or_solver_set_start(or_solver* s, const float* values);
void or_solver_field(const or_solver* s, float* out);
int64_t or_solver_num_points(const or_solver* s);
int64_t or_solver_num_targets(const or_solver* s);
/* Points of the current diagram, in diagram order. tgt = index into the target
 * list (target order) or -1 for the diagonal. */
void or_solver_points(const or_solver* s, int32_t* dim, int32_t* essential, uint32_t* vb,
                      uint32_t* vd, float* birth, float* death, int32_t* tgt, int32_t* still,
                      uint64_t* cb, uint64_t* cd);
void or_solver_targets(const or_solver* s, int32_t* dim, int32_t* essential, uint32_t* vb,
                       uint32_t* vd, float* birth, float* death);
/* stats[0]=iteration j, [1]=#uncancelled diagonal points, [2]=#still points,
 * [3]=#vertices whose value changed in the last step, [4]=#non-still points
 * matched to a target. loss[0]=loss_j, loss[1]=loss_0. */
void or_solver_stats(const or_solver* s, int64_t* stats, double* loss);
void or_solver_free(or_solver* s);

/* Exact reduced assignment on its own (for brute-force pins).  np points and
 * nt targets, all of one finite group; out_tgt[i] = target of point i or -1.
 * Returns the total W2^2 cost. */
double or_assign(int64_t np, const float* pb, const float* pd, int64_t nt, const float* tb,
                 const float* td, int32_t* out_tgt);
/* The same with the auction at relative precision prec (> 0; 0 is exact).
 * Returns -1.0 if the auction did not finish. */
double or_assign_prec(int64_t np, const float* pb, const float* pd, int64_t nt, const float* tb,
                      const float* td, double prec, int32_t* out_tgt);

#ifdef __cplusplus
}
#endif
#endif
