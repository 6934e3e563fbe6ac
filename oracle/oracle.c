/*
 * oracle.c -- plain, slow CPU oracle for the topological simplification solver.
 *
 * TEST INFRASTRUCTURE ONLY.  The product path never includes, links or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code with the CUDA path.
 *
 * Everything here follows the paper's definitions literally, with no
 * blocking, fusion or reordering beyond them:
 *   - Section 2.1: the field lives on the vertices of the Freudenthal
 *     triangulation of the grid; ties are broken by vertex id (a variant of
 *     simulation of simplicity), -0.0 and +0.0 compare equal.
 *   - Section 2.2: every simplex is the list of its vertices' positions in
 *     the global vertex order, sorted decreasingly; simplices are ordered
 *     lexicographically (a proper prefix sorts first).  The persistence pairs
 *     of that filtration come from the standard column reduction of the Z/2
 *     boundary matrix (here with the twist/clearing shortcut, which does not
 *     change the pairs).  v_b / v_d are the highest vertices of the birth /
 *     death simplices; pairs with v_b == v_d are zero-persistence pairs and
 *     are not points of the diagram; the one essential class is reported at
 *     (f(v_min), f(v_max)).
 *   - Section 3 / Eq. 2: the target diagram is D(f0) without the non-signal
 *     pairs; the energy is W2(D(f), D_T)^2 (Eq. 1 with q = 2).
 *   - Section 4.1: the direct gradient step, birth and death gradients with
 *     step sizes alpha_b, alpha_d.
 *   - Section 4.3: still pairs (same v_b and v_d as a pair of the previous
 *     diagram) keep their previous assignment; the rest is solved on the
 *     reduced diagram against the reduced target.
 *   - Algorithm 1: the iteration order (step, diagram, assignment).
 * Where the paper is silent, the reading taken is stated at the function
 * that implements it.
 */
#include "oracle.h"

#include <float.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Grid and Freudenthal triangulation (Section 2.1).                         */
/* A simplex is a chain base < base+A < base+A+B < base+(1,1,1) of vertices  */
/* of one grid cube, each step adding a disjoint non-empty set of axes.      */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t lx, ly, lz, nv;
} grid_t;

static void vcoords(const grid_t* g, int64_t v, int64_t c[3]) {
  c[0] = v % g->lx;
  c[1] = (v / g->lx) % g->ly;
  c[2] = v / (g->lx * g->ly);
}

static int64_t vplus(const grid_t* g, int64_t v, int mask) {
  return v + ((mask & 1) ? 1 : 0) + ((mask & 2) ? g->lx : 0) + ((mask & 4) ? g->lx * g->ly : 0);
}

static int mask_fits(const grid_t* g, int64_t v, int mask) {
  int64_t c[3];
  vcoords(g, v, c);
  if ((mask & 1) && c[0] + 1 >= g->lx) return 0;
  if ((mask & 2) && c[1] + 1 >= g->ly) return 0;
  if ((mask & 4) && c[2] + 1 >= g->lz) return 0;
  return 1;
}

static int vdiff_mask(const grid_t* g, int64_t lo, int64_t hi) {
  int64_t a[3], b[3];
  vcoords(g, lo, a);
  vcoords(g, hi, b);
  int m = 0;
  for (int k = 0; k < 3; ++k) {
    int64_t d = b[k] - a[k];
    if (d == 1) m |= (1 << k);
    else if (d != 0) return -1;
  }
  return m;
}

#define CELL(dim, base, type) (((uint64_t)(dim) << 60) | ((uint64_t)(base) << 6) | (uint64_t)(type))
#define CELL_DIM(c) ((int)((c) >> 60))
#define CELL_BASE(c) ((int64_t)(((c) >> 6) & ((1ull << 54) - 1)))
#define CELL_TYPE(c) ((int)((c)&63))

/* Vertices of a cell in chain order; returns dim+1. */
static int cell_chain(const grid_t* g, uint64_t cell, int64_t w[4]) {
  int dim = CELL_DIM(cell);
  int64_t base = CELL_BASE(cell);
  int type = CELL_TYPE(cell);
  w[0] = base;
  if (dim == 1) w[1] = vplus(g, base, type);
  if (dim >= 2) {
    int a = type >> 3, b = type & 7;
    w[1] = vplus(g, base, a);
    w[2] = vplus(g, w[1], b);
  }
  if (dim == 3) w[3] = vplus(g, base, 7);
  return dim + 1;
}

static uint64_t chain_cell(const grid_t* g, const int64_t* w, int n) {
  int dim = n - 1;
  if (dim == 0) return CELL(0, w[0], 0);
  if (dim == 1) return CELL(1, w[0], vdiff_mask(g, w[0], w[1]));
  return CELL(dim, w[0], vdiff_mask(g, w[0], w[1]) * 8 + vdiff_mask(g, w[1], w[2]));
}

/* Compact per-dimension type index (for the cell -> position table). */
static int NT[4] = {1, 7, 12, 6};
static int type_compact[4][64];
static int type_list[4][12];
static int tables_ready = 0;

static void init_tables(void) {
  if (tables_ready) return;
  for (int d = 0; d < 4; ++d)
    for (int t = 0; t < 64; ++t) type_compact[d][t] = -1;
  type_compact[0][0] = 0;
  type_list[0][0] = 0;
  for (int m = 1; m < 8; ++m) {
    type_compact[1][m] = m - 1;
    type_list[1][m - 1] = m;
  }
  int n2 = 0, n3 = 0;
  for (int a = 1; a < 8; ++a)
    for (int b = 1; b < 8; ++b) {
      if (a & b) continue;
      int t = a * 8 + b;
      type_compact[2][t] = n2;
      type_list[2][n2++] = t;
      int single = (a == 1 || a == 2 || a == 4) && (b == 1 || b == 2 || b == 4);
      if (single) {
        type_compact[3][t] = n3;
        type_list[3][n3++] = t;
      }
    }
  tables_ready = 1;
}

static int cell_exists(const grid_t* g, int dim, int64_t base, int type) {
  if (dim == 0) return 1;
  int u = (dim == 1) ? type : (dim == 2 ? ((type >> 3) | (type & 7)) : 7);
  return mask_fits(g, base, u);
}

/* ------------------------------------------------------------------------ */
/* Global vertex order (Section 2.1, Section 2.2).                           */
/* ------------------------------------------------------------------------ */

/* Monotone map float -> uint32 (total order of the values; -0.0 == +0.0). */
static uint32_t value_key(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if (u == 0x80000000u) u = 0;
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

static const float* g_sort_f;
static int cmp_vertex(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  uint32_t kx = value_key(g_sort_f[x]), ky = value_key(g_sort_f[y]);
  if (kx != ky) return kx < ky ? -1 : 1;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* ------------------------------------------------------------------------ */
/* Lexicographic filtration (Section 2.2).                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t cell;
  uint32_t key[4]; /* vertex ranks, decreasing; only dim+1 entries used */
} simplex_t;

static int cmp_simplex(const void* a, const void* b) {
  const simplex_t* x = (const simplex_t*)a;
  const simplex_t* y = (const simplex_t*)b;
  int nx = CELL_DIM(x->cell) + 1, ny = CELL_DIM(y->cell) + 1;
  int n = nx < ny ? nx : ny;
  for (int i = 0; i < n; ++i)
    if (x->key[i] != y->key[i]) return x->key[i] < y->key[i] ? -1 : 1;
  /* a proper prefix sorts first */
  return nx < ny ? -1 : (nx > ny ? 1 : 0);
}

typedef struct {
  int32_t dim, ess;
  uint32_t vb, vd;
  uint64_t cb, cd;
} rawpair_t;

struct or_diagram {
  grid_t g;
  int64_t nsimp;
  uint64_t* filtration; /* cells in filtration order */
  uint32_t* rank;
  rawpair_t* pairs;
  int64_t npairs;
  rawpair_t* zpairs;
  int64_t nzpairs;
};

/* Sorted-set symmetric difference (Z/2 column addition). */
static int64_t xor_merge(const uint32_t* a, int64_t na, const uint32_t* b, int64_t nb, uint32_t* out) {
  int64_t i = 0, j = 0, k = 0;
  while (i < na && j < nb) {
    if (a[i] < b[j]) out[k++] = a[i++];
    else if (b[j] < a[i]) out[k++] = b[j++];
    else {
      ++i;
      ++j;
    }
  }
  while (i < na) out[k++] = a[i++];
  while (j < nb) out[k++] = b[j++];
  return k;
}

static int cmp_u32(const void* a, const void* b) {
  uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

static void diag_free_internal(or_diagram* d) {
  if (!d) return;
  free(d->filtration);
  free(d->rank);
  free(d->pairs);
  free(d->zpairs);
  free(d);
}

or_diagram* or_diagram_compute(int lx, int ly, int lz, const float* f, int* status) {
  init_tables();
  if (status) *status = 0;
  if (lx < 2 || ly < 2 || lz < 2) {
    if (status) *status = -1;
    return NULL;
  }
  grid_t g = {lx, ly, lz, (int64_t)lx * ly * lz};
  for (int64_t v = 0; v < g.nv; ++v)
    if (!isfinite(f[v])) {
      if (status) *status = -2;
      return NULL;
    }
  or_diagram* D = (or_diagram*)calloc(1, sizeof(or_diagram));
  D->g = g;

  /* vertex order: sort ids by (value, id) */
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * g.nv);
  D->rank = (uint32_t*)malloc(sizeof(uint32_t) * g.nv);
  for (int64_t v = 0; v < g.nv; ++v) order[v] = v;
  g_sort_f = f;
  qsort(order, g.nv, sizeof(int64_t), cmp_vertex);
  for (int64_t r = 0; r < g.nv; ++r) D->rank[order[r]] = (uint32_t)r;

  /* enumerate every simplex with its key */
  int64_t ns = 0;
  for (int64_t v = 0; v < g.nv; ++v)
    for (int d = 0; d < 4; ++d)
      for (int t = 0; t < NT[d]; ++t) ns += cell_exists(&g, d, v, type_list[d][t]);
  simplex_t* S = (simplex_t*)malloc(sizeof(simplex_t) * ns);
  int64_t k = 0;
  for (int64_t v = 0; v < g.nv; ++v)
    for (int d = 0; d < 4; ++d)
      for (int t = 0; t < NT[d]; ++t) {
        int type = type_list[d][t];
        if (!cell_exists(&g, d, v, type)) continue;
        uint64_t c = CELL(d, v, type);
        int64_t w[4];
        int n = cell_chain(&g, c, w);
        uint32_t r[4] = {0, 0, 0, 0};
        for (int i = 0; i < n; ++i) r[i] = D->rank[w[i]];
        /* sort decreasing */
        for (int i = 1; i < n; ++i)
          for (int j = i; j > 0 && r[j] > r[j - 1]; --j) {
            uint32_t tmp = r[j];
            r[j] = r[j - 1];
            r[j - 1] = tmp;
          }
        S[k].cell = c;
        memcpy(S[k].key, r, sizeof(r));
        ++k;
      }
  qsort(S, ns, sizeof(simplex_t), cmp_simplex);
  D->nsimp = ns;
  D->filtration = (uint64_t*)malloc(sizeof(uint64_t) * ns);
  for (int64_t i = 0; i < ns; ++i) D->filtration[i] = S[i].cell;

  /* cell -> filtration position */
  uint32_t* pos[4];
  for (int d = 0; d < 4; ++d) pos[d] = (uint32_t*)malloc(sizeof(uint32_t) * g.nv * NT[d]);
  for (int64_t i = 0; i < ns; ++i) {
    uint64_t c = S[i].cell;
    int d = CELL_DIM(c);
    pos[d][CELL_BASE(c) * NT[d] + type_compact[d][CELL_TYPE(c)]] = (uint32_t)i;
  }

  /* Column reduction with twist: dimensions 3, 2, 1 in turn, each column in
   * filtration order; a column whose low is already the low of an earlier
   * column gets that (reduced) column added. */
  const uint32_t NONE = 0xFFFFFFFFu;
  uint32_t* pivot_col = (uint32_t*)malloc(sizeof(uint32_t) * ns); /* row -> column */
  uint8_t* cleared = (uint8_t*)calloc(ns, 1);
  uint8_t* has_col = (uint8_t*)calloc(ns, 1);
  int64_t* col_off = (int64_t*)malloc(sizeof(int64_t) * ns);
  int64_t* col_len = (int64_t*)malloc(sizeof(int64_t) * ns);
  for (int64_t i = 0; i < ns; ++i) pivot_col[i] = NONE;
  int64_t pool_cap = 1 << 20, pool_n = 0;
  uint32_t* pool = (uint32_t*)malloc(sizeof(uint32_t) * pool_cap);
  int64_t wcap = 1 << 16;
  uint32_t* work = (uint32_t*)malloc(sizeof(uint32_t) * wcap);
  uint32_t* tmp = (uint32_t*)malloc(sizeof(uint32_t) * wcap);

  for (int dim = 3; dim >= 1; --dim) {
    for (int64_t j = 0; j < ns; ++j) {
      uint64_t c = S[j].cell;
      if (CELL_DIM(c) != dim || cleared[j]) continue;
      int64_t w[4], fw[3];
      int n = cell_chain(&g, c, w);
      int64_t nw = 0;
      for (int drop = 0; drop < n; ++drop) {
        int m = 0;
        for (int i = 0; i < n; ++i)
          if (i != drop) fw[m++] = w[i];
        uint64_t fc = chain_cell(&g, fw, n - 1);
        int fd = CELL_DIM(fc);
        work[nw++] = pos[fd][CELL_BASE(fc) * NT[fd] + type_compact[fd][CELL_TYPE(fc)]];
      }
      qsort(work, nw, sizeof(uint32_t), cmp_u32);
      while (nw > 0) {
        uint32_t low = work[nw - 1];
        uint32_t p = pivot_col[low];
        if (p == NONE) {
          pivot_col[low] = (uint32_t)j;
          cleared[low] = 1;
          has_col[j] = 1;
          if (pool_n + nw > pool_cap) {
            while (pool_n + nw > pool_cap) pool_cap *= 2;
            pool = (uint32_t*)realloc(pool, sizeof(uint32_t) * pool_cap);
          }
          memcpy(pool + pool_n, work, sizeof(uint32_t) * nw);
          col_off[j] = pool_n;
          col_len[j] = nw;
          pool_n += nw;
          break;
        }
        int64_t need = nw + col_len[p];
        if (need > wcap) {
          while (need > wcap) wcap *= 2;
          work = (uint32_t*)realloc(work, sizeof(uint32_t) * wcap);
          tmp = (uint32_t*)realloc(tmp, sizeof(uint32_t) * wcap);
        }
        nw = xor_merge(work, nw, pool + col_off[p], col_len[p], tmp);
        uint32_t* sw = work;
        work = tmp;
        tmp = sw;
      }
    }
  }

  /* collect pairs */
  int64_t np = 0, nz = 0;
  for (int64_t i = 0; i < ns; ++i)
    if (pivot_col[i] != NONE) {
      uint32_t vb = (uint32_t)order[S[i].key[0]];
      uint32_t vd = (uint32_t)order[S[pivot_col[i]].key[0]];
      if (vb == vd) ++nz;
      else ++np;
    }
  int64_t ness = 0;
  for (int64_t i = 0; i < ns; ++i)
    if (pivot_col[i] == NONE && !has_col[i]) ++ness;
  D->pairs = (rawpair_t*)malloc(sizeof(rawpair_t) * (np + ness + 1));
  D->zpairs = (rawpair_t*)malloc(sizeof(rawpair_t) * (nz + 1));
  int64_t a = 0, b = 0;
  uint32_t vmax = (uint32_t)order[g.nv - 1];
  for (int64_t i = 0; i < ns; ++i) {
    if (pivot_col[i] != NONE) {
      rawpair_t P;
      P.dim = CELL_DIM(S[i].cell);
      P.ess = 0;
      P.vb = (uint32_t)order[S[i].key[0]];
      P.vd = (uint32_t)order[S[pivot_col[i]].key[0]];
      P.cb = S[i].cell;
      P.cd = S[pivot_col[i]].cell;
      if (P.vb == P.vd) D->zpairs[b++] = P;
      else D->pairs[a++] = P;
    } else if (!has_col[i]) {
      rawpair_t P;
      P.dim = CELL_DIM(S[i].cell);
      P.ess = 1;
      P.vb = (uint32_t)order[S[i].key[0]];
      P.vd = vmax;
      P.cb = S[i].cell;
      P.cd = ~(uint64_t)0;
      D->pairs[a++] = P;
    }
  }
  D->npairs = a;
  D->nzpairs = b;

  free(pivot_col);
  free(cleared);
  free(has_col);
  free(col_off);
  free(col_len);
  free(pool);
  free(work);
  free(tmp);
  for (int d = 0; d < 4; ++d) free(pos[d]);
  free(S);
  free(order);
  return D;
}

int64_t or_diagram_count(const or_diagram* d, int which) {
  if (which == 0) return d->npairs;
  if (which == 1) return d->nzpairs;
  return d->nsimp;
}

void or_diagram_get(const or_diagram* d, int which, int32_t* dim, int32_t* essential, uint32_t* vb,
                    uint32_t* vd, uint64_t* cb, uint64_t* cd) {
  const rawpair_t* P = which == 0 ? d->pairs : d->zpairs;
  int64_t n = which == 0 ? d->npairs : d->nzpairs;
  for (int64_t i = 0; i < n; ++i) {
    dim[i] = P[i].dim;
    essential[i] = P[i].ess;
    vb[i] = P[i].vb;
    vd[i] = P[i].vd;
    cb[i] = P[i].cb;
    cd[i] = P[i].cd;
  }
}

void or_diagram_filtration(const or_diagram* d, uint64_t* cells) {
  memcpy(cells, d->filtration, sizeof(uint64_t) * d->nsimp);
}

void or_diagram_ranks(const or_diagram* d, uint32_t* rank) {
  memcpy(rank, d->rank, sizeof(uint32_t) * d->g.nv);
}

void or_diagram_free(or_diagram* d) { diag_free_internal(d); }

/* ------------------------------------------------------------------------ */
/* Solver (Algorithm 1 with Sections 4.1 and 4.3).                           */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t dim, ess;
  uint32_t vb, vd;
  uint64_t cb, cd;
  float b, d;
  int32_t tgt, still;
} opoint_t;

typedef struct {
  int32_t dim, ess;
  uint32_t vb, vd;
  float b, d;
  uint64_t src; /* birth cell of the D(f0) pair it came from, or input index */
} otarget_t;

struct or_solver {
  grid_t g;
  float* f;
  otarget_t* T;
  int64_t nt;
  opoint_t* P;
  int64_t np;
  int64_t j;
  double loss, loss0;
  int64_t n_unc, n_still, n_updated, n_nssp;
  int fast_assign; /* Section 4.3 still-pair reuse after each step (default on) */
  double assign_prec; /* 0: exact reduced assignment; > 0: auction at this relative precision */
};

/* Diagram order: increasing birth, then death (Section 2.4); the remaining
 * keys (birth vertex, death vertex, dimension, essential flag, birth cell,
 * death cell) are this project's tie-break, making the order total. */
static int cmp_point(const void* a, const void* b) {
  const opoint_t* x = (const opoint_t*)a;
  const opoint_t* y = (const opoint_t*)b;
  if (x->b < y->b) return -1;
  if (x->b > y->b) return 1;
  if (x->d < y->d) return -1;
  if (x->d > y->d) return 1;
  if (x->vb != y->vb) return x->vb < y->vb ? -1 : 1;
  if (x->vd != y->vd) return x->vd < y->vd ? -1 : 1;
  if (x->dim != y->dim) return x->dim < y->dim ? -1 : 1;
  if (x->ess != y->ess) return x->ess < y->ess ? -1 : 1;
  if (x->cb != y->cb) return x->cb < y->cb ? -1 : 1;
  if (x->cd != y->cd) return x->cd < y->cd ? -1 : 1;
  return 0;
}

static int cmp_target(const void* a, const void* b) {
  const otarget_t* x = (const otarget_t*)a;
  const otarget_t* y = (const otarget_t*)b;
  if (x->b < y->b) return -1;
  if (x->b > y->b) return 1;
  if (x->d < y->d) return -1;
  if (x->d > y->d) return 1;
  if (x->vb != y->vb) return x->vb < y->vb ? -1 : 1;
  if (x->vd != y->vd) return x->vd < y->vd ? -1 : 1;
  if (x->dim != y->dim) return x->dim < y->dim ? -1 : 1;
  if (x->ess != y->ess) return x->ess < y->ess ? -1 : 1;
  if (x->src != y->src) return x->src < y->src ? -1 : 1;
  return 0;
}

/* The persistence diagram D(f) as points with their values, in diagram order. */
static int compute_points(const grid_t* g, const float* f, opoint_t** out, int64_t* nout) {
  int st = 0;
  or_diagram* D = or_diagram_compute((int)g->lx, (int)g->ly, (int)g->lz, f, &st);
  if (!D) return st ? st : -3;
  opoint_t* P = (opoint_t*)malloc(sizeof(opoint_t) * (D->npairs + 1));
  for (int64_t i = 0; i < D->npairs; ++i) {
    P[i].dim = D->pairs[i].dim;
    P[i].ess = D->pairs[i].ess;
    P[i].vb = D->pairs[i].vb;
    P[i].vd = D->pairs[i].vd;
    P[i].cb = D->pairs[i].cb;
    P[i].cd = D->pairs[i].cd;
    P[i].b = f[P[i].vb];
    P[i].d = f[P[i].vd];
    P[i].tgt = -1;
    P[i].still = 0;
  }
  qsort(P, D->npairs, sizeof(opoint_t), cmp_point);
  *out = P;
  *nout = D->npairs;
  diag_free_internal(D);
  return 0;
}

/* --- costs (Eq. 1 with q = 2; diagonal projection of Section 2.3) --------- */
/* fp64 from fp32 inputs; every operation rounded on its own (no FMA). */
static double cost_pt(float pb, float pd, float tb, float td) {
  double db = (double)pb - (double)tb;
  double dd = (double)pd - (double)td;
  double s1 = db * db;
  double s2 = dd * dd;
  return s1 + s2;
}

static double cost_diag(float b, float d) {
  double e = (double)d - (double)b;
  double s = e * e;
  return s * 0.5;
}

typedef struct {
  double w;
  int64_t p;
} cand_t;

static int cmp_cand(const void* a, const void* b) {
  const cand_t* x = (const cand_t*)a;
  const cand_t* y = (const cand_t*)b;
  if (x->w < y->w) return -1;
  if (x->w > y->w) return 1;
  return x->p < y->p ? -1 : (x->p > y->p ? 1 : 0);
}

/*
 * Exact minimum of W2^2 (Eq. 1, q = 2) between points P and targets T of one
 * finite group, each side augmented with the other's diagonal projections and
 * diagonal-to-diagonal matches free (Section 2.3).
 *
 * Reading (the paper uses an approximate auction): a target t either takes a
 * point p, at cost c(p,t), or stays on the diagonal, at diag(t); every point
 * left over goes to its own projection at diag(p).  Up to the constant sum of
 * diag(p), the objective is the sum over targets of w(p,t) = c(p,t) - diag(p)
 * (matched) or diag(t) (unmatched).  Only pairs with w(p,t) < diag(t) can
 * help, and a target never needs more than its k = |T| cheapest such points
 * (one of them is always free), so each target keeps those, ordered by
 * (w, point index).  The resulting k x m problem (m = candidate points + one
 * private diagonal column per target) is solved exactly with the shortest
 * augmenting path method (Hungarian algorithm with potentials), rows in target
 * order, ties to the lowest column index.
 */
static int auction_rows(int64_t k, int64_t np, const int64_t* cand_p, const double* cand_w, const int64_t* ncand,
                        const float* pb, const float* pd, const float* tb, const float* td, double prec,
                        int32_t* out);

static int assign_group(int64_t np, const float* pb, const float* pd, int64_t nt, const float* tb,
                        const float* td, double prec, int32_t* out) {
  for (int64_t i = 0; i < np; ++i) out[i] = -1;
  if (nt == 0 || np == 0) return 0;
  int64_t k = nt;
  cand_t* buf = (cand_t*)malloc(sizeof(cand_t) * np);
  int64_t* cand_p = (int64_t*)malloc(sizeof(int64_t) * k * k);
  double* cand_w = (double*)malloc(sizeof(double) * k * k);
  int64_t* ncand = (int64_t*)calloc(k, sizeof(int64_t));
  uint8_t* is_col = (uint8_t*)calloc(np, 1);
  for (int64_t t = 0; t < k; ++t) {
    double dt = cost_diag(tb[t], td[t]);
    int64_t nb = 0;
    for (int64_t p = 0; p < np; ++p) {
      double w = cost_pt(pb[p], pd[p], tb[t], td[t]) - cost_diag(pb[p], pd[p]);
      if (w < dt) {
        buf[nb].w = w;
        buf[nb].p = p;
        ++nb;
      }
    }
    qsort(buf, nb, sizeof(cand_t), cmp_cand);
    int64_t keep = nb < k ? nb : k;
    for (int64_t i = 0; i < keep; ++i) {
      cand_p[t * k + i] = buf[i].p;
      cand_w[t * k + i] = buf[i].w;
      is_col[buf[i].p] = 1;
    }
    ncand[t] = keep;
  }
  if (prec > 0.0) {
    int st = auction_rows(k, np, cand_p, cand_w, ncand, pb, pd, tb, td, prec, out);
    free(buf);
    free(cand_p);
    free(cand_w);
    free(ncand);
    free(is_col);
    return st;
  }
  /* columns: candidate points in point order, then k private diagonal columns */
  int64_t mc = 0;
  int64_t* col_of_p = (int64_t*)malloc(sizeof(int64_t) * np);
  int64_t* p_of_col = (int64_t*)malloc(sizeof(int64_t) * (np + 1));
  for (int64_t p = 0; p < np; ++p) {
    col_of_p[p] = -1;
    if (is_col[p]) {
      col_of_p[p] = mc;
      p_of_col[mc++] = p;
    }
  }
  int64_t m = mc + k;
  const double INF = HUGE_VAL;
  double* u = (double*)calloc(k + 1, sizeof(double));
  double* v = (double*)calloc(m + 1, sizeof(double));
  double* minv = (double*)malloc(sizeof(double) * (m + 1));
  double* row = (double*)malloc(sizeof(double) * (m + 1));
  int64_t* pm = (int64_t*)calloc(m + 1, sizeof(int64_t));
  int64_t* way = (int64_t*)calloc(m + 1, sizeof(int64_t));
  uint8_t* used = (uint8_t*)malloc(m + 1);
  for (int64_t i = 1; i <= k; ++i) {
    pm[0] = i;
    int64_t j0 = 0;
    for (int64_t j = 0; j <= m; ++j) {
      minv[j] = INF;
      used[j] = 0;
    }
    do {
      used[j0] = 1;
      int64_t i0 = pm[j0];
      double delta = INF;
      int64_t j1 = 0;
      /* row i0 of the cost matrix (1-based columns) */
      for (int64_t j = 1; j <= m; ++j) row[j] = INF;
      for (int64_t c = 0; c < ncand[i0 - 1]; ++c) row[1 + col_of_p[cand_p[(i0 - 1) * k + c]]] = cand_w[(i0 - 1) * k + c];
      row[1 + mc + (i0 - 1)] = cost_diag(tb[i0 - 1], td[i0 - 1]);
      for (int64_t j = 1; j <= m; ++j) {
        if (used[j]) continue;
        double cur = row[j] - u[i0] - v[j];
        if (cur < minv[j]) {
          minv[j] = cur;
          way[j] = j0;
        }
        if (minv[j] < delta) {
          delta = minv[j];
          j1 = j;
        }
      }
      for (int64_t j = 0; j <= m; ++j) {
        if (used[j]) {
          u[pm[j]] += delta;
          v[j] -= delta;
        } else {
          minv[j] -= delta;
        }
      }
      j0 = j1;
    } while (pm[j0] != 0);
    do {
      int64_t j1 = way[j0];
      pm[j0] = pm[j1];
      j0 = j1;
    } while (j0);
  }
  for (int64_t j = 1; j <= mc; ++j)
    if (pm[j] != 0) out[p_of_col[j - 1]] = (int32_t)(pm[j] - 1);
  free(buf);
  free(cand_p);
  free(cand_w);
  free(ncand);
  free(is_col);
  free(col_of_p);
  free(p_of_col);
  free(u);
  free(v);
  free(minv);
  free(row);
  free(pm);
  free(way);
  free(used);
  return 0;
}

/*
 * Approximate reduced assignment by the Auction algorithm (Bertsekas; the
 * paper's implementation, Section 5, runs it at relative precision 0.01),
 * on the same rows (targets in order) and options (kept candidates, then
 * the private diagonal column, which comes after every point column) as the
 * exact solve.  Net cost of an option: w(r,j) + price(j).
 *
 * Forward auction in synchronous (Jacobi) rounds:
 *   - every unassigned row r finds its lowest net cost n1 (ties: lowest
 *     column) at column j1 and the lowest net cost n2 among its other
 *     options, and bids price(j1) + ((n2 - n1) + eps) for j1;
 *   - each point column takes its highest bid (ties: lowest row), its price
 *     becomes that bid, its previous row is unassigned; a bid for the row's
 *     own diagonal always wins;
 * until every row is assigned.  A row with no candidate takes its diagonal.
 *
 * eps-scaling: eps starts at max diag(t) / 4 and is divided by 5 per
 * phase.  Each later phase keeps the previous assignment and prices, except
 * that (repeatedly, until nothing changes) every column without a row gets
 * price 0 and every row whose net cost exceeds its lowest one by more than
 * the new eps is released.  So at the end of a phase every column without a
 * row has price 0 (a column once bid on keeps a row) and the prices give the
 * dual bound LB = sum_r min_j (w(r,j) + price(j)) - sum_j price(j) <= the
 * optimum, with W - LB <= k * eps for the assignment's cost W.  One step of
 * block coordinate ascent on the dual (prices lowered to
 * p'(j) = max(0, max_r (u_r - w(r,j))) for the row values u_r above, then
 * the row values raised to min_j (w(r,j) + p'(j))) gives a second bound; LB
 * is the larger.  The auction stops after the first phase with
 * W + D <= (1 + prec)^2 (LB + D), D the sum of diag(p) over the points: the
 * reduced Wasserstein distance sqrt(W2^2) within a factor (1 + prec) of
 * its minimum, the paper's relative precision; or once eps reaches
 * 2^-40 max diag(t).  Sums run in row order, prices in column order
 * (points, then diagonals).
 * Returns 0, or -1 if 2^24 rounds did not finish.
 */
static int auction_rows(int64_t k, int64_t np, const int64_t* cand_p, const double* cand_w, const int64_t* ncand,
                        const float* pb, const float* pd, const float* tb, const float* td, double prec,
                        int32_t* out) {
  const double INF = HUGE_VAL;
  double* diag_t = (double*)malloc(sizeof(double) * k);
  double* price = (double*)calloc(np + k, sizeof(double)); /* point columns, then diagonals */
  double* pt = (double*)malloc(sizeof(double) * (np + k));  /* tightened prices */
  int64_t* owner = (int64_t*)malloc(sizeof(int64_t) * np);
  int64_t* rowcol = (int64_t*)malloc(sizeof(int64_t) * k);
  int64_t* bcol = (int64_t*)malloc(sizeof(int64_t) * k);
  double* bid = (double*)malloc(sizeof(double) * k);
  int64_t* win = (int64_t*)malloc(sizeof(int64_t) * np);
  double* best = (double*)malloc(sizeof(double) * np);
  uint8_t* viol = (uint8_t*)malloc(k);
  double dsum = 0.0, cmax = 0.0;
  for (int64_t r = 0; r < k; ++r) {
    diag_t[r] = cost_diag(tb[r], td[r]);
    if (diag_t[r] > cmax) cmax = diag_t[r];
    rowcol[r] = ncand[r] > 0 ? -1 : np + r;
  }
  for (int64_t p = 0; p < np; ++p) {
    dsum += cost_diag(pb[p], pd[p]);
    owner[p] = -1;
    win[p] = -1;
  }
  double emin = ldexp(cmax, -40);
  if (!(emin > 0.0)) emin = DBL_MIN;
  double eps = cmax * 0.25;
  if (eps < emin) eps = emin;
  double onep = 1.0 + prec; /* the precision is on W2 = sqrt(W2^2) */
  onep = onep * onep;
  int st = 0;
  int64_t rounds = 0;
  for (int phase = 0;; ++phase) {
    if (phase > 0) {
      for (;;) { /* release the rows that break eps-complementary slackness */
        for (int64_t p = 0; p < np; ++p)
          if (owner[p] < 0) price[p] = 0.0;
        for (int64_t r = 0; r < k; ++r)
          if (rowcol[r] != np + r) price[np + r] = 0.0;
        int64_t nviol = 0;
        for (int64_t r = 0; r < k; ++r) {
          viol[r] = 0;
          if (rowcol[r] < 0) continue; /* released earlier in this cascade */
          double n1 = INF, cur = INF;
          for (int64_t c = 0; c <= ncand[r]; ++c) {
            int64_t j = c < ncand[r] ? cand_p[r * k + c] : np + r;
            double w = c < ncand[r] ? cand_w[r * k + c] : diag_t[r];
            double n = w + price[j];
            if (n < n1) n1 = n;
            if (j == rowcol[r]) cur = n;
          }
          double lim = n1 + eps;
          if (cur > lim) {
            viol[r] = 1;
            ++nviol;
          }
        }
        if (nviol == 0) break;
        for (int64_t r = 0; r < k; ++r) {
          if (!viol[r]) continue;
          if (rowcol[r] < np) owner[rowcol[r]] = -1;
          rowcol[r] = -1;
        }
      }
    }
    for (;; ++rounds) {
      if (rounds >= ((int64_t)1 << 24)) {
        st = -1;
        break;
      }
      int64_t nun = 0;
      for (int64_t r = 0; r < k; ++r) {
        bcol[r] = -1;
        if (rowcol[r] >= 0) continue;
        ++nun;
        double n1 = INF, n2 = INF;
        int64_t j1 = -1;
        for (int64_t c = 0; c <= ncand[r]; ++c) {
          int64_t j = c < ncand[r] ? cand_p[r * k + c] : np + r;
          double w = c < ncand[r] ? cand_w[r * k + c] : diag_t[r];
          double n = w + price[j];
          if (n < n1 || (n == n1 && j < j1)) {
            n2 = n1;
            n1 = n;
            j1 = j;
          } else if (n < n2) {
            n2 = n;
          }
        }
        double g = n2 - n1;
        g = g + eps;
        bid[r] = price[j1] + g;
        bcol[r] = j1;
      }
      if (nun == 0) break;
      for (int64_t r = 0; r < k; ++r) {
        int64_t j = bcol[r];
        if (j < 0) continue;
        if (j >= np) { /* the row's own diagonal: no competition */
          price[j] = bid[r];
          rowcol[r] = j;
          bcol[r] = -1;
        } else if (win[j] < 0 || bid[r] > best[j]) { /* rows in increasing order: ties keep the lower */
          win[j] = r;
          best[j] = bid[r];
        }
      }
      for (int64_t r = 0; r < k; ++r) {
        int64_t j = bcol[r];
        if (j < 0 || win[j] != r) continue;
        if (owner[j] >= 0) rowcol[owner[j]] = -1;
        owner[j] = r;
        rowcol[r] = j;
        price[j] = bid[r];
      }
      for (int64_t r = 0; r < k; ++r)
        if (bcol[r] >= 0) win[bcol[r]] = -1;
    }
    if (st) break;
    /* phase end: the assignment's cost W and the dual bound LB */
    double W = 0.0, U = 0.0, P = 0.0;
    for (int64_t r = 0; r < k; ++r) {
      double n1 = INF, wcur = INF;
      for (int64_t c = 0; c <= ncand[r]; ++c) {
        int64_t j = c < ncand[r] ? cand_p[r * k + c] : np + r;
        double w = c < ncand[r] ? cand_w[r * k + c] : diag_t[r];
        double n = w + price[j];
        if (n < n1) n1 = n;
        if (j == rowcol[r]) wcur = w;
      }
      W += wcur;
      U += n1;
    }
    for (int64_t j = 0; j < np + k; ++j) P += price[j];
    double lb = U - P;
    /* one step of block coordinate ascent on the dual: every price down to
     * what the row values u_r = min_j (w(r,j) + price(j)) need, then the
     * row values up to their new minima; still a dual bound, often tighter */
    for (int64_t j = 0; j < np + k; ++j) pt[j] = 0.0;
    for (int64_t r = 0; r < k; ++r) {
      double u = INF;
      for (int64_t c = 0; c <= ncand[r]; ++c) {
        int64_t j = c < ncand[r] ? cand_p[r * k + c] : np + r;
        double w = c < ncand[r] ? cand_w[r * k + c] : diag_t[r];
        double n = w + price[j];
        if (n < u) u = n;
      }
      for (int64_t c = 0; c <= ncand[r]; ++c) {
        int64_t j = c < ncand[r] ? cand_p[r * k + c] : np + r;
        double w = c < ncand[r] ? cand_w[r * k + c] : diag_t[r];
        double need = u - w;
        if (need > pt[j]) pt[j] = need;
      }
    }
    double U2 = 0.0, P2 = 0.0;
    for (int64_t r = 0; r < k; ++r) {
      double u = INF;
      for (int64_t c = 0; c <= ncand[r]; ++c) {
        int64_t j = c < ncand[r] ? cand_p[r * k + c] : np + r;
        double w = c < ncand[r] ? cand_w[r * k + c] : diag_t[r];
        double n = w + pt[j];
        if (n < u) u = n;
      }
      U2 += u;
    }
    for (int64_t j = 0; j < np + k; ++j) P2 += pt[j];
    double lb2 = U2 - P2;
    if (lb2 > lb) lb = lb2;
    double lhs = W + dsum;
    double rhs = lb + dsum;
    rhs = rhs * onep;
    if (lhs <= rhs || !(eps > emin)) break;
    eps = eps / 5.0;
    if (eps < emin) eps = emin;
  }
  if (st == 0)
    for (int64_t p = 0; p < np; ++p) out[p] = owner[p] >= 0 ? (int32_t)owner[p] : -1;
  free(diag_t);
  free(price);
  free(pt);
  free(owner);
  free(rowcol);
  free(bcol);
  free(bid);
  free(win);
  free(best);
  free(viol);
  return st;
}

double or_assign(int64_t np, const float* pb, const float* pd, int64_t nt, const float* tb, const float* td,
                 int32_t* out_tgt) {
  return or_assign_prec(np, pb, pd, nt, tb, td, 0.0, out_tgt);
}

double or_assign_prec(int64_t np, const float* pb, const float* pd, int64_t nt, const float* tb, const float* td,
                      double prec, int32_t* out_tgt) {
  if (assign_group(np, pb, pd, nt, tb, td, prec, out_tgt)) return -1.0;
  double total = 0.0;
  uint8_t* taken = (uint8_t*)calloc(nt + 1, 1);
  for (int64_t i = 0; i < np; ++i) {
    if (out_tgt[i] >= 0) {
      total += cost_pt(pb[i], pd[i], tb[out_tgt[i]], td[out_tgt[i]]);
      taken[out_tgt[i]] = 1;
    } else {
      total += cost_diag(pb[i], pd[i]);
    }
  }
  for (int64_t t = 0; t < nt; ++t)
    if (!taken[t]) total += cost_diag(tb[t], td[t]);
  free(taken);
  return total;
}

static int group_of(int32_t dim, int32_t ess) { return ess ? 3 : dim; }

/* Key order used to match points with equal (dim, essential, v_b, v_d):
 * duplicates pair up in (birth cell, death cell) order. */
static const opoint_t* g_keyP;
static int cmp_key_idx(const void* a, const void* b) {
  const opoint_t* x = &g_keyP[*(const int64_t*)a];
  const opoint_t* y = &g_keyP[*(const int64_t*)b];
  if (x->ess != y->ess) return x->ess < y->ess ? -1 : 1;
  if (x->dim != y->dim) return x->dim < y->dim ? -1 : 1;
  if (x->vb != y->vb) return x->vb < y->vb ? -1 : 1;
  if (x->vd != y->vd) return x->vd < y->vd ? -1 : 1;
  if (x->cb != y->cb) return x->cb < y->cb ? -1 : 1;
  if (x->cd != y->cd) return x->cd < y->cd ? -1 : 1;
  return 0;
}

static int key_cmp4(int32_t ea, int32_t da, uint32_t ba, uint32_t xa, int32_t eb, int32_t db, uint32_t bb,
                    uint32_t xb) {
  if (ea != eb) return ea < eb ? -1 : 1;
  if (da != db) return da < db ? -1 : 1;
  if (ba != bb) return ba < bb ? -1 : 1;
  if (xa != xb) return xa < xb ? -1 : 1;
  return 0;
}

/*
 * Assignment phi*_j (Section 4.3).  A point is *still* when a point of the
 * reference list R has the same (dim, essential, v_b, v_d); duplicates pair
 * up in key order.  A still point inherits R's assignment (a target index or
 * the diagonal).  Every other point is matched against the targets no still
 * point took, group by group (finite dimension 0/1/2, and the essential
 * class, Eq. 1), with assign_group.
 * At j = 0 the reference list is the target diagram itself, each target
 * "assigned" to itself: with a threshold this is the identity (Section 4.3).
 */
static int assign_points(or_solver* s, const opoint_t* R, int64_t nr, int r_is_targets, double prec) {
  int status = 0;
  int64_t np = s->np;
  opoint_t* P = s->P;
  int64_t* ip = (int64_t*)malloc(sizeof(int64_t) * (np + 1));
  int64_t* ir = (int64_t*)malloc(sizeof(int64_t) * (nr + 1));
  for (int64_t i = 0; i < np; ++i) {
    ip[i] = i;
    P[i].tgt = -1;
    P[i].still = 0;
  }
  for (int64_t i = 0; i < nr; ++i) ir[i] = i;
  g_keyP = P;
  qsort(ip, np, sizeof(int64_t), cmp_key_idx);
  g_keyP = R;
  qsort(ir, nr, sizeof(int64_t), cmp_key_idx);
  uint8_t* taken = (uint8_t*)calloc(s->nt + 1, 1);
  int64_t a = 0, b = 0;
  while (a < np && b < nr) {
    const opoint_t* x = &P[ip[a]];
    const opoint_t* y = &R[ir[b]];
    int c = key_cmp4(x->ess, x->dim, x->vb, x->vd, y->ess, y->dim, y->vb, y->vd);
    if (c < 0) ++a;
    else if (c > 0) ++b;
    else {
      P[ip[a]].still = 1;
      int32_t t = r_is_targets ? (int32_t)ir[b] : y->tgt;
      P[ip[a]].tgt = t;
      if (t >= 0) taken[t] = 1;
      ++a;
      ++b;
    }
  }
  /* reduced problems, one per group */
  float* pb = (float*)malloc(sizeof(float) * (np + 1));
  float* pd = (float*)malloc(sizeof(float) * (np + 1));
  int64_t* pidx = (int64_t*)malloc(sizeof(int64_t) * (np + 1));
  float* tb = (float*)malloc(sizeof(float) * (s->nt + 1));
  float* td = (float*)malloc(sizeof(float) * (s->nt + 1));
  int64_t* tidx = (int64_t*)malloc(sizeof(int64_t) * (s->nt + 1));
  int32_t* res = (int32_t*)malloc(sizeof(int32_t) * (np + 1));
  for (int grp = 0; grp < 4; ++grp) {
    int64_t n1 = 0, n2 = 0;
    for (int64_t i = 0; i < np; ++i)
      if (!P[i].still && group_of(P[i].dim, P[i].ess) == grp) {
        pb[n1] = P[i].b;
        pd[n1] = P[i].d;
        pidx[n1++] = i;
      }
    for (int64_t t = 0; t < s->nt; ++t)
      if (!taken[t] && group_of(s->T[t].dim, s->T[t].ess) == grp) {
        tb[n2] = s->T[t].b;
        td[n2] = s->T[t].d;
        tidx[n2++] = t;
      }
    if (grp == 3) {
      /* infinite classes only match infinite classes (Eq. 1), in order */
      for (int64_t i = 0; i < n1 && i < n2; ++i) P[pidx[i]].tgt = (int32_t)tidx[i];
      continue;
    }
    if (assign_group(n1, pb, pd, n2, tb, td, prec, res)) status = -1;
    for (int64_t i = 0; i < n1; ++i) P[pidx[i]].tgt = res[i] >= 0 ? (int32_t)tidx[res[i]] : -1;
  }
  free(pb);
  free(pd);
  free(pidx);
  free(tb);
  free(td);
  free(tidx);
  free(res);
  free(taken);
  free(ip);
  free(ir);
  return status;
}

/* W2^2 of the current assignment (Eq. 2) and the stop counters. */
static void eval_loss(or_solver* s) {
  double L = 0.0;
  uint8_t* taken = (uint8_t*)calloc(s->nt + 1, 1);
  s->n_unc = 0;
  s->n_still = 0;
  s->n_nssp = 0;
  for (int64_t i = 0; i < s->np; ++i) {
    const opoint_t* p = &s->P[i];
    if (p->still) s->n_still++;
    if (p->tgt >= 0) {
      L += cost_pt(p->b, p->d, s->T[p->tgt].b, s->T[p->tgt].d);
      taken[p->tgt] = 1;
      if (!p->still) s->n_nssp++;
    } else {
      L += cost_diag(p->b, p->d);
      if (p->d > p->b) s->n_unc++;  /* strict count; or_solver_done refines it */
    }
  }
  for (int64_t t = 0; t < s->nt; ++t)
    if (!taken[t]) L += cost_diag(s->T[t].b, s->T[t].d);
  free(taken);
  s->loss = L;
}

typedef struct {
  uint32_t v;
  uint32_t key;
  float c;
} contrib_t;

static int cmp_contrib(const void* a, const void* b) {
  const contrib_t* x = (const contrib_t*)a;
  const contrib_t* y = (const contrib_t*)b;
  if (x->v != y->v) return x->v < y->v ? -1 : 1;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return 0;
}

/*
 * Gradient step (Section 4.1): for each point p matched to phi*(p) (a target,
 * or its diagonal projection ((b+d)/2, (b+d)/2)), the birth vertex gets
 * alpha_b * 2 (f(v_b) - phi*_b) and the death vertex alpha_d * 2 (f(v_d) -
 * phi*_d); f <- f - sum of contributions.  fp32, each operation rounded on
 * its own.  Reading: several contributions to one vertex are summed from
 * +0.0 in increasing order of their value (equal values commute), and the
 * essential class contributes at its birth vertex only (it has no death
 * simplex).
 */
static void gradient_step(or_solver* s, float alpha_b, float alpha_d) {
  contrib_t* C = (contrib_t*)malloc(sizeof(contrib_t) * (2 * s->np + 1));
  int64_t nc = 0;
  for (int64_t i = 0; i < s->np; ++i) {
    const opoint_t* p = &s->P[i];
    float tb, td;
    if (p->tgt >= 0) {
      tb = s->T[p->tgt].b;
      td = s->T[p->tgt].d;
    } else {
      float sum = p->b + p->d;
      float m = sum * 0.5f;
      tb = m;
      td = m;
    }
    float db = p->b - tb;
    float gb = 2.0f * db;
    float cb = alpha_b * gb;
    C[nc].v = p->vb;
    C[nc].c = cb;
    C[nc].key = value_key(cb);
    ++nc;
    if (!p->ess) {
      float dd = p->d - td;
      float gd = 2.0f * dd;
      float cd = alpha_d * gd;
      C[nc].v = p->vd;
      C[nc].c = cd;
      C[nc].key = value_key(cd);
      ++nc;
    }
  }
  qsort(C, nc, sizeof(contrib_t), cmp_contrib);
  s->n_updated = 0;
  int64_t i = 0;
  while (i < nc) {
    uint32_t v = C[i].v;
    float acc = 0.0f;
    while (i < nc && C[i].v == v) {
      acc = acc + C[i].c;
      ++i;
    }
    float old = s->f[v];
    float nw = old - acc;
    uint32_t ob, nb;
    memcpy(&ob, &old, 4);
    memcpy(&nb, &nw, 4);
    if (ob != nb) s->n_updated++;
    s->f[v] = nw;
  }
  free(C);
}

static or_solver* solver_alloc(int lx, int ly, int lz, const float* f0, int* status) {
  if (status) *status = 0;
  if (lx < 2 || ly < 2 || lz < 2) {
    if (status) *status = -1;
    return NULL;
  }
  or_solver* s = (or_solver*)calloc(1, sizeof(or_solver));
  s->g.lx = lx;
  s->g.ly = ly;
  s->g.lz = lz;
  s->g.nv = (int64_t)lx * ly * lz;
  s->f = (float*)malloc(sizeof(float) * s->g.nv);
  memcpy(s->f, f0, sizeof(float) * s->g.nv);
  int st = compute_points(&s->g, s->f, &s->P, &s->np);
  if (st) {
    if (status) *status = st;
    free(s->f);
    free(s);
    return NULL;
  }
  return s;
}

static void solver_start(or_solver* s) {
  s->fast_assign = 1;
  s->assign_prec = 0.0;
  qsort(s->T, s->nt, sizeof(otarget_t), cmp_target);
  /* j = 0: the targets play the previous diagram, each assigned to itself */
  opoint_t* R = (opoint_t*)malloc(sizeof(opoint_t) * (s->nt + 1));
  for (int64_t t = 0; t < s->nt; ++t) {
    R[t].dim = s->T[t].dim;
    R[t].ess = s->T[t].ess;
    R[t].vb = s->T[t].vb;
    R[t].vd = s->T[t].vd;
    R[t].cb = s->T[t].src; /* duplicates of one key pair up in source order */
    R[t].cd = 0;
    R[t].b = s->T[t].b;
    R[t].d = s->T[t].d;
    R[t].tgt = (int32_t)t;
    R[t].still = 0;
  }
  assign_points(s, R, s->nt, 1, 0.0); /* the j = 0 problem is solved exactly */
  free(R);
  s->j = 0;
  eval_loss(s);
  s->loss0 = s->loss;
}

/* Target diagram (Section 3): D(f0) minus the non-signal pairs, here the
 * pairs with persistence fl(d - b) >= fl(tau * fl(max f0 - min f0)), plus the
 * essential class. */
or_solver* or_solver_create(int lx, int ly, int lz, const float* f0, float tau, int* status) {
  or_solver* s = solver_alloc(lx, ly, lz, f0, status);
  if (!s) return NULL;
  float lo = f0[0], hi = f0[0];
  for (int64_t v = 1; v < s->g.nv; ++v) {
    if (f0[v] < lo) lo = f0[v];
    if (f0[v] > hi) hi = f0[v];
  }
  float range = hi - lo;
  float theta = tau * range;
  s->T = (otarget_t*)malloc(sizeof(otarget_t) * (s->np + 1));
  s->nt = 0;
  for (int64_t i = 0; i < s->np; ++i) {
    const opoint_t* p = &s->P[i];
    float pers = p->d - p->b;
    if (p->ess || pers >= theta) {
      otarget_t* t = &s->T[s->nt++];
      t->dim = p->dim;
      t->ess = p->ess;
      t->vb = p->vb;
      t->vd = p->vd;
      t->b = p->b;
      t->d = p->d;
      t->src = p->cb;
    }
  }
  solver_start(s);
  return s;
}

or_solver* or_solver_create_targets(int lx, int ly, int lz, const float* f0, int64_t n, const int32_t* dim,
                                    const int32_t* essential, const uint32_t* vb, const uint32_t* vd,
                                    const float* birth, const float* death, int* status) {
  or_solver* s = solver_alloc(lx, ly, lz, f0, status);
  if (!s) return NULL;
  s->T = (otarget_t*)malloc(sizeof(otarget_t) * (n + 2));
  s->nt = 0;
  int has_ess = 0;
  for (int64_t i = 0; i < n; ++i) {
    otarget_t* t = &s->T[s->nt++];
    t->dim = dim[i];
    t->ess = essential[i];
    t->vb = vb[i];
    t->vd = vd[i];
    t->b = birth[i];
    t->d = death[i];
    t->src = (uint64_t)i;
    if (essential[i]) has_ess = 1;
  }
  if (!has_ess)
    for (int64_t i = 0; i < s->np; ++i)
      if (s->P[i].ess) {
        otarget_t* t = &s->T[s->nt++];
        t->dim = s->P[i].dim;
        t->ess = 1;
        t->vb = s->P[i].vb;
        t->vd = s->P[i].vd;
        t->b = s->P[i].b;
        t->d = s->P[i].d;
        t->src = (uint64_t)n;
      }
  solver_start(s);
  return s;
}

/*
 * Stop rule.  Algorithm 1 stops when L(f_j) <= s * L(f_0) or j = j_max.
 * Reading: with stop_s <= 0 the loss test is off; the solver also stops as
 * soon as no diagonal-matched point has persistence fl(d - b) > cancel_eps
 * (every non-signal pair cancelled; cancel_eps = 0 asks for exact zeros).
 */
static int64_t count_uncancelled(const or_solver* s, float cancel_eps) {
  int64_t n = 0;
  for (int64_t i = 0; i < s->np; ++i) {
    const opoint_t* p = &s->P[i];
    if (p->tgt < 0) {
      float pers = p->d - p->b;
      if (pers > cancel_eps) ++n;
    }
  }
  return n;
}

int or_solver_done(or_solver* s, float stop_s, float cancel_eps, int max_iters) {
  s->n_unc = count_uncancelled(s, cancel_eps);
  if (s->n_unc == 0) return 1;
  if (stop_s > 0.0f && s->loss <= (double)stop_s * s->loss0) return 1;
  return s->j >= max_iters ? 1 : 0;
}

int or_solver_iterate(or_solver* s, float alpha_b, float alpha_d, float stop_s, float cancel_eps, int max_iters) {
  gradient_step(s, alpha_b, alpha_d);
  opoint_t* prev = s->P;
  int64_t nprev = s->np;
  int st = compute_points(&s->g, s->f, &s->P, &s->np);
  if (st) {
    s->P = prev;
    s->np = nprev;
    return st;
  }
  /* without the Section 4.3 reuse no point of the previous diagram is
   * consulted: every point is matched by the exact solver */
  int ast = assign_points(s, prev, s->fast_assign ? nprev : 0, 0, s->assign_prec);
  free(prev);
  if (ast) return -4;
  s->j += 1;
  eval_loss(s);
  return or_solver_done(s, stop_s, cancel_eps, max_iters);
}

/*
 * Warm start (not in the paper): the values are replaced by a start field
 * g0 and the solver continues from it with the same target diagram and
 * loss_0.  Reading: g0 takes the place of the next iterate, so its diagram
 * is matched as after a step (Section 4.3): points with the (dim,
 * essential, v_b, v_d) of a point of the current diagram keep that point's
 * assignment, the others go to the exact reduced assignment; the iteration
 * count restarts at 0.
 */
int or_solver_set_start(or_solver* s, const float* values) {
  for (int64_t v = 0; v < s->g.nv; ++v) {
    if (!isfinite(values[v])) return -2;
  }
  memcpy(s->f, values, sizeof(float) * (size_t)s->g.nv);
  opoint_t* prev = s->P;
  int64_t nprev = s->np;
  int st = compute_points(&s->g, s->f, &s->P, &s->np);
  if (st) {
    s->P = prev;
    s->np = nprev;
    return st;
  }
  int ast = assign_points(s, prev, nprev, 0, 0.0);
  free(prev);
  if (ast) return -4;
  s->j = 0;
  eval_loss(s);
  return 0;
}

void or_solver_set_fast_assignment(or_solver* s, int on) { s->fast_assign = on ? 1 : 0; }

void or_solver_set_assignment_precision(or_solver* s, double prec) { s->assign_prec = prec > 0.0 ? prec : 0.0; }

/*
 * Topological loss of the field `values` against the solver's target
 * diagram (Eq. 2, q = 2): the diagram of `values`, every point matched by
 * the exact solver (no still-pair reuse), L, and dL/df in fp64.  Where the
 * pairing and the matching do not change, L is a sum of squares of vertex
 * values, so: a point matched to target t adds 2 (b - t_b) at v_b and
 * 2 (d - t_d) at v_d (the essential class too: its death value is the
 * global maximum's); a point matched to the diagonal adds b - d at v_b and
 * d - b at v_d, the derivative of (d - b)^2 / 2.  Contributions are added
 * in diagram order, birth before death.  The solver's state becomes this
 * field, its diagram and matching.
 */
int or_solver_loss_grad(or_solver* s, const float* values, double* loss, double* grad) {
  memcpy(s->f, values, sizeof(float) * s->g.nv);
  opoint_t* prev = s->P;
  int64_t nprev = s->np;
  int st = compute_points(&s->g, s->f, &s->P, &s->np);
  if (st) {
    s->P = prev;
    s->np = nprev;
    return st;
  }
  free(prev);
  assign_points(s, NULL, 0, 0, 0.0);
  eval_loss(s);
  *loss = s->loss;
  memset(grad, 0, sizeof(double) * s->g.nv);
  for (int64_t i = 0; i < s->np; ++i) {
    const opoint_t* p = &s->P[i];
    double b = (double)p->b, d = (double)p->d, gb, gd;
    if (p->tgt >= 0) {
      gb = 2.0 * (b - (double)s->T[p->tgt].b);
      gd = 2.0 * (d - (double)s->T[p->tgt].d);
    } else {
      gb = b - d;
      gd = d - b;
    }
    grad[p->vb] += gb;
    grad[p->vd] += gd;
  }
  return 0;
}

void or_solver_field(const or_solver* s, float* out) { memcpy(out, s->f, sizeof(float) * s->g.nv); }
int64_t or_solver_num_points(const or_solver* s) { return s->np; }
int64_t or_solver_num_targets(const or_solver* s) { return s->nt; }

void or_solver_points(const or_solver* s, int32_t* dim, int32_t* essential, uint32_t* vb, uint32_t* vd,
                      float* birth, float* death, int32_t* tgt, int32_t* still, uint64_t* cb, uint64_t* cd) {
  for (int64_t i = 0; i < s->np; ++i) {
    dim[i] = s->P[i].dim;
    essential[i] = s->P[i].ess;
    vb[i] = s->P[i].vb;
    vd[i] = s->P[i].vd;
    birth[i] = s->P[i].b;
    death[i] = s->P[i].d;
    tgt[i] = s->P[i].tgt;
    still[i] = s->P[i].still;
    cb[i] = s->P[i].cb;
    cd[i] = s->P[i].cd;
  }
}

void or_solver_targets(const or_solver* s, int32_t* dim, int32_t* essential, uint32_t* vb, uint32_t* vd,
                       float* birth, float* death) {
  for (int64_t t = 0; t < s->nt; ++t) {
    dim[t] = s->T[t].dim;
    essential[t] = s->T[t].ess;
    vb[t] = s->T[t].vb;
    vd[t] = s->T[t].vd;
    birth[t] = s->T[t].b;
    death[t] = s->T[t].d;
  }
}

void or_solver_stats(const or_solver* s, int64_t* stats, double* loss) {
  stats[0] = s->j;
  stats[1] = s->n_unc;
  stats[2] = s->n_still;
  stats[3] = s->n_updated;
  stats[4] = s->n_nssp;
  loss[0] = s->loss;
  loss[1] = s->loss0;
}

void or_solver_free(or_solver* s) {
  if (!s) return;
  free(s->f);
  free(s->T);
  free(s->P);
  free(s);
}
