/*
 * vls_oracle.c -- plain FP64 CPU oracle of the variational loop-shrinking hot path.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the benchmark).
 * Shares no code with the CUDA library.  Built with -ffp-contract=off so every
 * product and sum is rounded on its own, in the order written here.
 *
 * What it computes (Weinrauch et al., "A Variational Loop Shrinking Analogy ..."):
 *   - Sec. 2, Eq. (2) with g' = sqrt(phi_i phi_j): multi-layer phase field on the mesh,
 *     explicit Euler with a constant step, column normalisation after every step,
 *     base layer implicit (1 - sum of stored layers), e_ij / mu_ij non-zero only
 *     against the base (Sec. 2, "Implementation details");
 *   - Sec. 3.1: splits (a layer whose narrow band has several components moves each
 *     component to a new layer), merges (layers meeting at a vertex are summed into
 *     one new layer; the involved fronts minus one are handle loops);
 *   - Sec. 3.2: one tunnel pass per handle -- single-layer diffusion (Sec. 4) from the
 *     inside of the handle loop with the loop as a border, restricted to the area
 *     covered when the handle was found, then a trace back from the first point
 *     reached on the far side;
 *   - Sec. 5: Reeb graph from the events (nodes: seed, split, merge, end; arcs: layers),
 *     node position = mean of the narrow band.
 *
 * Readings where the paper is silent (each restated in the design notes):
 *   - Eq. (2) is used as printed (a_ik^2 terms); a_ii = w_ii = 0, a = 1/25, w = a/5,
 *     mu = 1/4, e = 1/30.  e_ij is antisymmetric, +e for (layer, base), so that the rates
 *     at a vertex sum to zero and the front grows into the base.  n is the number of
 *     layers present in the vertex's closed neighbourhood (including the base).
 *   - Operator: uniform scaled Laplacian L_vu = s/d_v (u ~ v), L_vv = -s, s = 4/lbar^2,
 *     lbar = eta/4, eta = pi a / sqrt(2 w) (band width of the travelling wave of Eq. (2)).
 *   - dt = c lbar^2 / (4 D), D = mu a^2 / 2, c = 0.5.
 *   - After each Euler step: clamp to [0,1], snap (< eps0 -> 0, > 1 - eps0 -> 1), divide by
 *     the column sum.  Band of layer l: 0 < phi_l < 1.
 *   - Only vertices whose closed neighbourhood holds the base and at least one other layer
 *     change (all rates vanish otherwise); restricting the update to them is exact.
 *   - Seed region: the closed 1-ring of the seed vertex (a single vertex is below the
 *     critical nucleus of Eq. (2) and dies out).
 *   - Split/merge bookkeeping is vertex-major (one row per vertex: (layer, value)
 *     entries).  On a split only band entries move to the children; phi = 1 entries keep
 *     the parent id, the parent becomes DEAD and those vertices are frozen.  A DEAD entry
 *     read from a vertex whose only layer is l counts as value 1 of l.
 *   - Per step: update (Jacobi) -> merges -> splits/extinctions -> cover step -> stop test.
 *   - Handle loop of a layer: theta-isoline of its field (crossing edge (a,b): psi(a) >=
 *     theta > psi(b), one endpoint holding the layer), the component with the most
 *     crossing edges; the loop dropped in a merge is the one with the most crossing edges
 *     (Sec. 3.1 says the choice does not matter).
 *   - Tunnel pass: domain = vertices covered by the step of the handle (the whole surface when
 *     the handle loop separates that area); the loop's crossing edges are cut; inside
 *     endpoints held at 1; arrival step T(v) = first step with phi >= theta; trace from
 *     the smallest-id outside endpoint reached first, depth first over unvisited reached
 *     neighbours in the order (T larger than here, T, id), stepping back along the path
 *     from dead ends, down to a source; close along the loop.
 *
 * Parity unpinned: the FP64 coordinates of handle-loop points (isoline interpolation) and of
 * Reeb-graph nodes (band means).  The paper prints no worked example and its meshes are not
 * available; the pins cover the loops' crossing edges, vertex cycles and homology classes and
 * the Reeb graph's topology, not these coordinates.
 */
#include "vls_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define KM 8 /* entry capacity per vertex row (transient co-presence included) */

enum { ST_OK = 0, ST_EINVAL = 1, ST_ENOTMANIFOLD = 2, ST_ENONORIENTABLE = 3, ST_EDISCONNECTED = 4,
       ST_EMAXSTEPS = 5, ST_ESLOTS = 6, ST_ELAYERS = 7, ST_ELOOPFAIL = 8, ST_ENOMEM = 10, ST_ESTALL = 12 };
enum { L_UNUSED = 0, L_ALIVE = 1, L_DEAD = 2, L_MERGED = 3, L_ENDED = 4 };
enum { N_SEED = 0, N_SPLIT = 1, N_MERGE = 2, N_END = 3 };

typedef struct {
  int32_t info[5];
  int32_t *edges;
  int32_t *verts;
  double *pts;
  double len;
  int32_t tinfo[4];
  int32_t *tverts;
  int32_t *arrival;
  int32_t rinfo[4];   /* refined handle (Sec. 3.3): status, stop step, first vertex reached, n verts */
  int32_t *rverts;
  double dlen[3];     /* length change under the normal offset (Sec. 3.5): handle, tunnel, refined */
  /* PL streamlines (Sec. 3.2) of the tunnel pass [0] and the refinement pass [1]: status (-1 not run),
     points of the closed polyline, its length */
  int32_t sst[2];
  int64_t sn[2];
  double *spts[2];
  double slen[2];
  double *tfa;        /* fractional arrival times of the tunnel pass, kept when record_steps is set */
} handle_t;

struct orc_run {
  int32_t status, genus, steps;
  int64_t cnt[8];
  int64_t nv, nf, nnz;
  orc_options opt;
  double eta, lbar, dt, s, ah, one_m_eps;
  /* mesh */
  double *X;
  int32_t *F;
  int64_t *rp;
  int32_t *col, *hface;
  double *Lv, *Ld;
  /* state (vertex-major rows of (layer, value) entries, ascending layer id) */
  int32_t *en, *el;
  double *ex;
  int32_t *cover;
  /* layers */
  int32_t nl, capl;
  int32_t *lst, *lbirth, *ldeath;
  /* Reeb nodes */
  int32_t nn, capn;
  int32_t *nodes;
  double *npos;
  /* handles */
  int32_t nh, caph;
  handle_t *h;
  /* outputs */
  int32_t *out_layer;
  double *out_phi;
  int64_t *rec;
  int32_t nrec, caprec;
  int32_t *layers_out;
  /* scratch */
  int32_t *stamp;
  int32_t stamp_id;
  /* loop classification (Sec. 3.5): unit vertex normals, mean edge length */
  double *vn;
  double mean_edge;
};

/* ------------------------------------------------------------------ utils */
void orc_default_options(orc_options *o) {
  memset(o, 0, sizeof(*o));
  o->mu = 0.25;
  o->e = 1.0 / 30.0;
  o->a = 1.0 / 25.0;
  o->w = o->a / 5.0;
  o->dt_factor = 0.5;
  o->eps0 = 1e-3;
  o->theta_iso = 0.5;
  o->lbar = 0.0;
  o->max_steps = 200000;
  o->max_pass_steps = 200000;
  o->seed_ring = 1;
  o->naive = 0;
  o->tunnels = 1;
  o->record_steps = 0;
  o->refine = 1;
  o->offset = 0.5;
  o->max_passes = 0;
  o->streamlines = 1;
}

void orc_constants(const orc_options *o, double out[4]) {
  const double pi = 3.14159265358979323846;
  double eta = pi * o->a / sqrt(2.0 * o->w);
  double lbar = o->lbar > 0 ? o->lbar : eta / 4.0;
  double D = o->mu * o->a * o->a / 2.0;
  double dt = o->dt_factor * lbar * lbar / (4.0 * D);
  out[0] = eta;
  out[1] = lbar;
  out[2] = dt;
  out[3] = 4.0 / (lbar * lbar);
}

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}
typedef struct { int32_t a, b; int32_t f; } hedge_t;
static int cmp_hedge(const void *p, const void *q) {
  const hedge_t *x = (const hedge_t *)p, *y = (const hedge_t *)q;
  if (x->a != y->a) return (x->a > y->a) - (x->a < y->a);
  return (x->b > y->b) - (x->b < y->b);
}

/* slot of half-edge u->w in the CSR, -1 if absent */
static int64_t slot_of(const orc_run *R, int32_t u, int32_t w) {
  int64_t lo = R->rp[u], hi = R->rp[u + 1] - 1;
  while (lo <= hi) {
    int64_t m = (lo + hi) / 2;
    if (R->col[m] == w) return m;
    if (R->col[m] < w) lo = m + 1;
    else hi = m - 1;
  }
  return -1;
}

/* ----------------------------------------------------- mesh + operator */
static int build_mesh(orc_run *R, const double *X, const int32_t *F) {
  int64_t nv = R->nv, nf = R->nf;
  if (nv < 4 || nf < 4) return ST_EINVAL;
  for (int64_t i = 0; i < 3 * nf; ++i)
    if (F[i] < 0 || F[i] >= nv) return ST_EINVAL;
  for (int64_t f = 0; f < nf; ++f)
    if (F[3 * f] == F[3 * f + 1] || F[3 * f + 1] == F[3 * f + 2] || F[3 * f] == F[3 * f + 2]) return ST_EINVAL;
  R->X = (double *)malloc(sizeof(double) * 3 * nv);
  R->F = (int32_t *)malloc(sizeof(int32_t) * 3 * nf);
  memcpy(R->X, X, sizeof(double) * 3 * nv);
  memcpy(R->F, F, sizeof(int32_t) * 3 * nf);
  int64_t nh = 3 * nf;
  hedge_t *he = (hedge_t *)malloc(sizeof(hedge_t) * nh);
  for (int64_t f = 0; f < nf; ++f)
    for (int k = 0; k < 3; ++k) {
      he[3 * f + k].a = F[3 * f + k];
      he[3 * f + k].b = F[3 * f + (k + 1) % 3];
      he[3 * f + k].f = (int32_t)f;
    }
  qsort(he, nh, sizeof(hedge_t), cmp_hedge);
  int st = ST_OK;
  for (int64_t i = 1; i < nh && st == ST_OK; ++i)
    if (he[i].a == he[i - 1].a && he[i].b == he[i - 1].b) st = ST_ENONORIENTABLE;
  R->rp = (int64_t *)calloc(nv + 1, sizeof(int64_t));
  R->col = (int32_t *)malloc(sizeof(int32_t) * nh);
  R->hface = (int32_t *)malloc(sizeof(int32_t) * nh);
  for (int64_t i = 0; i < nh; ++i) {
    R->rp[he[i].a + 1]++;
    R->col[i] = he[i].b;
    R->hface[i] = he[i].f;
  }
  free(he);
  for (int64_t v = 0; v < nv; ++v) R->rp[v + 1] += R->rp[v];
  R->nnz = nh;
  if (st != ST_OK) return st;
  /* every half-edge needs its twin (closed, edge-manifold) */
  for (int64_t v = 0; v < nv; ++v)
    for (int64_t k = R->rp[v]; k < R->rp[v + 1]; ++k)
      if (slot_of(R, R->col[k], (int32_t)v) < 0) return ST_ENOTMANIFOLD;
  /* every vertex used; its fan is a single cycle (vertex-manifold) */
  for (int64_t v = 0; v < nv; ++v) {
    int64_t d = R->rp[v + 1] - R->rp[v];
    if (d == 0) return ST_EDISCONNECTED;
    int32_t start = R->col[R->rp[v]], cur = start;
    int64_t steps = 0;
    do {
      int64_t k = slot_of(R, (int32_t)v, cur);
      const int32_t *t = R->F + 3 * R->hface[k];
      int32_t nxt = -1;
      for (int q = 0; q < 3; ++q)
        if (t[q] != v && t[q] != cur) nxt = t[q];
      cur = nxt;
      ++steps;
    } while (cur != start && steps <= d);
    if (steps != d) return ST_ENOTMANIFOLD;
  }
  /* connectivity */
  int32_t *q = (int32_t *)malloc(sizeof(int32_t) * nv);
  char *seen = (char *)calloc(nv, 1);
  int64_t qh = 0, qt = 0;
  q[qt++] = 0; seen[0] = 1;
  while (qh < qt) {
    int32_t v = q[qh++];
    for (int64_t k = R->rp[v]; k < R->rp[v + 1]; ++k)
      if (!seen[R->col[k]]) { seen[R->col[k]] = 1; q[qt++] = R->col[k]; }
  }
  free(q); free(seen);
  if (qt != nv) return ST_EDISCONNECTED;
  int64_t E = nh / 2;
  int64_t chi = nv - E + nf;
  R->genus = (int32_t)((2 - chi) / 2);
  /* operator (uniform scaled Laplacian) */
  R->Lv = (double *)malloc(sizeof(double) * nh);
  R->Ld = (double *)malloc(sizeof(double) * nv);
  for (int64_t v = 0; v < nv; ++v) {
    int64_t d = R->rp[v + 1] - R->rp[v];
    double off = R->s / (double)d;
    for (int64_t k = R->rp[v]; k < R->rp[v + 1]; ++k) R->Lv[k] = off;
    R->Ld[v] = -R->s;
  }
  return ST_OK;
}

/* ------------------------------------------------------------- state */
static int is_frozen(const orc_run *R, int64_t v) {
  for (int k = 0; k < R->en[v]; ++k) {
    int32_t s = R->lst[R->el[v * KM + k]];
    if (s == L_DEAD || s == L_ENDED) return 1;
  }
  return 0;
}
static double entry_val(const orc_run *R, int64_t u, int32_t l) {
  for (int k = 0; k < R->en[u]; ++k)
    if (R->el[u * KM + k] == l) return R->ex[u * KM + k];
  return 0.0;
}
static int holds(const orc_run *R, int64_t u, int32_t l) {
  for (int k = 0; k < R->en[u]; ++k)
    if (R->el[u * KM + k] == l) return 1;
  return 0;
}
static double base_val(const orc_run *R, int64_t u) {
  double s = 0.0;
  for (int k = 0; k < R->en[u]; ++k) s = s + R->ex[u * KM + k];
  return 1.0 - s;
}
/* the single alive layer held by v, or 0 */
static int32_t own_layer(const orc_run *R, int64_t v) {
  if (R->en[v] == 1 && R->lst[R->el[v * KM]] == L_ALIVE) return R->el[v * KM];
  return 0;
}
/* value of layer l at u as read from a vertex whose own layer is o */
static double psi_read(const orc_run *R, int64_t u, int32_t l, int32_t o) {
  if (is_frozen(R, u)) return (o != 0 && l == o) ? 1.0 : 0.0;
  return entry_val(R, u, l);
}

static int32_t new_layer(orc_run *R, int32_t birth) {
  if (R->nl + 1 >= R->capl) {
    R->capl = R->capl * 2 + 16;
    R->lst = (int32_t *)realloc(R->lst, sizeof(int32_t) * R->capl);
    R->lbirth = (int32_t *)realloc(R->lbirth, sizeof(int32_t) * R->capl);
    R->ldeath = (int32_t *)realloc(R->ldeath, sizeof(int32_t) * R->capl);
  }
  int32_t id = ++R->nl;
  R->lst[id] = L_ALIVE;
  R->lbirth[id] = birth;
  R->ldeath[id] = -1;
  R->cnt[6]++;
  return id;
}
static int32_t add_node(orc_run *R, int32_t kind, int32_t step, const double *pos) {
  if (R->nn == R->capn) {
    R->capn = R->capn * 2 + 16;
    R->nodes = (int32_t *)realloc(R->nodes, sizeof(int32_t) * 2 * R->capn);
    R->npos = (double *)realloc(R->npos, sizeof(double) * 3 * R->capn);
  }
  R->nodes[2 * R->nn] = kind;
  R->nodes[2 * R->nn + 1] = step;
  for (int d = 0; d < 3; ++d) R->npos[3 * R->nn + d] = pos[d];
  return R->nn++;
}

/* Entry row writes: set row v to the given (ascending) layers/values, dropping zeros. */
static int set_row(orc_run *R, int64_t v, int n, const int32_t *ls, const double *xs) {
  int m = 0;
  for (int i = 0; i < n; ++i)
    if (xs[i] > 0.0) {
      if (m == KM) return ST_ESLOTS;
      R->el[v * KM + m] = ls[i];
      R->ex[v * KM + m] = xs[i];
      ++m;
    }
  R->en[v] = m;
  return ST_OK;
}

/* ----------------------------------------------- Eq. (2) at one vertex */
/*
 * Layers 0..nl-1 (non-base, ascending id) with own values x[] and Laplacians lap[],
 * base value xb and Laplacian lapb; the base is present.  n = nl + 1 phases meet here.
 * rate_l = (mu/n) [ w (x_l - x_b) + (a^2/2)(lap_l - lap_b) + e sqrt(x_l x_b) ]  (Eq. 2 with
 * mu_ij, e_ij non-zero only against the base), rate_b = -sum_l rate_l; explicit Euler;
 * clamp to [0,1]; snap at eps0 / 1-eps0; divide by the column sum.
 * Returns 0 on success, -1 if the column sum vanished (values left unchanged).
 */
static int vertex_update(const orc_run *R, int nl, const double *x, const double *lap, double xb, double lapb,
                         double *out) {
  const orc_options *o = &R->opt;
  int n = nl + 1;
  double mun = o->mu / (double)n;
  double y[KM + 1];
  double sr = 0.0;
  for (int i = 0; i < nl; ++i) {
    double r = mun * ((o->w * (x[i] - xb) + R->ah * (lap[i] - lapb)) + o->e * sqrt(x[i] * xb));
    sr = sr + r;
    y[i] = x[i] + R->dt * r;
  }
  double yb = xb + R->dt * (-sr);
  for (int i = 0; i <= nl; ++i) {
    double *p = (i < nl) ? &y[i] : &yb;
    if (*p < 0.0) *p = 0.0;
    if (*p > 1.0) *p = 1.0;
    if (*p < o->eps0) *p = 0.0;
    if (*p > R->one_m_eps) *p = 1.0;
  }
  double S = yb;
  for (int i = 0; i < nl; ++i) S = S + y[i];
  if (S == 0.0) return -1;
  for (int i = 0; i < nl; ++i) out[i] = y[i] / S;
  return 0;
}

/* layers present in the closed neighbourhood of v (alive, ascending) and whether the base is */
static int gather_layers(orc_run *R, int64_t v, int32_t *ls, int *has_base) {
  int n = 0;
  *has_base = 0;
  for (int64_t k = R->rp[v] - 1; k < R->rp[v + 1]; ++k) {
    int64_t u = (k < R->rp[v]) ? v : R->col[k];
    if (is_frozen(R, u)) continue; /* reads as the vertex's own layer (already present) */
    for (int q = 0; q < R->en[u]; ++q) {
      int32_t l = R->el[u * KM + q];
      if (R->lst[l] != L_ALIVE) continue;
      int dup = 0;
      for (int i = 0; i < n; ++i)
        if (ls[i] == l) dup = 1;
      if (!dup) {
        if (n == KM) return -1;
        ls[n++] = l;
      }
    }
    if (base_val(R, u) > 0.0) *has_base = 1;
  }
  qsort(ls, n, sizeof(int32_t), cmp_i32);
  return n;
}

static int in_frontier(orc_run *R, int64_t v) {
  if (is_frozen(R, v)) return 0;
  int32_t ls[KM];
  int hb;
  int n = gather_layers(R, v, ls, &hb);
  if (n < 0) return 1; /* overflow surfaces as ESLOTS in the update */
  return hb && n >= 1;
}

/* new row of v (not applied): returns count of layers, fills ls/xs; -1 on slot overflow */
static int compute_update(orc_run *R, int64_t v, int32_t *ls, double *xs) {
  int hb;
  int n = gather_layers(R, v, ls, &hb);
  if (n < 0) return -1;
  int32_t o = own_layer(R, v);
  if (o == 0) /* a plateau next to a vertex without a single own layer is an anomaly */
    for (int64_t k = R->rp[v]; k < R->rp[v + 1]; ++k)
      if (is_frozen(R, R->col[k])) { R->cnt[1]++; break; }
  double x[KM], lap[KM];
  for (int i = 0; i < n; ++i) {
    int32_t l = ls[i];
    double acc = 0.0;
    for (int64_t k = R->rp[v]; k < R->rp[v + 1]; ++k) acc = acc + R->Lv[k] * psi_read(R, R->col[k], l, o);
    acc = acc + R->Ld[v] * entry_val(R, v, l);
    lap[i] = acc;
    x[i] = entry_val(R, v, l);
  }
  double xb = base_val(R, v);
  double accb = 0.0;
  for (int64_t k = R->rp[v]; k < R->rp[v + 1]; ++k) accb = accb + R->Lv[k] * base_val(R, R->col[k]);
  accb = accb + R->Ld[v] * xb;
  if (vertex_update(R, n, x, lap, xb, accb, xs) != 0) {
    R->cnt[1]++;
    for (int i = 0; i < n; ++i) xs[i] = x[i];
  }
  return n;
}

/* ------------------------------------------------------- isoline trace */
typedef struct { int32_t a, b; int64_t k; } xedge_t;

static double psi_iso(const orc_run *R, int64_t u, int32_t l) {
  if (is_frozen(R, u)) return 1.0;
  return entry_val(R, u, l);
}
static int64_t find_xedge(const xedge_t *E, int64_t n, int32_t a, int32_t b) {
  int64_t lo = 0, hi = n - 1;
  while (lo <= hi) {
    int64_t m = (lo + hi) / 2;
    if (E[m].a == a && E[m].b == b) return m;
    if (E[m].a < a || (E[m].a == a && E[m].b < b)) lo = m + 1;
    else hi = m - 1;
  }
  return -1;
}
static int64_t uf_find(int64_t *p, int64_t x) {
  while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
  return x;
}

/* The theta-isoline of layer l: its largest component as an ordered crossing-edge cycle. */
static int64_t trace_isoline(orc_run *R, int32_t l, xedge_t **out) {
  double th = R->opt.theta_iso;
  int64_t cap = 1024, n = 0;
  xedge_t *E = (xedge_t *)malloc(sizeof(xedge_t) * cap);
  for (int64_t a = 0; a < R->nv; ++a) {
    double pa = psi_iso(R, a, l);
    if (!(pa >= th)) continue;
    int ha = holds(R, a, l);
    for (int64_t k = R->rp[a]; k < R->rp[a + 1]; ++k) {
      int32_t b = R->col[k];
      double pb = psi_iso(R, b, l);
      if (pb >= th) continue;
      if (!(ha || holds(R, b, l))) continue;
      if (n == cap) { cap *= 2; E = (xedge_t *)realloc(E, sizeof(xedge_t) * cap); }
      E[n].a = (int32_t)a; E[n].b = b; E[n].k = k; ++n;
    }
  }
  if (n == 0) { free(E); *out = NULL; return 0; }
  int64_t *succ = (int64_t *)malloc(sizeof(int64_t) * n);
  int64_t *pred = (int64_t *)malloc(sizeof(int64_t) * n);
  int64_t *par = (int64_t *)malloc(sizeof(int64_t) * n);
  for (int64_t i = 0; i < n; ++i) { pred[i] = -1; par[i] = i; }
  for (int64_t i = 0; i < n; ++i) {
    const int32_t *t = R->F + 3 * R->hface[E[i].k];
    int32_t c = -1;
    for (int q = 0; q < 3; ++q)
      if (t[q] != E[i].a && t[q] != E[i].b) c = t[q];
    int64_t j;
    if (psi_iso(R, c, l) >= th) j = find_xedge(E, n, c, E[i].b);
    else j = find_xedge(E, n, E[i].a, c);
    succ[i] = j;
    if (j >= 0) {
      pred[j] = i;
      int64_t ra = uf_find(par, i), rb = uf_find(par, j);
      if (ra != rb) par[ra > rb ? ra : rb] = ra < rb ? ra : rb;
    }
  }
  /* component sizes; root = smallest edge index = smallest key */
  int64_t *size = (int64_t *)calloc(n, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) size[uf_find(par, i)]++;
  int64_t best = -1;
  for (int64_t i = 0; i < n; ++i)
    if (par[i] == i && (best < 0 || size[i] > size[best])) best = i;
  /* walk from the smallest edge of the chosen component */
  xedge_t *W = (xedge_t *)malloc(sizeof(xedge_t) * size[best]);
  int64_t m = 0, cur = best;
  int closed = 0;
  while (m < size[best]) {
    W[m++] = E[cur];
    cur = succ[cur];
    if (cur == best) { closed = 1; break; }
    if (cur < 0) break;
  }
  if (!closed) {
    /* open chain (a crossing edge failed the holding rule): prepend the part behind the start */
    R->cnt[1]++;
    int64_t back = pred[best], nb = 0;
    xedge_t *B = (xedge_t *)malloc(sizeof(xedge_t) * size[best]);
    while (back >= 0 && nb + m < size[best]) { B[nb++] = E[back]; back = pred[back]; }
    xedge_t *W2 = (xedge_t *)malloc(sizeof(xedge_t) * (nb + m));
    for (int64_t i = 0; i < nb; ++i) W2[i] = B[nb - 1 - i];
    for (int64_t i = 0; i < m; ++i) W2[nb + i] = W[i];
    free(W); free(B);
    W = W2;
    m += nb;
  }
  free(E); free(succ); free(pred); free(par); free(size);
  *out = W;
  return m;
}

static void emit_handle(orc_run *R, int32_t step, int32_t l, int32_t node, const xedge_t *W, int64_t m) {
  if (R->nh == R->caph) {
    R->caph = R->caph * 2 + 8;
    R->h = (handle_t *)realloc(R->h, sizeof(handle_t) * R->caph);
  }
  handle_t *H = &R->h[R->nh++];
  memset(H, 0, sizeof(*H));
  double th = R->opt.theta_iso;
  H->edges = (int32_t *)malloc(sizeof(int32_t) * 2 * (m > 0 ? m : 1));
  H->verts = (int32_t *)malloc(sizeof(int32_t) * (m > 0 ? m : 1));
  H->pts = (double *)malloc(sizeof(double) * 3 * (m > 0 ? m : 1));
  int64_t nvs = 0;
  for (int64_t i = 0; i < m; ++i) {
    int32_t a = W[i].a, b = W[i].b;
    H->edges[2 * i] = a;
    H->edges[2 * i + 1] = b;
    double pa = psi_iso(R, a, l), pb = psi_iso(R, b, l);
    double t = (pa - th) / (pa - pb);
    for (int d = 0; d < 3; ++d) H->pts[3 * i + d] = R->X[3 * a + d] + t * (R->X[3 * b + d] - R->X[3 * a + d]);
    if (nvs == 0 || H->verts[nvs - 1] != a) H->verts[nvs++] = a;
  }
  while (nvs > 1 && H->verts[nvs - 1] == H->verts[0]) --nvs;
  double len = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    const double *p = H->pts + 3 * i, *q = H->pts + 3 * ((i + 1) % m);
    len = len + sqrt((q[0] - p[0]) * (q[0] - p[0]) + (q[1] - p[1]) * (q[1] - p[1]) + (q[2] - p[2]) * (q[2] - p[2]));
  }
  H->len = len;
  H->info[0] = step;
  H->info[1] = l;
  H->info[2] = node;
  H->info[3] = (int32_t)m;
  H->info[4] = (int32_t)nvs;
  H->tinfo[0] = -1;
  H->sst[0] = H->sst[1] = -1;
}

/* mean position of the vertices v in list (or all vertices when list == NULL) with pred */
static void mean_pos(const orc_run *R, const int64_t *vs, int64_t nvs, double *pos) {
  double s[3] = {0.0, 0.0, 0.0};
  for (int64_t i = 0; i < nvs; ++i)
    for (int d = 0; d < 3; ++d) s[d] = s[d] + R->X[3 * vs[i] + d];
  for (int d = 0; d < 3; ++d) pos[d] = nvs ? s[d] / (double)nvs : 0.0;
}

/* ------------------------------------------------------------- merges */
static int do_merges(orc_run *R, int32_t t, const int64_t *Fl, int64_t nF) {
  int64_t L = R->nl + 1;
  int64_t *par = (int64_t *)malloc(sizeof(int64_t) * L);
  for (int64_t i = 0; i < L; ++i) par[i] = i;
  int any = 0;
  for (int64_t i = 0; i < nF; ++i) {
    int64_t v = Fl[i];
    if (R->en[v] < 2) continue;
    any = 1;
    for (int q = 1; q < R->en[v]; ++q) {
      int64_t ra = uf_find(par, R->el[v * KM]), rb = uf_find(par, R->el[v * KM + q]);
      if (ra != rb) par[ra > rb ? ra : rb] = ra < rb ? ra : rb;
    }
  }
  if (!any) { free(par); return ST_OK; }
  /* groups in order of their smallest member (= root) */
  for (int64_t r = 1; r < L; ++r) {
    if (uf_find(par, r) != r) continue;
    int32_t mem[256];
    int nm = 0;
    for (int64_t l = r; l < L; ++l)
      if (uf_find(par, l) == r) {
        if (nm == 256) { free(par); return ST_ELAYERS; }
        mem[nm++] = (int32_t)l;
      }
    if (nm < 2) continue;
    R->cnt[3]++;
    /* handle-loop candidates on the pre-merge state */
    xedge_t *W[256];
    int64_t Wn[256];
    int drop = 0;
    for (int i = 0; i < nm; ++i) {
      Wn[i] = trace_isoline(R, mem[i], &W[i]);
      if (Wn[i] >= Wn[drop]) drop = i; /* most crossing edges; tie -> larger id */
    }
    /* node position: mean of the involved narrow bands */
    int64_t *bv = (int64_t *)malloc(sizeof(int64_t) * R->nv);
    int64_t nb = 0;
    for (int64_t v = 0; v < R->nv; ++v) {
      int inb = 0;
      for (int q = 0; q < R->en[v]; ++q)
        for (int i = 0; i < nm; ++i)
          if (R->el[v * KM + q] == mem[i] && R->ex[v * KM + q] > 0.0 && R->ex[v * KM + q] < 1.0) inb = 1;
      if (inb) bv[nb++] = v;
    }
    double pos[3];
    mean_pos(R, bv, nb, pos);
    free(bv);
    int32_t node = add_node(R, N_MERGE, t, pos);
    for (int i = 0; i < nm; ++i) {
      if (i != drop) {
        if (Wn[i] == 0) R->cnt[1]++;
        emit_handle(R, t, mem[i], node, W[i], Wn[i]);
      }
      free(W[i]);
    }
    int32_t N = new_layer(R, node);
    for (int i = 0; i < nm; ++i) {
      R->lst[mem[i]] = L_MERGED;
      R->ldeath[mem[i]] = node;
    }
    /* literal relabel: sum the members' values (ascending layer order) into layer N */
    for (int64_t v = 0; v < R->nv; ++v) {
      int32_t ls[KM];
      double xs[KM];
      int nk = 0, hit = 0;
      double acc = 0.0;
      for (int q = 0; q < R->en[v]; ++q) {
        int32_t l = R->el[v * KM + q];
        int member = 0;
        for (int i = 0; i < nm; ++i)
          if (mem[i] == l) member = 1;
        if (member) { acc = acc + R->ex[v * KM + q]; hit = 1; }
        else { ls[nk] = l; xs[nk] = R->ex[v * KM + q]; ++nk; }
      }
      if (!hit) continue;
      ls[nk] = N; xs[nk] = acc; ++nk; /* N is the largest id: stays ascending */
      int st = set_row(R, v, nk, ls, xs);
      if (st) { free(par); return st; }
    }
  }
  free(par);
  return ST_OK;
}

/* ---------------------------------------------- splits and extinctions */
static int do_splits(orc_run *R, int32_t t, const int64_t *Fl, int64_t nF, const int64_t *Ft, int64_t nFt) {
  /* snapshot of the alive layers */
  int32_t na = 0;
  int32_t *alive = (int32_t *)malloc(sizeof(int32_t) * (R->nl + 1));
  for (int32_t l = 1; l <= R->nl; ++l)
    if (R->lst[l] == L_ALIVE) alive[na++] = l;
  int64_t *bandv = (int64_t *)malloc(sizeof(int64_t) * (nF + 1));
  int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (nF + 1));
  int64_t *compstart = (int64_t *)malloc(sizeof(int64_t) * (nF + 2));
  int32_t *mark = R->stamp;
  for (int32_t ai = 0; ai < na; ++ai) {
    int32_t l = alive[ai];
    int64_t nb = 0;
    for (int64_t i = 0; i < nF; ++i) {
      int64_t v = Fl[i];
      for (int q = 0; q < R->en[v]; ++q)
        if (R->el[v * KM + q] == l && R->ex[v * KM + q] > 0.0 && R->ex[v * KM + q] < 1.0) bandv[nb++] = v;
    }
    /* BFS components over band vertices of l, in ascending order of their smallest vertex */
    int32_t sid = ++R->stamp_id;
    int64_t qn = 0, nc = 0;
    for (int64_t i = 0; i < nb; ++i) {
      if (mark[bandv[i]] == sid) continue;
      compstart[nc++] = qn;
      int64_t qh = qn;
      queue[qn++] = bandv[i];
      mark[bandv[i]] = sid;
      while (qh < qn) {
        int64_t v = queue[qh++];
        for (int64_t k = R->rp[v]; k < R->rp[v + 1]; ++k) {
          int64_t u = R->col[k];
          if (mark[u] == sid) continue;
          int inb = 0;
          for (int q = 0; q < R->en[u]; ++q)
            if (R->el[u * KM + q] == l && R->ex[u * KM + q] > 0.0 && R->ex[u * KM + q] < 1.0) inb = 1;
          if (inb) { mark[u] = sid; queue[qn++] = u; }
        }
      }
    }
    compstart[nc] = qn;
    if (nc == 1) continue;
    if (nc == 0) {
      /* extinction: node at the mean of this step's updated vertices holding l */
      int64_t *vs = (int64_t *)malloc(sizeof(int64_t) * (nFt + 1));
      int64_t m = 0;
      for (int64_t i = 0; i < nFt; ++i)
        if (holds(R, Ft[i], l)) vs[m++] = Ft[i];
      double pos[3];
      mean_pos(R, vs, m, pos);
      free(vs);
      int32_t node = add_node(R, N_END, t, pos);
      R->lst[l] = L_ENDED;
      R->ldeath[l] = node;
      R->cnt[5]++;
      continue;
    }
    /* split: band in ascending vertex order for the node position */
    double pos[3];
    mean_pos(R, bandv, nb, pos);
    int32_t node = add_node(R, N_SPLIT, t, pos);
    R->lst[l] = L_DEAD;
    R->ldeath[l] = node;
    R->cnt[4]++;
    for (int64_t c = 0; c < nc; ++c) {
      int32_t child = new_layer(R, node);
      for (int64_t i = compstart[c]; i < compstart[c + 1]; ++i) {
        int64_t v = queue[i];
        for (int q = 0; q < R->en[v]; ++q)
          if (R->el[v * KM + q] == l) R->el[v * KM + q] = child;
        /* keep the row ascending */
        int32_t ls[KM];
        double xs[KM];
        int n = R->en[v];
        for (int q = 0; q < n; ++q) { ls[q] = R->el[v * KM + q]; xs[q] = R->ex[v * KM + q]; }
        for (int p = 1; p < n; ++p)
          for (int q = p; q > 0 && ls[q - 1] > ls[q]; --q) {
            int32_t tl = ls[q]; ls[q] = ls[q - 1]; ls[q - 1] = tl;
            double tx = xs[q]; xs[q] = xs[q - 1]; xs[q - 1] = tx;
          }
        set_row(R, v, n, ls, xs);
      }
    }
  }
  free(alive); free(bandv); free(queue); free(compstart);
  return ST_OK;
}

/* ------------------------------------------------------- initial pass */
static int initial_pass(orc_run *R, int32_t seed) {
  int64_t nv = R->nv;
  R->en = (int32_t *)calloc(nv, sizeof(int32_t));
  R->el = (int32_t *)malloc(sizeof(int32_t) * nv * KM);
  R->ex = (double *)malloc(sizeof(double) * nv * KM);
  R->cover = (int32_t *)malloc(sizeof(int32_t) * nv);
  for (int64_t v = 0; v < nv; ++v) R->cover[v] = -1;
  double pos[3] = {R->X[3 * seed], R->X[3 * seed + 1], R->X[3 * seed + 2]};
  int32_t node = add_node(R, N_SEED, 0, pos);
  int32_t l1 = new_layer(R, node);
  int64_t *F0 = (int64_t *)malloc(sizeof(int64_t) * (nv + 1));
  int64_t nF0 = 0;
  /* seed region, value 1; the column sum is already 1 */
  F0[nF0++] = seed;
  if (R->opt.seed_ring)
    for (int64_t k = R->rp[seed]; k < R->rp[seed + 1]; ++k) F0[nF0++] = R->col[k];
  for (int64_t i = 0; i < nF0; ++i) {
    int64_t v = F0[i];
    R->en[v] = 1;
    R->el[v * KM] = l1;
    R->ex[v * KM] = 1.0;
    R->cover[v] = 0;
  }
  /* candidate set for the first frontier: the seed region and its neighbours */
  int64_t *cand = (int64_t *)malloc(sizeof(int64_t) * (nv + 1));
  int64_t *Fl = (int64_t *)malloc(sizeof(int64_t) * (nv + 1));
  int32_t *nls = (int32_t *)malloc(sizeof(int32_t) * (nv + 1) * KM);
  double *nxs = (double *)malloc(sizeof(double) * (nv + 1) * KM);
  int32_t *nn = (int32_t *)malloc(sizeof(int32_t) * (nv + 1));
  int64_t ncand = 0;
  int32_t sid = ++R->stamp_id;
  for (int64_t i = 0; i < nF0; ++i) {
    int64_t v = F0[i];
    for (int64_t k = R->rp[v] - 1; k < R->rp[v + 1]; ++k) {
      int64_t u = (k < R->rp[v]) ? v : R->col[k];
      if (R->stamp[u] != sid) { R->stamp[u] = sid; cand[ncand++] = u; }
    }
  }
  free(F0);
  int st = ST_OK;
  int32_t t = 0;
  for (;;) {
    /* frontier of step t+1 */
    int64_t nF = 0;
    if (R->opt.naive) {
      for (int64_t v = 0; v < nv; ++v)
        if (in_frontier(R, v)) Fl[nF++] = v;
    } else {
      /* ascending order */
      int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (ncand + 1));
      for (int64_t i = 0; i < ncand; ++i) tmp[i] = (int32_t)cand[i];
      qsort(tmp, ncand, sizeof(int32_t), cmp_i32);
      for (int64_t i = 0; i < ncand; ++i)
        if (in_frontier(R, tmp[i])) Fl[nF++] = tmp[i];
      free(tmp);
    }
    if (nF == 0) break;
    if (t >= R->opt.max_steps) { st = ST_EMAXSTEPS; break; }
    ++t;
    R->cnt[0] += nF;
    /* Jacobi update */
    for (int64_t i = 0; i < nF; ++i) {
      int n = compute_update(R, Fl[i], nls + i * KM, nxs + i * KM);
      if (n < 0) { st = ST_ESLOTS; break; }
      nn[i] = n;
    }
    if (st) break;
    for (int64_t i = 0; i < nF; ++i) {
      /* frozen entries never reach here; the row becomes exactly the updated layers */
      st = set_row(R, Fl[i], nn[i], nls + i * KM, nxs + i * KM);
      if (st) break;
    }
    if (st) break;
    const int64_t *scan = Fl;
    int64_t nscan = nF;
    int64_t *all = NULL;
    if (R->opt.naive) {
      all = (int64_t *)malloc(sizeof(int64_t) * nv);
      for (int64_t v = 0; v < nv; ++v) all[v] = v;
      scan = all;
      nscan = nv;
    }
    st = do_merges(R, t, scan, nscan);
    if (!st) st = do_splits(R, t, scan, nscan, Fl, nF);
    if (st) { free(all); break; }
    for (int64_t i = 0; i < nscan; ++i) {
      int64_t v = scan[i];
      if (R->cover[v] < 0 && R->en[v] > 0) R->cover[v] = t;
    }
    if (R->opt.record_steps) {
      uint64_t hsh = 0;
      int64_t nb = 0;
      for (int64_t i = 0; i < nscan; ++i) {
        int64_t v = scan[i];
        for (int q = 0; q < R->en[v]; ++q) {
          int32_t l = R->el[v * KM + q];
          double x = R->ex[v * KM + q];
          if (R->lst[l] == L_ALIVE && x > 0.0 && x < 1.0) {
            hsh += mix64(((uint64_t)v << 32) | (uint32_t)l);
            ++nb;
          }
        }
      }
      if (R->nrec == R->caprec) {
        R->caprec = R->caprec * 2 + 256;
        R->rec = (int64_t *)realloc(R->rec, sizeof(int64_t) * 4 * R->caprec);
      }
      R->rec[4 * R->nrec] = nF;
      R->rec[4 * R->nrec + 1] = nb;
      R->rec[4 * R->nrec + 2] = (int64_t)(hsh & 0xffffffffull);
      R->rec[4 * R->nrec + 3] = (int64_t)(hsh >> 32);
      R->nrec++;
    }
    free(all);
    /* candidates of the next frontier: closed neighbourhood of this step's frontier */
    sid = ++R->stamp_id;
    ncand = 0;
    for (int64_t i = 0; i < nF; ++i) {
      int64_t v = Fl[i];
      for (int64_t k = R->rp[v] - 1; k < R->rp[v + 1]; ++k) {
        int64_t u = (k < R->rp[v]) ? v : R->col[k];
        if (R->stamp[u] != sid) { R->stamp[u] = sid; cand[ncand++] = u; }
      }
    }
  }
  R->steps = t;
  free(cand); free(Fl); free(nls); free(nxs); free(nn);
  if (st == ST_OK) {
    for (int64_t v = 0; v < nv; ++v)
      if (R->en[v] == 0 || base_val(R, v) > 0.0) { st = ST_ESTALL; break; }
    for (int32_t l = 1; l <= R->nl && st == ST_OK; ++l)
      if (R->lst[l] == L_ALIVE) st = ST_ESTALL;
  }
  return st;
}

/* ------------------------------------------------- PL streamline (Sec. 3.2) */
/* The tunnel pass's streamline: steepest descent of the arrival time interpolated linearly over the
   faces of the cut, restricted domain, from the first far-side vertex reached back to a source.
   Arrival time: the step at which theta is crossed, with the fraction of that step found by linear
   interpolation of the value in time; sources 0, unreached -1.  A face is usable when its three
   vertices are reached and none of its edges is cut.  In a face with corners (p0, p1, p2), the
   gradient is g = al e1 + be e2 (e1 = p1 - p0, e2 = p2 - p0), from the Gram system of e1, e2.
   At a vertex: among the usable faces around it (CSR order) whose descent direction -g points into
   the face's corner there, the steepest (largest |g|, the first on ties); the path crosses that face
   to its opposite edge.  With none, it follows the steepest descending kept edge.  On an edge: into
   the face beyond it if -g enters that face (and the face is usable), to the edge where the ray
   leaves it; else along the edge to its lower end (smaller arrival, then smaller id).  It ends at a
   source; a vertex with no descent left fails.  Points: the start vertex, every edge crossing, every
   vertex passed.  Point budget, the closure included: min(SL_MAX, nv / 4 + 64) for a mesh of nv
   vertices (the loops seen take a few hundredths of nv); a trace past it fails with ST_ELAYERS. */
#define SL_MAX 16384
static int64_t sl_budget(const orc_run *R) { return R->nv / 4 + 64 < SL_MAX ? R->nv / 4 + 64 : SL_MAX; }
static int face_usable(const orc_run *R, const double *tf, const char *cut, int32_t f) {
  const int32_t *t = R->F + 3 * f;
  for (int q = 0; q < 3; ++q) {
    if (tf[t[q]] < 0.0) return 0;
    int64_t k = slot_of(R, t[q], t[(q + 1) % 3]);
    if (k < 0 || cut[k]) return 0;
  }
  return 1;
}
static int32_t third_vertex(const orc_run *R, int32_t f, int32_t a, int32_t b) {
  const int32_t *t = R->F + 3 * f;
  for (int q = 0; q < 3; ++q)
    if (t[q] != a && t[q] != b) return t[q];
  return -1;
}
/* gradient coefficients (al, be) and |g|^2 of the arrival time on the face (p0, p1, p2); 0 if degenerate */
static int grad_face(const orc_run *R, const double *tf, int32_t p0, int32_t p1, int32_t p2, double *al, double *be,
                     double *n2) {
  const double *x0 = R->X + 3 * p0, *x1 = R->X + 3 * p1, *x2 = R->X + 3 * p2;
  double e1[3], e2[3];
  for (int d = 0; d < 3; ++d) { e1[d] = x1[d] - x0[d]; e2[d] = x2[d] - x0[d]; }
  double g11 = (e1[0] * e1[0] + e1[1] * e1[1]) + e1[2] * e1[2];
  double g12 = (e1[0] * e2[0] + e1[1] * e2[1]) + e1[2] * e2[2];
  double g22 = (e2[0] * e2[0] + e2[1] * e2[1]) + e2[2] * e2[2];
  double det = g11 * g22 - g12 * g12;
  if (!(det > 0.0)) return 0;
  double d1 = tf[p1] - tf[p0], d2 = tf[p2] - tf[p0];
  double a = (g22 * d1 - g12 * d2) / det, b = (g11 * d2 - g12 * d1) / det;
  *al = a;
  *be = b;
  *n2 = ((a * a) * g11 + ((a + a) * b) * g12) + (b * b) * g22;
  return 1;
}
static int sl_push(double **pts, int64_t *n, int64_t *cap, const double *p, int64_t budget) {
  if (*n >= budget) return 0;
  if (*n == *cap) { *cap *= 2; *pts = (double *)realloc(*pts, sizeof(double) * 3 * *cap); }
  for (int d = 0; d < 3; ++d) (*pts)[3 * *n + d] = p[d];
  ++*n;
  return 1;
}
static int streamline(const orc_run *R, const double *tf, const char *cut, int32_t start, double **pts_out,
                      int64_t *n_out, int32_t *end_vertex) {
  int64_t cap = 256, n = 0;
  double *pts = (double *)malloc(sizeof(double) * 3 * cap);
  int32_t v = start, ex = -1, ey = -1;
  double mu = 0.0;
  int at_vertex = 1, st = ST_ELOOPFAIL;
  const int64_t budget = sl_budget(R);
  sl_push(&pts, &n, &cap, R->X + 3 * v, budget);
  for (int64_t it = 0; it < 4 * SL_MAX; ++it) {
    if (at_vertex) {
      if (tf[v] == 0.0) { st = ST_OK; *end_vertex = v; break; }
      double best = -1.0, bal = 0.0, bbe = 0.0;
      int32_t bu = -1, bw = -1;
      for (int64_t k = R->rp[v]; k < R->rp[v + 1]; ++k) {
        int32_t u = R->col[k], f = R->hface[k], w = third_vertex(R, f, v, u);
        double al, be, n2;
        if (!face_usable(R, tf, cut, f) || !grad_face(R, tf, v, u, w, &al, &be, &n2)) continue;
        if (!(al <= 0.0 && be <= 0.0 && (al < 0.0 || be < 0.0))) continue; /* -g not into this corner */
        if (n2 > best) { best = n2; bal = al; bbe = be; bu = u; bw = w; }
      }
      if (bu >= 0) {
        double lam = bbe / (bal + bbe); /* where the ray meets edge u -> w, from u */
        if (lam <= 0.0) { v = bu; if (!sl_push(&pts, &n, &cap, R->X + 3 * v, budget)) break; continue; }
        if (lam >= 1.0) { v = bw; if (!sl_push(&pts, &n, &cap, R->X + 3 * v, budget)) break; continue; }
        double p[3];
        for (int d = 0; d < 3; ++d) p[d] = R->X[3 * bu + d] + lam * (R->X[3 * bw + d] - R->X[3 * bu + d]);
        if (!sl_push(&pts, &n, &cap, p, budget)) break;
        ex = bw; ey = bu; mu = 1.0 - lam; /* into the face left of w -> u */
        at_vertex = 0;
        continue;
      }
      double bs = 0.0;
      int32_t bn = -1;
      for (int64_t k = R->rp[v]; k < R->rp[v + 1]; ++k) {
        int32_t u = R->col[k];
        if (cut[k] || tf[u] < 0.0) continue;
        const double *a = R->X + 3 * v, *b = R->X + 3 * u;
        double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
        double sl = (tf[v] - tf[u]) / sqrt((dx * dx + dy * dy) + dz * dz);
        if (sl > bs) { bs = sl; bn = u; }
      }
      if (bn < 0) break; /* no descent left */
      v = bn;
      if (!sl_push(&pts, &n, &cap, R->X + 3 * v, budget)) break;
      continue;
    }
    /* on edge ex -> ey at mu from ex, entering the face left of it */
    int64_t k = slot_of(R, ex, ey);
    int32_t f = k >= 0 ? R->hface[k] : -1, z = f >= 0 ? third_vertex(R, f, ex, ey) : -1;
    double al = 0.0, be = 0.0, n2 = 0.0;
    if (f < 0 || !face_usable(R, tf, cut, f) || !grad_face(R, tf, ex, ey, z, &al, &be, &n2) || !(be < 0.0)) {
      v = (tf[ex] < tf[ey] || (tf[ex] == tf[ey] && ex < ey)) ? ex : ey; /* along the edge to its lower end */
      at_vertex = 1;
      if (!sl_push(&pts, &n, &cap, R->X + 3 * v, budget)) break;
      continue;
    }
    /* ray (u, w) = (mu - s al, -s be) in the frame (e1, e2) of the face (ex, ey, z) */
    double su = al > 0.0 ? mu / al : INFINITY;
    double suw = (al + be) < 0.0 ? (mu - 1.0) / (al + be) : INFINITY;
    double p[3];
    if (su <= suw) { /* leaves through the edge from ex to z (u = 0) */
      double w = -(su * be);
      if (w >= 1.0) { v = z; at_vertex = 1; if (!sl_push(&pts, &n, &cap, R->X + 3 * v, budget)) break; continue; }
      if (w <= 0.0) { v = ex; at_vertex = 1; if (!sl_push(&pts, &n, &cap, R->X + 3 * v, budget)) break; continue; }
      for (int d = 0; d < 3; ++d) p[d] = R->X[3 * ex + d] + w * (R->X[3 * z + d] - R->X[3 * ex + d]);
      ey = z; mu = w; /* into the face left of ex -> z */
    } else { /* leaves through the edge from ey to z (u + w = 1) */
      double w = -(suw * be);
      if (w >= 1.0) { v = z; at_vertex = 1; if (!sl_push(&pts, &n, &cap, R->X + 3 * v, budget)) break; continue; }
      if (w <= 0.0) { v = ey; at_vertex = 1; if (!sl_push(&pts, &n, &cap, R->X + 3 * v, budget)) break; continue; }
      for (int d = 0; d < 3; ++d) p[d] = R->X[3 * ey + d] + w * (R->X[3 * z + d] - R->X[3 * ey + d]);
      ex = z; mu = 1.0 - w; /* into the face left of z -> ey */
    }
    if (!sl_push(&pts, &n, &cap, p, budget)) break;
  }
  *pts_out = pts;
  *n_out = n;
  return st;
}
/* close the streamline along the loop, as the vertex trace is closed: from the source reached, the
   shorter way along the loop to a crossing edge ending at the start */
static int close_streamline(const orc_run *R, const handle_t *H, int64_t m, int32_t bstar, int32_t xs, double **pts,
                            int64_t *n) {
  int64_t bd = -1, bj = -1;
  int dir = 1;
  for (int64_t i = 0; i < m; ++i) {
    if (H->edges[2 * i + 1] != bstar) continue;
    for (int64_t j = 0; j < m; ++j) {
      if (H->edges[2 * j] != xs) continue;
      int64_t fwd = ((i - j) % m + m) % m, bwd = ((j - i) % m + m) % m;
      int64_t d = fwd <= bwd ? fwd : bwd;
      if (bd < 0 || d < bd) { bd = d; bj = j; dir = fwd <= bwd ? 1 : -1; }
    }
  }
  if (bd < 0) return ST_ELOOPFAIL;
  int64_t cap = *n > 0 ? *n : 1;
  int32_t last = xs;
  for (int64_t s = 1; s <= bd; ++s) {
    int64_t idx = ((bj + dir * s) % m + m) % m;
    int32_t a = H->edges[2 * idx];
    if (a == last) continue;
    if (*n >= sl_budget(R)) return ST_ELAYERS;
    *pts = (double *)realloc(*pts, sizeof(double) * 3 * (*n + 1));
    for (int d = 0; d < 3; ++d) (*pts)[3 * *n + d] = R->X[3 * a + d];
    ++*n;
    last = a;
  }
  (void)cap;
  return ST_OK;
}
static double polyline_length(const double *p, int64_t n) {
  double len = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double *a = p + 3 * i, *b = p + 3 * ((i + 1) % n);
    double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
    len = len + sqrt((dx * dx + dy * dy) + dz * dz);
  }
  return len;
}

/* --------------------------------------------------------- tunnel pass */
static int tunnel_pass(orc_run *R, handle_t *H, int32_t th_step) {
  int64_t nv = R->nv;
  int64_t m = H->info[3];
  double th = R->opt.theta_iso;
  if (m == 0) { H->tinfo[0] = ST_ELOOPFAIL; return ST_ELOOPFAIL; }
  char *dom = (char *)calloc(nv, 1);
  char *cut = (char *)calloc(R->nnz, 1);
  char *src = (char *)calloc(nv, 1), *tgt = (char *)calloc(nv, 1);
  for (int64_t v = 0; v < nv; ++v) dom[v] = R->cover[v] >= 0 && R->cover[v] <= th_step;
  for (int64_t i = 0; i < m; ++i) {
    int32_t a = H->edges[2 * i], b = H->edges[2 * i + 1];
    cut[slot_of(R, a, b)] = 1;
    cut[slot_of(R, b, a)] = 1;
    src[a] = 1;
    tgt[b] = 1;
  }
  /* restricted operator: kept edges inside the domain, rows renormalised */
  int64_t *hp = (int64_t *)calloc(nv + 1, sizeof(int64_t));
  for (int64_t v = 0; v < nv; ++v) {
    int64_t d = 0;
    if (dom[v])
      for (int64_t k = R->rp[v]; k < R->rp[v + 1]; ++k)
        if (dom[R->col[k]] && !cut[k]) ++d;
    hp[v + 1] = hp[v] + d;
  }
  int32_t *hc = (int32_t *)malloc(sizeof(int32_t) * (hp[nv] + 1));
  double *hv = (double *)malloc(sizeof(double) * (hp[nv] + 1));
  double *hd = (double *)malloc(sizeof(double) * nv);
  for (int64_t v = 0; v < nv; ++v) {
    int64_t d = hp[v + 1] - hp[v], q = hp[v];
    hd[v] = d > 0 ? -R->s : 0.0;
    if (!dom[v]) continue;
    for (int64_t k = R->rp[v]; k < R->rp[v + 1]; ++k)
      if (dom[R->col[k]] && !cut[k]) { hc[q] = R->col[k]; hv[q] = R->s / (double)d; ++q; }
  }
  double *phi = (double *)calloc(nv, sizeof(double));
  int32_t *T = (int32_t *)malloc(sizeof(int32_t) * nv);
  double *tf = (double *)malloc(sizeof(double) * nv); /* arrival step with its fraction (-1 unreached) */
  for (int64_t v = 0; v < nv; ++v) {
    T[v] = -1;
    tf[v] = -1.0;
    if (src[v]) { phi[v] = 1.0; T[v] = 0; tf[v] = 0.0; }
  }
  int64_t *cand = (int64_t *)malloc(sizeof(int64_t) * (nv + 1));
  int64_t *Fl = (int64_t *)malloc(sizeof(int64_t) * (nv + 1));
  double *nphi = (double *)malloc(sizeof(double) * (nv + 1));
  int64_t ncand = 0;
  int32_t sid = ++R->stamp_id;
  for (int64_t v = 0; v < nv; ++v)
    if (src[v])
      for (int64_t k = hp[v] - 1; k < hp[v + 1]; ++k) {
        int64_t u = (k < hp[v]) ? v : hc[k];
        if (R->stamp[u] != sid) { R->stamp[u] = sid; cand[ncand++] = u; }
      }
  int st = ST_OK;
  int32_t tau = 0, bstar = -1;
  for (;;) {
    int64_t nF = 0;
    int64_t lim = R->opt.naive ? nv : ncand;
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (lim + 1));
    for (int64_t i = 0; i < lim; ++i) tmp[i] = R->opt.naive ? (int32_t)i : (int32_t)cand[i];
    if (!R->opt.naive) qsort(tmp, lim, sizeof(int32_t), cmp_i32);
    for (int64_t i = 0; i < lim; ++i) {
      int64_t v = tmp[i];
      if (!dom[v] || src[v]) continue;
      int lay = 0, bas = 0;
      for (int64_t k = hp[v] - 1; k < hp[v + 1]; ++k) {
        int64_t u = (k < hp[v]) ? v : hc[k];
        if (phi[u] > 0.0) lay = 1;
        if (1.0 - phi[u] > 0.0) bas = 1;
      }
      if (lay && bas) Fl[nF++] = v;
    }
    free(tmp);
    if (nF == 0) { st = ST_ELOOPFAIL; break; }
    if (tau >= R->opt.max_pass_steps) { st = ST_EMAXSTEPS; break; }
    ++tau;
    R->cnt[2] += nF;
    for (int64_t i = 0; i < nF; ++i) {
      int64_t v = Fl[i];
      double acc = 0.0, accb = 0.0;
      for (int64_t k = hp[v]; k < hp[v + 1]; ++k) acc = acc + hv[k] * phi[hc[k]];
      acc = acc + hd[v] * phi[v];
      for (int64_t k = hp[v]; k < hp[v + 1]; ++k) accb = accb + hv[k] * (1.0 - phi[hc[k]]);
      accb = accb + hd[v] * (1.0 - phi[v]);
      double x = phi[v], out;
      if (vertex_update(R, 1, &x, &acc, 1.0 - x, accb, &out) != 0) { R->cnt[1]++; out = x; }
      nphi[i] = out;
    }
    for (int64_t i = 0; i < nF; ++i) {
      int64_t v = Fl[i];
      double old = phi[v];
      phi[v] = nphi[i];
      if (T[v] < 0 && phi[v] >= th) {
        T[v] = tau;
        /* theta crossed between the step's old and new value: linear in time within the step */
        tf[v] = (double)(tau - 1) + (th - old) / (phi[v] - old);
      }
    }
    for (int64_t i = 0; i < nF; ++i) {
      int64_t v = Fl[i];
      if (tgt[v] && T[v] == tau && (bstar < 0 || v < bstar)) bstar = (int32_t)v;
    }
    if (bstar >= 0) break;
    sid = ++R->stamp_id;
    ncand = 0;
    for (int64_t i = 0; i < nF; ++i) {
      int64_t v = Fl[i];
      for (int64_t k = hp[v] - 1; k < hp[v + 1]; ++k) {
        int64_t u = (k < hp[v]) ? v : hc[k];
        if (R->stamp[u] != sid) { R->stamp[u] = sid; cand[ncand++] = u; }
      }
    }
  }
  H->tinfo[1] = tau;
  H->tinfo[2] = bstar;
  if (st == ST_OK) {
    /* descent on the arrival steps in the cut, restricted graph, depth first: from the path's
       last vertex x go to the unvisited reached neighbour u with the least key
       (T(u) > T(x), T(u), u) -- steps that do not raise the arrival step first, then the
       earliest, then the smallest id; with none left, drop x from the path and go on from the
       vertex before it.  Ends at a source (T = 0); fails only when the path empties. */
    int32_t *path = (int32_t *)malloc(sizeof(int32_t) * (nv + 1));
    int64_t np = 0;
    sid = ++R->stamp_id;
    int32_t x = bstar;
    path[np++] = x;
    R->stamp[x] = sid;
    while (T[x] != 0) {
      int32_t best = -1, bup = 0;
      for (int64_t k = hp[x]; k < hp[x + 1]; ++k) {
        int32_t u = hc[k];
        if (T[u] < 0 || R->stamp[u] == sid) continue;
        int up = T[u] > T[x];
        if (best < 0 || up < bup || (up == bup && (T[u] < T[best] || (T[u] == T[best] && u < best)))) {
          best = u;
          bup = up;
        }
      }
      if (best < 0) {
        if (np <= 1) { st = ST_ELOOPFAIL; break; }
        --np;
        x = path[np - 1];
        continue;
      }
      R->stamp[best] = sid;
      path[np++] = best;
      x = best;
    }
    if (st == ST_OK) {
      /* close along the handle loop from the reached source to an edge ending at b* */
      int64_t bi = -1, bj = -1, bd = -1;
      int bdir = 0;
      for (int64_t i = 0; i < m; ++i) {
        if (H->edges[2 * i + 1] != bstar) continue;
        for (int64_t j = 0; j < m; ++j) {
          if (H->edges[2 * j] != x) continue;
          int64_t fwd = ((i - j) % m + m) % m, bwd = ((j - i) % m + m) % m;
          int64_t d = fwd <= bwd ? fwd : bwd;
          int dir = fwd <= bwd ? 1 : -1;
          if (bd < 0 || d < bd) { bd = d; bi = i; bj = j; bdir = dir; }
        }
      }
      int32_t *cyc = (int32_t *)malloc(sizeof(int32_t) * (np + m + 2));
      int64_t nc = 0;
      for (int64_t i = 0; i < np; ++i) cyc[nc++] = path[i];
      for (int64_t s = 1; s <= bd; ++s) {
        int64_t idx = ((bj + bdir * s) % m + m) % m;
        int32_t a = H->edges[2 * idx];
        if (cyc[nc - 1] != a) cyc[nc++] = a;
      }
      (void)bi;
      while (nc > 1 && cyc[nc - 1] == cyc[0]) --nc;
      H->tverts = cyc;
      H->tinfo[3] = (int32_t)nc;
    }
    free(path);
    if (st == ST_OK && R->opt.streamlines) {
      int32_t xs = -1;
      double *sp = NULL;
      int64_t sn = 0;
      int sst = streamline(R, tf, cut, bstar, &sp, &sn, &xs);
      if (sst == ST_OK) sst = close_streamline(R, H, m, bstar, xs, &sp, &sn);
      H->sst[0] = sst;
      H->spts[0] = sp;
      H->sn[0] = sst == ST_OK ? sn : 0;
      H->slen[0] = sst == ST_OK ? polyline_length(sp, sn) : 0.0;
    }
  }
  H->tinfo[0] = st;
  if (R->opt.record_steps) { H->arrival = T; H->tfa = tf; tf = NULL; }
  else free(T);
  free(dom); free(cut); free(src); free(tgt); free(hp); free(hc); free(hv); free(hd);
  free(phi); free(tf); free(cand); free(Fl); free(nphi);
  return st;
}

/* -------------------------------------------------- handle refinement pass */
/* The third vertex of the face left of half-edge c->u, i.e. the neighbour that follows u in
   counter-clockwise order around c (faces are counter-clockwise); -1 if c->u is no half-edge. */
static int32_t next_ccw(const orc_run *R, int32_t c, int32_t u) {
  int64_t k = slot_of(R, c, u);
  if (k < 0) return -1;
  const int32_t *t = R->F + 3 * R->hface[k];
  for (int q = 0; q < 3; ++q)
    if (t[q] != c && t[q] != u) return t[q];
  return -1;
}

/* Sec. 3.3: the refined handle loop comes from the same single-layer pass as the tunnel loop, now
   started on one side of the tunnel loop, with the tunnel loop as the only border (no restriction
   to a covered area); the trace from the first far-side vertex reached, closed along the tunnel
   loop, is the refined handle.
   The tunnel cycle is first made simple by erasing its closed sub-loops in order along it from its
   first vertex: the cycle crosses the handle loop once, on its closing edge, which the erasure
   keeps, and an erased sub-loop never crosses it, so the simple cycle lies in the same class
   modulo loops that pair evenly with the handle loop.  Sources: the cycle's vertices.  Border: the
   edges from a cycle vertex c_i to its neighbours on the right, those met counter-clockwise from
   c_{i-1} to c_{i+1} around c_i (the surface is oriented by its counter-clockwise faces); those
   neighbours are the far side.  Returns the pass status. */
static int refine_pass(orc_run *R, handle_t *H) {
  H->rinfo[0] = ST_ELOOPFAIL;
  H->rinfo[1] = 0;
  H->rinfo[2] = -1;
  H->rinfo[3] = 0;
  if (H->tinfo[0] != ST_OK || !H->tverts || H->tinfo[3] < 3) return ST_ELOOPFAIL;
  int64_t k = H->tinfo[3];
  int32_t *cyc = (int32_t *)malloc(sizeof(int32_t) * k);
  int64_t n = 0;
  for (int64_t i = 0; i < k; ++i) {
    int32_t v = H->tverts[i];
    int64_t j = 0;
    while (j < n && cyc[j] != v) ++j;
    if (j < n) n = j + 1; /* v closes a sub-loop: erase it */
    else cyc[n++] = v;
  }
  if (n < 3) { free(cyc); return ST_ELOOPFAIL; }
  int32_t sid = ++R->stamp_id;
  for (int64_t i = 0; i < n; ++i) R->stamp[cyc[i]] = sid;
  int64_t cap = 64, m = 0;
  int32_t *xe = (int32_t *)malloc(sizeof(int32_t) * 2 * cap);
  for (int64_t i = 0; i < n; ++i) {
    int32_t c = cyc[i], prv = cyc[(i + n - 1) % n], nxt = cyc[(i + 1) % n];
    int64_t deg = R->rp[c + 1] - R->rp[c], guard = 0;
    int32_t u = prv;
    for (;;) {
      u = next_ccw(R, c, u);
      if (u < 0 || u == nxt || ++guard > deg) break;
      if (R->stamp[u] == sid) continue; /* a chord to another cycle vertex */
      if (m == cap) { cap *= 2; xe = (int32_t *)realloc(xe, sizeof(int32_t) * 2 * cap); }
      xe[2 * m] = c;
      xe[2 * m + 1] = u;
      ++m;
    }
  }
  free(cyc);
  if (m == 0) { free(xe); return ST_ELOOPFAIL; }
  handle_t T;
  memset(&T, 0, sizeof(T));
  T.sst[0] = -1;
  T.edges = xe;
  T.info[3] = (int32_t)m;
  int st = tunnel_pass(R, &T, INT32_MAX);
  for (int q = 0; q < 4; ++q) H->rinfo[q] = T.tinfo[q];
  H->rinfo[0] = st;
  H->rverts = T.tverts;
  H->sst[1] = T.sst[0];
  H->spts[1] = T.spts[0];
  H->sn[1] = T.sn[0];
  H->slen[1] = T.slen[0];
  free(T.arrival);
  free(T.tfa);
  free(xe);
  return st;
}

/* ------------------------------------------------ loop classification */
/* Sec. 3.5: a loop is offset slightly along the surface normals and its length compared: tunnel
   loops sit in saddle-shaped parts and shrink, handle loops grow.  Normals: the unit vertex normal
   is the sum of the (area-weighted) normals of the faces around the vertex, taken in the vertex's
   CSR order; an isoline point on edge (a, b) takes the normalised sum of a's and b's.  Offset: the
   option's fraction of the mean edge length.  Returns length(offset loop) - length(loop). */
static void vertex_normals(orc_run *R) {
  int64_t nv = R->nv, nf = R->nf;
  double *fn = (double *)malloc(sizeof(double) * 3 * nf);
  for (int64_t f = 0; f < nf; ++f) {
    const double *a = R->X + 3 * R->F[3 * f], *b = R->X + 3 * R->F[3 * f + 1], *c = R->X + 3 * R->F[3 * f + 2];
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    fn[3 * f] = u[1] * w[2] - u[2] * w[1];
    fn[3 * f + 1] = u[2] * w[0] - u[0] * w[2];
    fn[3 * f + 2] = u[0] * w[1] - u[1] * w[0];
  }
  R->vn = (double *)malloc(sizeof(double) * 3 * nv);
  double esum = 0.0;
  for (int64_t v = 0; v < nv; ++v) {
    double n[3] = {0.0, 0.0, 0.0};
    for (int64_t k = R->rp[v]; k < R->rp[v + 1]; ++k) {
      const double *g = fn + 3 * R->hface[k];
      for (int d = 0; d < 3; ++d) n[d] = n[d] + g[d];
      int32_t u = R->col[k];
      if (u > v) {
        double dx = R->X[3 * u] - R->X[3 * v], dy = R->X[3 * u + 1] - R->X[3 * v + 1], dz = R->X[3 * u + 2] - R->X[3 * v + 2];
        esum = esum + sqrt(dx * dx + dy * dy + dz * dz);
      }
    }
    double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int d = 0; d < 3; ++d) R->vn[3 * v + d] = len > 0.0 ? n[d] / len : 0.0;
  }
  R->mean_edge = esum / (double)(R->nnz / 2);
  free(fn);
}
static double dist3(const double *p, const double *q) {
  double dx = q[0] - p[0], dy = q[1] - p[1], dz = q[2] - p[2];
  return sqrt(dx * dx + dy * dy + dz * dz);
}
/* points P[n][3] with unit normals N[n][3], closed polyline */
static double offset_change(const orc_run *R, const double *P, const double *N, int64_t n) {
  double del = R->opt.offset * R->mean_edge, l0 = 0.0, l1 = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t j = (i + 1) % n;
    double p[3], q[3];
    for (int d = 0; d < 3; ++d) { p[d] = P[3 * i + d] + del * N[3 * i + d]; q[d] = P[3 * j + d] + del * N[3 * j + d]; }
    l0 = l0 + dist3(P + 3 * i, P + 3 * j);
    l1 = l1 + dist3(p, q);
  }
  return l1 - l0;
}
static double cycle_offset_change(const orc_run *R, const int32_t *verts, int64_t n) {
  if (n < 2) return NAN;
  double *P = (double *)malloc(sizeof(double) * 3 * n), *N = (double *)malloc(sizeof(double) * 3 * n);
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) { P[3 * i + d] = R->X[3 * verts[i] + d]; N[3 * i + d] = R->vn[3 * verts[i] + d]; }
  double r = offset_change(R, P, N, n);
  free(P); free(N);
  return r;
}
static double isoline_offset_change(const orc_run *R, const handle_t *H) {
  int64_t n = H->info[3];
  if (n < 2) return NAN;
  double *N = (double *)malloc(sizeof(double) * 3 * n);
  for (int64_t i = 0; i < n; ++i) {
    const double *na = R->vn + 3 * H->edges[2 * i], *nb = R->vn + 3 * H->edges[2 * i + 1];
    double s[3] = {na[0] + nb[0], na[1] + nb[1], na[2] + nb[2]};
    double len = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    for (int d = 0; d < 3; ++d) N[3 * i + d] = len > 0.0 ? s[d] / len : 0.0;
  }
  double r = offset_change(R, H->pts, N, n);
  free(N);
  return r;
}

/* ------------------------------------------------------------------ API */
orc_run *orc_detect(const double *X, int64_t nv, const int32_t *F, int64_t nf, int32_t seed_vertex,
                    const orc_options *o) {
  orc_run *R = (orc_run *)calloc(1, sizeof(orc_run));
  R->opt = *o;
  R->nv = nv;
  R->nf = nf;
  double c[4];
  orc_constants(o, c);
  R->eta = c[0]; R->lbar = c[1]; R->dt = c[2]; R->s = c[3];
  R->ah = o->a * o->a / 2.0;
  R->one_m_eps = 1.0 - o->eps0;
  R->status = build_mesh(R, X, F);
  if (R->status == ST_OK && (seed_vertex < 0 || seed_vertex >= nv)) R->status = ST_EINVAL;
  if (R->status != ST_OK) return R;
  R->stamp = (int32_t *)calloc(nv, sizeof(int32_t));
  R->status = initial_pass(R, seed_vertex);
  const int initial_ok = R->status == ST_OK;
  const int32_t npass = o->max_passes > 0 && o->max_passes < R->nh ? o->max_passes : R->nh;
  for (int32_t h = 0; h < R->nh; ++h) R->h[h].tinfo[0] = -1;
  if (R->status == ST_OK && o->tunnels)
    for (int32_t h = 0; h < npass; ++h) {
      /* Sec. 3.2: the pass is restricted to the area covered when the handle was found.  When
         the kept handle loop separates that area (its far side cannot be reached), the pass
         runs again on the whole surface. */
      handle_t *H = &R->h[h];
      int st = tunnel_pass(R, H, H->info[0]);
      if (st == ST_ELOOPFAIL && H->info[3] > 0 && H->tinfo[2] < 0) {
        free(H->arrival);
        free(H->tfa);
        H->arrival = NULL;
        H->tfa = NULL;
        st = tunnel_pass(R, H, INT32_MAX);
      }
      if (st != ST_OK && R->status == ST_OK) R->status = st;
    }
  /* Sec. 3.3: a refinement pass for every handle whose tunnel pass succeeded */
  for (int32_t h = 0; h < R->nh; ++h) R->h[h].rinfo[0] = -1;
  if (initial_ok && o->tunnels && o->refine)
    for (int32_t h = 0; h < npass; ++h) {
      if (R->h[h].tinfo[0] != ST_OK) continue;
      int st = refine_pass(R, &R->h[h]);
      if (st != ST_OK && R->status == ST_OK) R->status = st;
    }
  vertex_normals(R);
  for (int32_t h = 0; h < R->nh; ++h) {
    handle_t *H = &R->h[h];
    H->dlen[0] = isoline_offset_change(R, H);
    H->dlen[1] = H->tinfo[0] == ST_OK ? cycle_offset_change(R, H->tverts, H->tinfo[3]) : NAN;
    H->dlen[2] = H->rinfo[0] == ST_OK ? cycle_offset_change(R, H->rverts, H->rinfo[3]) : NAN;
  }
  /* outputs */
  R->out_layer = (int32_t *)malloc(sizeof(int32_t) * nv);
  R->out_phi = (double *)malloc(sizeof(double) * nv);
  for (int64_t v = 0; v < nv; ++v) {
    if (R->en[v] == 0) { R->out_layer[v] = 0; R->out_phi[v] = 0.0; }
    else if (R->en[v] == 1) { R->out_layer[v] = R->el[v * KM]; R->out_phi[v] = R->ex[v * KM]; }
    else { R->out_layer[v] = -1; R->out_phi[v] = R->ex[v * KM]; }
  }
  R->layers_out = (int32_t *)malloc(sizeof(int32_t) * 3 * (R->nl + 1));
  for (int32_t l = 1; l <= R->nl; ++l) {
    R->layers_out[3 * (l - 1)] = R->lbirth[l];
    R->layers_out[3 * (l - 1) + 1] = R->ldeath[l];
    R->layers_out[3 * (l - 1) + 2] = R->lst[l];
  }
  return R;
}

void orc_free(orc_run *R) {
  if (!R) return;
  free(R->X); free(R->F); free(R->rp); free(R->col); free(R->hface); free(R->Lv); free(R->Ld);
  free(R->en); free(R->el); free(R->ex); free(R->cover);
  free(R->lst); free(R->lbirth); free(R->ldeath); free(R->nodes); free(R->npos);
  for (int32_t i = 0; i < R->nh; ++i) {
    free(R->h[i].edges); free(R->h[i].verts); free(R->h[i].pts); free(R->h[i].tverts); free(R->h[i].arrival);
    free(R->h[i].rverts); free(R->h[i].spts[0]); free(R->h[i].spts[1]);
    free(R->h[i].tfa);
  }
  free(R->vn);
  free(R->h); free(R->out_layer); free(R->out_phi); free(R->rec); free(R->layers_out); free(R->stamp);
  free(R);
}

int32_t orc_status(const orc_run *r) { return r->status; }
int32_t orc_genus(const orc_run *r) { return r->genus; }
int32_t orc_steps(const orc_run *r) { return r->steps; }
const int64_t *orc_counters(const orc_run *r) { return r->cnt; }
const int32_t *orc_state_layer(const orc_run *r) { return r->out_layer; }
const double *orc_state_phi(const orc_run *r) { return r->out_phi; }
const int32_t *orc_cover(const orc_run *r) { return r->cover; }
const int64_t *orc_step_records(const orc_run *r, int32_t *n) { *n = r->nrec; return r->rec; }
int32_t orc_num_nodes(const orc_run *r) { return r->nn; }
const int32_t *orc_nodes(const orc_run *r) { return r->nodes; }
const double *orc_node_pos(const orc_run *r) { return r->npos; }
int32_t orc_num_layers(const orc_run *r) { return r->nl; }
const int32_t *orc_layers(const orc_run *r) { return r->layers_out; }
int32_t orc_num_handles(const orc_run *r) { return r->nh; }
const int32_t *orc_handle_info(const orc_run *r, int32_t h) { return r->h[h].info; }
const int32_t *orc_handle_edges(const orc_run *r, int32_t h) { return r->h[h].edges; }
const int32_t *orc_handle_verts(const orc_run *r, int32_t h) { return r->h[h].verts; }
const double *orc_handle_points(const orc_run *r, int32_t h) { return r->h[h].pts; }
double orc_handle_length(const orc_run *r, int32_t h) { return r->h[h].len; }
const int32_t *orc_tunnel_info(const orc_run *r, int32_t h) { return r->h[h].tinfo; }
const int32_t *orc_tunnel_verts(const orc_run *r, int32_t h) { return r->h[h].tverts; }
const int32_t *orc_tunnel_arrival(const orc_run *r, int32_t h) { return r->h[h].arrival; }
const double *orc_tunnel_arrival_time(const orc_run *r, int32_t h) { return r->h[h].tfa; }
const int32_t *orc_refined_info(const orc_run *r, int32_t h) { return r->h[h].rinfo; }
const int32_t *orc_refined_verts(const orc_run *r, int32_t h) { return r->h[h].rverts; }
const double *orc_loop_offset_change(const orc_run *r, int32_t h) { return r->h[h].dlen; }
int32_t orc_trace_streamline(const double *X, int64_t nv, const int32_t *F, int64_t nf, const double *tf,
                             const int32_t *cut_edges, int64_t ncut, int32_t start, double *pts, int64_t cap,
                             int64_t *n_out, int32_t *end_vertex) {
  orc_run *R = (orc_run *)calloc(1, sizeof(orc_run));
  R->nv = nv;
  R->nf = nf;
  int st = build_mesh(R, X, F);
  *n_out = 0;
  *end_vertex = -1;
  if (st == ST_OK && (start < 0 || start >= nv)) st = ST_EINVAL;
  char *cut = st == ST_OK ? (char *)calloc(R->nnz + 1, 1) : NULL;
  for (int64_t i = 0; st == ST_OK && i < ncut; ++i) {
    int64_t a = slot_of(R, cut_edges[2 * i], cut_edges[2 * i + 1]), b = slot_of(R, cut_edges[2 * i + 1], cut_edges[2 * i]);
    if (a < 0 || b < 0) { st = ST_EINVAL; break; }
    cut[a] = cut[b] = 1;
  }
  if (st == ST_OK) {
    double *sp = NULL;
    int64_t sn = 0;
    st = streamline(R, tf, cut, start, &sp, &sn, end_vertex);
    for (int64_t i = 0; i < sn && i < cap; ++i)
      for (int d = 0; d < 3; ++d) pts[3 * i + d] = sp[3 * i + d];
    *n_out = sn;
    free(sp);
  }
  free(cut);
  free(R->X); free(R->F); free(R->rp); free(R->col); free(R->hface); free(R->Lv); free(R->Ld);
  free(R);
  return st;
}
int32_t orc_streamline(const orc_run *r, int32_t h, int32_t kind, int64_t *n, double *len, const double **pts) {
  const handle_t *H = &r->h[h];
  *n = H->sn[kind];
  *len = H->slen[kind];
  *pts = H->spts[kind];
  return H->sst[kind];
}
double orc_mean_edge(const orc_run *r) { return r->mean_edge; }
