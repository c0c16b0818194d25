/*
 * meshgen.c -- seeded synthetic input generator (closed, oriented triangle meshes).
 *
 * Test and benchmark input generation only: this file holds none of the
 * loop-shrinking method's arithmetic.  Both the CPU oracle and the CUDA path
 * consume its meshes; neither is used here.
 *
 * Shapes (stand-ins for the paper's scanned models, Sec. 6 / Table 1):
 *   - parametric torus grid (u, v), each quad split along its (i,j)-(i+1,j+1) diagonal;
 *   - implicit solids polygonised by marching tetrahedra on the Kuhn (Freudenthal)
 *     six-tetrahedra split of every grid cube.  The split is face-consistent across
 *     cubes, so with no sample exactly on the iso-level the result is a closed
 *     2-manifold.  Triangle orientation is decided combinatorially (exact integer
 *     determinant on doubled edge midpoints), never from interpolated geometry.
 *     Fields: smooth union of z-axis tori ("tube chain"), Schwarz P and gyroid solids
 *     clipped to a cube, and a genus-0 union of capsules (branching shape).
 *   - normal jitter with Gaussian noise drawn from SplitMix64 + Box-Muller,
 *     rejecting any move that flips an incident face.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood 2014), u = (x >> 11) * 2^-53.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MG_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------ RNG */
MG_EXPORT uint64_t mg_splitmix64(uint64_t *state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
MG_EXPORT double mg_uniform(uint64_t *state) {
  return (double)(mg_splitmix64(state) >> 11) * (1.0 / 9007199254740992.0);
}
/* seed vertex for problem `seed` on a mesh with nv vertices: floor(U * nv) */
MG_EXPORT int32_t mg_seed_vertex(uint64_t seed, int64_t nv) {
  uint64_t st = seed;
  double u = mg_uniform(&st);
  int64_t v = (int64_t)floor(u * (double)nv);
  if (v >= nv) v = nv - 1;
  return (int32_t)v;
}

/* ---------------------------------------------------------------- torus */
MG_EXPORT void mg_torus(int32_t nu, int32_t nv, double R, double r, double *X, int32_t *F) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int32_t i = 0; i < nu; ++i)
    for (int32_t j = 0; j < nv; ++j) {
      double u = two_pi * i / nu, v = two_pi * j / nv;
      int64_t id = (int64_t)i * nv + j;
      X[3 * id + 0] = (R + r * cos(v)) * cos(u);
      X[3 * id + 1] = (R + r * cos(v)) * sin(u);
      X[3 * id + 2] = r * sin(v);
    }
  int64_t f = 0;
  for (int32_t i = 0; i < nu; ++i)
    for (int32_t j = 0; j < nv; ++j) {
      int32_t a = i * nv + j, b = ((i + 1) % nu) * nv + j;
      int32_t c = ((i + 1) % nu) * nv + (j + 1) % nv, d = i * nv + (j + 1) % nv;
      F[3 * f + 0] = a; F[3 * f + 1] = b; F[3 * f + 2] = c; ++f;
      F[3 * f + 0] = a; F[3 * f + 1] = c; F[3 * f + 2] = d; ++f;
    }
}

/* --------------------------------------------------------------- fields */
enum { MG_TUBE_CHAIN = 0, MG_SCHWARZ_P = 1, MG_GYROID = 2, MG_CAPSULES = 3, MG_SPHERE = 4 };

typedef struct {
  int kind;
  int count;        /* tube chain: number of tori; capsules: number of arms */
  double p[8];      /* shape parameters */
  double lo[3], hi[3];
} field_t;

static double torus_sdf(double x, double y, double z, double cx, double R, double r) {
  double qx = sqrt((x - cx) * (x - cx) + y * y) - R;
  return sqrt(qx * qx + z * z) - r;
}
static double smin(double a, double b, double k) {
  double h = 0.5 + 0.5 * (b - a) / k;
  if (h < 0) h = 0;
  if (h > 1) h = 1;
  return b * (1 - h) + a * h - k * h * (1 - h);
}
static double box_sdf(double x, double y, double z, const double *lo, const double *hi) {
  double c[3] = {(lo[0] + hi[0]) * 0.5, (lo[1] + hi[1]) * 0.5, (lo[2] + hi[2]) * 0.5};
  double e[3] = {(hi[0] - lo[0]) * 0.5, (hi[1] - lo[1]) * 0.5, (hi[2] - lo[2]) * 0.5};
  double q[3] = {fabs(x - c[0]) - e[0], fabs(y - c[1]) - e[1], fabs(z - c[2]) - e[2]};
  double m = q[0] > q[1] ? q[0] : q[1];
  m = m > q[2] ? m : q[2];
  double ox = q[0] > 0 ? q[0] : 0, oy = q[1] > 0 ? q[1] : 0, oz = q[2] > 0 ? q[2] : 0;
  double out = sqrt(ox * ox + oy * oy + oz * oz);
  return out + (m < 0 ? m : 0);
}
static double seg_sdf(double x, double y, double z, const double *a, const double *b, double r) {
  double pa[3] = {x - a[0], y - a[1], z - a[2]}, ba[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double h = (pa[0] * ba[0] + pa[1] * ba[1] + pa[2] * ba[2]) / (ba[0] * ba[0] + ba[1] * ba[1] + ba[2] * ba[2]);
  if (h < 0) h = 0;
  if (h > 1) h = 1;
  double d[3] = {pa[0] - ba[0] * h, pa[1] - ba[1] * h, pa[2] - ba[2] * h};
  return sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - r;
}

static double field_eval(const field_t *f, double x, double y, double z) {
  switch (f->kind) {
  case MG_TUBE_CHAIN: {
    /* p: R, r, spacing, blend k */
    double R = f->p[0], r = f->p[1], sp = f->p[2], k = f->p[3];
    double d = torus_sdf(x, y, z, 0.0, R, r);
    for (int i = 1; i < f->count; ++i) d = smin(d, torus_sdf(x, y, z, sp * i, R, r), k);
    return d;
  }
  case MG_SCHWARZ_P: {
    double v = cos(x) + cos(y) + cos(z);
    double b = box_sdf(x, y, z, f->p, f->p + 3);
    return v > b ? v : b;
  }
  case MG_GYROID: {
    double v = sin(x) * cos(y) + sin(y) * cos(z) + sin(z) * cos(x);
    double b = box_sdf(x, y, z, f->p, f->p + 3);
    return v > b ? v : b;
  }
  case MG_CAPSULES: {
    /* arms from the origin to points on a circle of radius p[0] tilted upwards, radius p[1], blend p[2] */
    const double two_pi = 6.283185307179586476925286766559;
    double o[3] = {0, 0, 0};
    double d = 1e30;
    for (int i = 0; i < f->count; ++i) {
      double ang = two_pi * i / f->count;
      double tip[3] = {f->p[0] * cos(ang), f->p[0] * sin(ang), 0.35 * f->p[0] * (i % 2 ? 1 : -1)};
      double di = seg_sdf(x, y, z, o, tip, f->p[1]);
      d = (i == 0) ? di : smin(d, di, f->p[2]);
    }
    return d;
  }
  case MG_SPHERE:
  default:
    return sqrt(x * x + y * y + z * z) - f->p[0];
  }
}

/* ------------------------------------------------------ edge -> vertex hash */
typedef struct {
  int64_t *keys;
  int32_t *vals;
  int64_t cap;
  int64_t n;
} hmap_t;

static uint64_t hmix(uint64_t x) {
  x ^= x >> 33; x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ull;
  return x ^ (x >> 33);
}
static int hmap_init(hmap_t *h, int64_t cap) {
  h->cap = cap; h->n = 0;
  h->keys = (int64_t *)malloc(sizeof(int64_t) * cap);
  h->vals = (int32_t *)malloc(sizeof(int32_t) * cap);
  if (!h->keys || !h->vals) return -1;
  for (int64_t i = 0; i < cap; ++i) h->keys[i] = -1;
  return 0;
}
static int hmap_grow(hmap_t *h);
/* returns slot of key, inserting with val=-1 if absent */
static int64_t hmap_slot(hmap_t *h, int64_t key) {
  if (2 * (h->n + 1) > h->cap) hmap_grow(h);
  int64_t i = (int64_t)(hmix((uint64_t)key) & (uint64_t)(h->cap - 1));
  while (h->keys[i] != -1 && h->keys[i] != key) i = (i + 1) & (h->cap - 1);
  if (h->keys[i] == -1) { h->keys[i] = key; h->vals[i] = -1; h->n++; }
  return i;
}
static int hmap_grow(hmap_t *h) {
  hmap_t g;
  if (hmap_init(&g, h->cap * 2)) return -1;
  for (int64_t i = 0; i < h->cap; ++i)
    if (h->keys[i] != -1) {
      int64_t s = hmap_slot(&g, h->keys[i]);
      g.vals[s] = h->vals[i];
    }
  free(h->keys); free(h->vals);
  *h = g;
  return 0;
}

/* ------------------------------------------------------------ mesh object */
typedef struct {
  double *X; int64_t nv, capv;
  int32_t *F; int64_t nf, capf;
} mg_mesh;

static int push_vertex(mg_mesh *m, double x, double y, double z) {
  if (m->nv == m->capv) {
    m->capv = m->capv ? m->capv * 2 : 1024;
    m->X = (double *)realloc(m->X, sizeof(double) * 3 * m->capv);
  }
  m->X[3 * m->nv] = x; m->X[3 * m->nv + 1] = y; m->X[3 * m->nv + 2] = z;
  return (int)(m->nv++);
}
static void push_face(mg_mesh *m, int32_t a, int32_t b, int32_t c) {
  if (m->nf == m->capf) {
    m->capf = m->capf ? m->capf * 2 : 2048;
    m->F = (int32_t *)realloc(m->F, sizeof(int32_t) * 3 * m->capf);
  }
  m->F[3 * m->nf] = a; m->F[3 * m->nf + 1] = b; m->F[3 * m->nf + 2] = c;
  m->nf++;
}

/* Polygonise field f < 0 on an n^3 sample grid spanning [lo, hi]. */
typedef struct {
  const field_t *f;
  int64_t n[3];
  double lo[3], h[3];
  double *plane[2]; /* samples of two consecutive z planes */
  hmap_t map;
  mg_mesh *m;
} mt_ctx;

static double sample_at(mt_ctx *c, int64_t i, int64_t j, int64_t k, int64_t kbase) {
  return c->plane[k - kbase][i * c->n[1] + j];
}

static int32_t edge_vertex(mt_ctx *c, const int64_t *p, const int64_t *q, double fp, double fq) {
  /* p is the lower corner; q = p + d with d in {0,1}^3 \ {0} */
  int64_t d = (q[0] - p[0]) | ((q[1] - p[1]) << 1) | ((q[2] - p[2]) << 2);
  int64_t key = ((p[2] * c->n[0] + p[0]) * c->n[1] + p[1]) * 8 + d;
  int64_t s = hmap_slot(&c->map, key);
  if (c->map.vals[s] >= 0) return c->map.vals[s];
  double t = fp / (fp - fq);
  if (t < 0.01) t = 0.01;
  if (t > 0.99) t = 0.99;
  double x = c->lo[0] + (p[0] + t * (q[0] - p[0])) * c->h[0];
  double y = c->lo[1] + (p[1] + t * (q[1] - p[1])) * c->h[1];
  double z = c->lo[2] + (p[2] + t * (q[2] - p[2])) * c->h[2];
  int32_t v = push_vertex(c->m, x, y, z);
  s = hmap_slot(&c->map, key); /* map may have grown */
  c->map.vals[s] = v;
  return v;
}

static int64_t det3(const int64_t *a, const int64_t *b, const int64_t *c) {
  return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
}

/* emit triangle on tet edges (e[0], e[1], e[2]), oriented so that the inside corner `pin` lies behind it */
static void emit_tri(mt_ctx *c, int64_t P[4][3], const double *fv, const int ea[3][2], int pin) {
  int64_t mid[3][3], w[3][3];
  int32_t vid[3];
  for (int t = 0; t < 3; ++t) {
    int a = ea[t][0], b = ea[t][1];
    for (int d = 0; d < 3; ++d) mid[t][d] = P[a][d] + P[b][d]; /* doubled midpoint */
    /* lower corner first for the weld key */
    const int64_t *lo = P[a], *hi = P[b];
    double flo = fv[a], fhi = fv[b];
    if (P[b][0] + P[b][1] + P[b][2] < P[a][0] + P[a][1] + P[a][2]) { lo = P[b]; hi = P[a]; flo = fv[b]; fhi = fv[a]; }
    vid[t] = edge_vertex(c, lo, hi, flo, fhi);
  }
  for (int d = 0; d < 3; ++d) {
    w[0][d] = mid[1][d] - mid[0][d];
    w[1][d] = mid[2][d] - mid[0][d];
    w[2][d] = 2 * P[pin][d] - mid[0][d];
  }
  int64_t s = det3(w[0], w[1], w[2]);
  if (s > 0) push_face(c->m, vid[0], vid[2], vid[1]);
  else push_face(c->m, vid[0], vid[1], vid[2]);
}

static void do_tet(mt_ctx *c, int64_t P[4][3], const double *fv) {
  int in[4], nin = 0;
  for (int t = 0; t < 4; ++t) { in[t] = fv[t] < 0; nin += in[t]; }
  if (nin == 0 || nin == 4) return;
  if (nin == 1 || nin == 3) {
    int apex = -1;
    for (int t = 0; t < 4; ++t)
      if (in[t] == (nin == 1)) apex = t;
    int o[3], k = 0;
    for (int t = 0; t < 4; ++t)
      if (t != apex) o[k++] = t;
    int ea[3][2] = {{apex, o[0]}, {apex, o[1]}, {apex, o[2]}};
    int pin = (nin == 1) ? apex : o[0];
    emit_tri(c, P, fv, ea, pin);
  } else {
    int I[2], O[2], ki = 0, ko = 0;
    for (int t = 0; t < 4; ++t) {
      if (in[t]) I[ki++] = t;
      else O[ko++] = t;
    }
    /* quad cycle: (I0,O0) (I0,O1) (I1,O1) (I1,O0) */
    int q0[2] = {I[0], O[0]}, q1[2] = {I[0], O[1]}, q2[2] = {I[1], O[1]}, q3[2] = {I[1], O[0]};
    int t1[3][2] = {{q0[0], q0[1]}, {q1[0], q1[1]}, {q2[0], q2[1]}};
    int t2[3][2] = {{q0[0], q0[1]}, {q2[0], q2[1]}, {q3[0], q3[1]}};
    emit_tri(c, P, fv, t1, I[0]);
    emit_tri(c, P, fv, t2, I[0]);
  }
}

static void fill_plane(mt_ctx *c, double *dst, int64_t k) {
  double z = c->lo[2] + k * c->h[2];
  for (int64_t i = 0; i < c->n[0]; ++i) {
    double x = c->lo[0] + i * c->h[0];
    for (int64_t j = 0; j < c->n[1]; ++j) {
      double y = c->lo[1] + j * c->h[1];
      double v = field_eval(c->f, x, y, z);
      if (fabs(v) < 1e-9) v = 1e-9; /* nudge: no sample exactly on the iso-level */
      dst[i * c->n[1] + j] = v;
    }
  }
}

static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

static mg_mesh *polygonise(const field_t *f, const int64_t *n) {
  mt_ctx c;
  memset(&c, 0, sizeof(c));
  c.f = f;
  for (int d = 0; d < 3; ++d) { c.n[d] = n[d]; c.lo[d] = f->lo[d]; c.h[d] = (f->hi[d] - f->lo[d]) / (double)(n[d] - 1); }
  c.plane[0] = (double *)malloc(sizeof(double) * n[0] * n[1]);
  c.plane[1] = (double *)malloc(sizeof(double) * n[0] * n[1]);
  c.m = (mg_mesh *)calloc(1, sizeof(mg_mesh));
  hmap_init(&c.map, 1 << 20);
  fill_plane(&c, c.plane[0], 0);
  for (int64_t k = 0; k + 1 < n[2]; ++k) {
    fill_plane(&c, c.plane[1], k + 1);
    for (int64_t i = 0; i + 1 < n[0]; ++i)
      for (int64_t j = 0; j + 1 < n[1]; ++j) {
        /* coordinate order (x=i, y=j, z=k) */
        for (int p = 0; p < 6; ++p) {
          int64_t P[4][3];
          double fv[4];
          int64_t cur[3] = {i, j, k};
          for (int t = 0; t < 4; ++t) {
            if (t > 0) cur[perms[p][t - 1]] += 1;
            P[t][0] = cur[0]; P[t][1] = cur[1]; P[t][2] = cur[2];
            fv[t] = sample_at(&c, cur[0], cur[1], cur[2], k);
          }
          do_tet(&c, P, fv);
        }
      }
    double *tmp = c.plane[0]; c.plane[0] = c.plane[1]; c.plane[1] = tmp;
  }
  free(c.plane[0]); free(c.plane[1]);
  free(c.map.keys); free(c.map.vals);
  return c.m;
}

/* ------------------------------------------------------------- jitter */
MG_EXPORT void mg_jitter(double *X, int64_t nv, const int32_t *F, int64_t nf, double sigma_rel, uint64_t seed) {
  if (sigma_rel <= 0) return;
  /* mean edge length (each undirected edge counted twice; ratio unaffected) */
  double sum = 0;
  for (int64_t f = 0; f < nf; ++f)
    for (int k = 0; k < 3; ++k) {
      const double *a = X + 3 * F[3 * f + k], *b = X + 3 * F[3 * f + (k + 1) % 3];
      sum += sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]));
    }
  double lmean = sum / (3.0 * nf);
  double sigma = sigma_rel * lmean;
  /* vertex -> incident faces */
  int64_t *off = (int64_t *)calloc(nv + 1, sizeof(int64_t));
  for (int64_t f = 0; f < 3 * nf; ++f) off[F[f] + 1]++;
  for (int64_t v = 0; v < nv; ++v) off[v + 1] += off[v];
  int32_t *inc = (int32_t *)malloc(sizeof(int32_t) * 3 * nf);
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * nv);
  memcpy(fill, off, sizeof(int64_t) * nv);
  for (int64_t f = 0; f < nf; ++f)
    for (int k = 0; k < 3; ++k) inc[fill[F[3 * f + k]]++] = (int32_t)f;
  uint64_t st = seed ^ 0xA5A5A5A5DEADBEEFull;
  for (int64_t v = 0; v < nv; ++v) {
    double n[3] = {0, 0, 0};
    double fn_old[64][3];
    int64_t deg = off[v + 1] - off[v];
    for (int64_t q = off[v]; q < off[v + 1]; ++q) {
      const int32_t *t = F + 3 * inc[q];
      const double *a = X + 3 * t[0], *b = X + 3 * t[1], *c = X + 3 * t[2];
      double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
      double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
      n[0] += cr[0]; n[1] += cr[1]; n[2] += cr[2];
      if (q - off[v] < 64) { fn_old[q - off[v]][0] = cr[0]; fn_old[q - off[v]][1] = cr[1]; fn_old[q - off[v]][2] = cr[2]; }
    }
    double u1 = mg_uniform(&st), u2 = mg_uniform(&st);
    if (deg > 64) continue;
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (nn == 0) continue;
    if (u1 < 1e-300) u1 = 1e-300;
    double g = sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
    double old[3] = {X[3 * v], X[3 * v + 1], X[3 * v + 2]};
    for (int d = 0; d < 3; ++d) X[3 * v + d] = old[d] + sigma * g * n[d] / nn;
    int ok = 1;
    for (int64_t q = off[v]; q < off[v + 1] && ok; ++q) {
      const int32_t *t = F + 3 * inc[q];
      const double *a = X + 3 * t[0], *b = X + 3 * t[1], *c = X + 3 * t[2];
      double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
      double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
      const double *o = fn_old[q - off[v]];
      if (cr[0] * o[0] + cr[1] * o[1] + cr[2] * o[2] <= 0) ok = 0;
    }
    if (!ok)
      for (int d = 0; d < 3; ++d) X[3 * v + d] = old[d];
  }
  free(off); free(inc); free(fill);
}

/* ------------------------------------------------------ exported builder */
MG_EXPORT mg_mesh *mg_implicit(int kind, int count, const double *params, int nparams, const double *lo,
                               const double *hi, const int64_t *n) {
  field_t f;
  memset(&f, 0, sizeof(f));
  f.kind = kind; f.count = count;
  for (int i = 0; i < nparams && i < 8; ++i) f.p[i] = params[i];
  for (int d = 0; d < 3; ++d) { f.lo[d] = lo[d]; f.hi[d] = hi[d]; }
  return polygonise(&f, n);
}
MG_EXPORT int64_t mg_mesh_nv(const mg_mesh *m) { return m->nv; }
MG_EXPORT int64_t mg_mesh_nf(const mg_mesh *m) { return m->nf; }
MG_EXPORT void mg_mesh_copy(const mg_mesh *m, double *X, int32_t *F) {
  memcpy(X, m->X, sizeof(double) * 3 * m->nv);
  memcpy(F, m->F, sizeof(int32_t) * 3 * m->nf);
}
MG_EXPORT void mg_mesh_free(mg_mesh *m) {
  if (!m) return;
  free(m->X); free(m->F); free(m);
}
