// refine.cu -- handle-refinement passes (Sec. 3.3) and the classification of loops by a normal
// offset (Sec. 3.5).
//
// Refinement.  The refined handle loop comes from the same single-layer pass as the tunnel loop
// (tunnel.cu), now started on one side of the tunnel loop with the tunnel loop as the only border:
// no restriction to a covered area (domain step INT32_MAX).  k_rprep turns each pass's tunnel
// cycle into the pass's border-edge list, which the tunnel-pass kernels then use as they use a
// handle loop's crossing edges:
//   1. the cycle is made simple by erasing its closed sub-loops in order along it from its first
//      vertex (the tunnel cycle crosses its handle loop once, on the closing edge, which the
//      erasure keeps; an erased sub-loop never crosses it);
//   2. border edges: from each cycle vertex c_i, the edges to the neighbours on its right -- those
//      met counter-clockwise from c_{i-1} to c_{i+1} around c_i (faces are counter-clockwise),
//      chords to other cycle vertices left out -- in cycle order, each vertex's in that sweep
//      order.  Inside endpoints (sources, held at 1): the cycle vertices; outside endpoints: their
//      right neighbours, which the pass reaches only around the handle.
// The trace from the first far-side vertex reached, closed along the cycle, is the refined loop.
//
// Classification.  A loop is offset along the unit vertex normals by a fraction of its mesh's
// mean edge length and its length compared with the original's: tunnel loops sit in saddle-shaped
// parts and shrink, handle loops grow.  Unit vertex normal: the sum, in the vertex's CSR order, of
// the (twice area-weighted) normals of the faces holding its outgoing half-edges, normalised; an
// isoline point on edge (a, b) takes the normalised sum of a's and b's normals.
#include "vls_batch.cuh"

namespace vls {
namespace {

// neighbour that follows u counter-clockwise around c: the third vertex of the face left of c->u
__device__ __forceinline__ int32_t next_ccw(const Dev &d, int32_t c, int32_t u) {
  const int32_t k = slot_of(d.rp, d.col, c, u);
  if (k < 0) return -1;
  const int32_t *t = d.F + 3 * (int64_t)d.hface[k];
  const int32_t a = t[0], b = t[1], e = t[2];
  return (a != c && a != u) ? a : (b != c && b != u) ? b : e;
}

// face normal (b - a) x (c - a), each product and difference rounded alone
__device__ __forceinline__ void face_normal(const Dev &d, int32_t f, double n[3]) {
  const int32_t *t = d.F + 3 * (int64_t)f;
  const double *a = d.X + 3 * (int64_t)t[0], *b = d.X + 3 * (int64_t)t[1], *c = d.X + 3 * (int64_t)t[2];
  const double u0 = dsub(b[0], a[0]), u1 = dsub(b[1], a[1]), u2 = dsub(b[2], a[2]);
  const double w0 = dsub(c[0], a[0]), w1 = dsub(c[1], a[1]), w2 = dsub(c[2], a[2]);
  n[0] = dsub(dmul(u1, w2), dmul(u2, w1));
  n[1] = dsub(dmul(u2, w0), dmul(u0, w2));
  n[2] = dsub(dmul(u0, w1), dmul(u1, w0));
}

__device__ __forceinline__ double dist3(const double p[3], const double q[3]) {
  const double dx = dsub(q[0], p[0]), dy = dsub(q[1], p[1]), dz = dsub(q[2], p[2]);
  return dsqrt(dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz)));
}

// unit vertex normals and, per vertex, the lengths of its edges to larger ids (for the mean)
__global__ void k_vnormals(Dev d, double *vn, double *elen) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < d.V; v += gridDim.x * blockDim.x) {
    double n[3] = {0.0, 0.0, 0.0}, es = 0.0;
    const double *xv = d.X + 3 * (int64_t)v;
    for (int32_t k = d.rp[v]; k < d.rp[v + 1]; ++k) {
      double g[3];
      face_normal(d, d.hface[k], g);
      n[0] = dadd(n[0], g[0]);
      n[1] = dadd(n[1], g[1]);
      n[2] = dadd(n[2], g[2]);
      const int32_t u = d.col[k];
      if (u > v) es = dadd(es, dist3(xv, d.X + 3 * (int64_t)u));
    }
    const double len = dsqrt(dadd(dadd(dmul(n[0], n[0]), dmul(n[1], n[1])), dmul(n[2], n[2])));
    for (int c = 0; c < 3; ++c) vn[3 * (int64_t)v + c] = len > 0.0 ? ddiv(n[c], len) : 0.0;
    elen[v] = es;
  }
}

// block-wide sum (every thread calls; the result is valid in every thread)
__device__ double block_sum(double x) {
  __shared__ double part[32];
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) part[w] = x;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += part[i];
  return s;
}

// mean edge length of each problem: one block per problem, a fixed summation order
__global__ void k_mean_edge(Dev d, const double *elen, double *pmedge) {
  for (int32_t p = blockIdx.x; p < d.P; p += gridDim.x) {
    const int32_t v0 = d.voff[p], v1 = d.voff[p + 1];
    double s = 0.0;
    for (int32_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) s += elen[v];
    s = block_sum(s);
    if (threadIdx.x == 0) {
      int64_t ne = (int64_t)(d.rp[v1] - d.rp[v0]) / 2;
      pmedge[p] = ne > 0 ? s / (double)ne : 0.0;
    }
  }
}

// length change of a closed polyline of n points under the normal offset; point i = pt(i, p, nrm)
template <class PT> __device__ double offset_change(int32_t n, double del, PT pt) {
  double l0 = 0.0, l1 = 0.0;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    double p[3], q[3], np[3], nq[3];
    pt(i, p, np);
    pt(i + 1 < n ? i + 1 : 0, q, nq);
    double po[3], qo[3];
    for (int c = 0; c < 3; ++c) {
      po[c] = dadd(p[c], dmul(del, np[c]));
      qo[c] = dadd(q[c], dmul(del, nq[c]));
    }
    l0 += dist3(p, q);
    l1 += dist3(po, qo);
  }
  l0 = block_sum(l0);
  l1 = block_sum(l1);
  return l1 - l0;
}

// handle (isoline) loops: one block per handle
__global__ void k_classify_iso(Dev d, Params P, const double *vn, const double *pmedge, double *hdl, int32_t nh) {
  for (int32_t h = blockIdx.x; h < nh; h += gridDim.x) {
    const int32_t off = d.hoff[h], n = d.hn[h];
    const double del = dmul(P.offset, pmedge[d.hprob[h]]);
    auto pt = [&](int32_t i, double p[3], double nn[3]) {
      const int64_t e = off + i;
      const int32_t a = d.hedge[2 * e], b = d.hedge[2 * e + 1];
      double s[3];
      for (int c = 0; c < 3; ++c) {
        p[c] = d.hpts[3 * e + c];
        s[c] = dadd(vn[3 * (int64_t)a + c], vn[3 * (int64_t)b + c]);
      }
      const double len = dsqrt(dadd(dadd(dmul(s[0], s[0]), dmul(s[1], s[1])), dmul(s[2], s[2])));
      for (int c = 0; c < 3; ++c) nn[c] = len > 0.0 ? ddiv(s[c], len) : 0.0;
    };
    const double r = n >= 2 ? offset_change(n, del, pt) : __longlong_as_double(0x7ff8000000000000LL);
    if (threadIdx.x == 0) hdl[h] = r;
  }
}

// the vertex cycles of a chunk of passes (tunnel or refined loops): one block per pass
__global__ void k_classify_cyc(Dev d, TDev T, Params P, const double *vn, const double *pmedge) {
  for (int32_t q = blockIdx.x; q < T.NP; q += gridDim.x) {
    const int32_t p = T.pprob[q], voff = d.voff[p];
    const int32_t n = T.qstatus[q] == VLS_OK ? T.tvn[q] : 0;
    const int32_t *cyc = T.tverts + T.tvoff[q];
    const double del = dmul(P.offset, pmedge[p]);
    auto pt = [&](int32_t i, double x[3], double nn[3]) {
      const int64_t v = voff + cyc[i];
      for (int c = 0; c < 3; ++c) {
        x[c] = d.X[3 * v + c];
        nn[c] = vn[3 * v + c];
      }
    };
    const double r = n >= 2 ? offset_change(n, del, pt) : __longlong_as_double(0x7ff8000000000000LL);
    if (threadIdx.x == 0) T.qdl[q] = r;
  }
}

// Refinement set-up, one block per pass: simple cycle, then its right-side border edges into the
// pass's stretch of xedge (capacity xcap[q] edges); T.hen / T.pcn receive the counts.  Scratch:
// the pass's stretch of T.path (cycle position of a vertex, checked against the cycle before use:
// the stretch is not cleared) and of T.onew (per-vertex edge counts and their prefix sums).
__global__ void __launch_bounds__(256) k_rprep(Dev d, TDev T, int32_t *cyc_pool, const int32_t *coff,
                                               const int32_t *clen, int32_t *xedge, const int32_t *xcap,
                                               int32_t *hen, int32_t *pcn) {
  __shared__ int32_t n_s;
  __shared__ int32_t part[256];
  const int32_t q = blockIdx.x;
  if (q >= T.NP) return;
  const int32_t p = T.pprob[q], voff = d.voff[p], base = T.pbase[q];
  const int32_t nvp = d.voff[p + 1] - voff;
  int32_t *cyc = cyc_pool + coff[q];
  int32_t *pos = T.path + base;
  int32_t *cnt = reinterpret_cast<int32_t *>(T.onew) + 2 * (int64_t)base; // 2 nvp ints
  if (threadIdx.x == 0) {
    // loop erasure in place (the kept prefix never passes the read position)
    int32_t n = 0;
    const int32_t k = clen[q];
    for (int32_t i = 0; i < k; ++i) {
      const int32_t v = cyc[i];
      const int32_t lv = v - voff;
      if (lv < 0 || lv >= nvp) { n = 0; break; }
      const int32_t j = pos[lv];
      if (j >= 0 && j < n && cyc[j] == v) n = j + 1; // v closes a sub-loop: erase it
      else {
        cyc[n] = v;
        pos[lv] = n;
        ++n;
      }
    }
    n_s = n;
  }
  __syncthreads();
  const int32_t n = n_s;
  if (n < 3) {
    if (threadIdx.x == 0) { hen[q] = 0; pcn[q] = 0; }
    return;
  }
  auto on_cycle = [&](int32_t u) {
    const int32_t lu = u - voff;
    if (lu < 0 || lu >= nvp) return false;
    const int32_t j = pos[lu];
    return j >= 0 && j < n && cyc[j] == u;
  };
  // right-side neighbours of each cycle vertex: counted, scanned, written in sweep order
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int32_t c = cyc[i], prv = cyc[i > 0 ? i - 1 : n - 1], nxt = cyc[i + 1 < n ? i + 1 : 0];
    const int32_t deg = d.rp[c + 1] - d.rp[c];
    int32_t u = prv, m = 0;
    for (int32_t g = 0; g < deg; ++g) {
      u = next_ccw(d, c, u);
      if (u < 0 || u == nxt) break;
      if (!on_cycle(u)) ++m;
    }
    cnt[i] = m;
  }
  __syncthreads();
  // exclusive scan of cnt[0, n): contiguous chunks per thread
  const int32_t per = (n + blockDim.x - 1) / blockDim.x;
  const int32_t b0 = threadIdx.x * per, b1 = min(b0 + per, n);
  int32_t s = 0;
  for (int32_t i = b0; i < b1; ++i) s += cnt[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t run = 0;
    for (int32_t t = 0; t < (int32_t)blockDim.x; ++t) {
      const int32_t x = part[t];
      part[t] = run;
      run += x;
    }
    const int32_t tot = run <= xcap[q] ? run : 0; // the capacity covers every sweep (checked)
    hen[q] = tot;
    pcn[q] = 2 * tot;
  }
  __syncthreads();
  int32_t o = part[threadIdx.x];
  for (int32_t i = b0; i < b1; ++i) {
    const int32_t x = cnt[i];
    cnt[i] = o;
    o += x;
  }
  __syncthreads();
  if (hen[q] == 0) return;
  int32_t *xe = xedge + 2 * (int64_t)T.heoff[q];
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int32_t c = cyc[i], prv = cyc[i > 0 ? i - 1 : n - 1], nxt = cyc[i + 1 < n ? i + 1 : 0];
    const int32_t deg = d.rp[c + 1] - d.rp[c];
    int32_t u = prv, w = cnt[i];
    for (int32_t g = 0; g < deg; ++g) {
      u = next_ccw(d, c, u);
      if (u < 0 || u == nxt) break;
      if (on_cycle(u)) continue;
      xe[2 * (int64_t)w] = c;
      xe[2 * (int64_t)w + 1] = u;
      ++w;
    }
  }
}

}  // namespace

cudaError_t launch_vnormals(Batch &b, double *vn, double *elen, double *pmedge) {
  k_vnormals<<<b.sm_count * 4, 256, 0, b.st>>>(b.d, vn, elen); VLS_LAUNCH(b);
  k_mean_edge<<<b.P < 1024 ? b.P : 1024, 256, 0, b.st>>>(b.d, elen, pmedge); VLS_LAUNCH(b);
  return cudaGetLastError();
}

cudaError_t launch_classify_handles(Batch &b, const double *vn, const double *pmedge, double *hdl, int32_t nh) {
  if (nh <= 0) return cudaSuccess;
  k_classify_iso<<<nh < 4096 ? nh : 4096, 128, 0, b.st>>>(b.d, b.prm, vn, pmedge, hdl, nh); VLS_LAUNCH(b);
  return cudaGetLastError();
}

cudaError_t launch_classify_passes(Batch &b, const TDev &T, cudaStream_t st, const double *vn, const double *pmedge) {
  if (T.NP <= 0) return cudaSuccess;
  k_classify_cyc<<<T.NP < 4096 ? T.NP : 4096, 128, 0, st>>>(b.d, T, b.prm, vn, pmedge); VLS_LAUNCH(b);
  return cudaGetLastError();
}

cudaError_t launch_refine_prep(Batch &b, const TDev &T, cudaStream_t st, int32_t *cyc_pool, const int32_t *coff,
                               const int32_t *clen, int32_t *xedge, const int32_t *xcap, int32_t *hen, int32_t *pcn) {
  if (T.NP <= 0) return cudaSuccess;
  k_rprep<<<T.NP, 256, 0, st>>>(b.d, T, cyc_pool, coff, clen, xedge, xcap, hen, pcn); VLS_LAUNCH(b);
  return cudaGetLastError();
}

}  // namespace vls
