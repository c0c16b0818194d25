// events.cu -- front events of the initial pass (Sec. 3.1) and Reeb-graph nodes (Sec. 5).
//
// Merge: a vertex holding several layers after the update joins those layers (union-find
// over layer ids); each group of m layers yields m - 1 handle loops -- the theta-isolines of
// the involved fronts before merging, the one with the most crossing edges left out -- and
// one new layer holding, per vertex, the sum of the members' values (ascending layer order).
// Split: a live layer whose narrow band (0 < phi < 1) has c >= 2 components (union-find over
// band vertices, canonical label = smallest vertex) moves component i (in label order) to a
// new layer; its phi = 1 plateau keeps the old id, which becomes DEAD (frozen).
// Extinction: a live layer without band ends.
// Node positions: mean of the involved narrow band (Sec. 5); an end node uses the vertices of
// the layer updated in its last step.
#include "vls_batch.cuh"

namespace vls {

namespace {

// value of layer l at u as seen by the isoline of l: the layer's value, 1 on a frozen plateau
__device__ __forceinline__ double psi_iso(const Dev &d, int32_t u, int32_t l) {
  const int32_t m = d.multi[u];
  if (m >= 0) {
    const int32_t n = d.onl[m];
    for (int q = 0; q < n; ++q)
      if (d.olay[(int64_t)m * KMAX + q] == l) return d.ophi[(int64_t)m * KMAX + q];
    return 0.0;
  }
  const int32_t lu = d.lay[u];
  if (lu == 0) return 0.0;
  if (frozen_state(d.lstate[lu])) return 1.0;
  return lu == l ? ph_ld(d, u) : 0.0;
}
__device__ __forceinline__ bool holds(const Dev &d, int32_t u, int32_t l) {
  const int32_t m = d.multi[u];
  if (m >= 0) {
    const int32_t n = d.onl[m];
    for (int q = 0; q < n; ++q)
      if (d.olay[(int64_t)m * KMAX + q] == l) return true;
    return false;
  }
  return d.lay[u] == l;
}
__device__ __forceinline__ bool in_band_of(const Dev &d, int32_t u, int32_t l) {
  const int32_t m = d.multi[u];
  if (m >= 0) {
    const int32_t n = d.onl[m];
    for (int q = 0; q < n; ++q)
      if (d.olay[(int64_t)m * KMAX + q] == l) {
        const double x = d.ophi[(int64_t)m * KMAX + q];
        return x > 0.0 && x < 1.0;
      }
    return false;
  }
  if (d.lay[u] != l) return false;
  return ph_band(d, u);
}

// block-wide FP64 sum of three coordinates and a count
__device__ void block_sum3(double *v, int32_t cnt, double *out, int32_t *outc) {
  __shared__ double s[3][32];
  __shared__ int32_t sc[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    for (int c = 0; c < 3; ++c) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
    cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  }
  if (lane == 0) {
    for (int c = 0; c < 3; ++c) s[c][wid] = v[c];
    sc[wid] = cnt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[3] = {0.0, 0.0, 0.0};
    int32_t tc = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      for (int c = 0; c < 3; ++c) t[c] += s[c][w];
      tc += sc[w];
    }
    for (int c = 0; c < 3; ++c) out[c] = t[c];
    *outc = tc;
  }
  __syncthreads();
}

__device__ int32_t new_node(Dev &d, int32_t p, int32_t kind, int32_t step) {
  const int32_t g = atomicAdd(d.nnodes, 1);
  if (g >= d.ncap) { atomicCAS(&d.pstatus[p], 0, (int32_t)VLS_ELAYERS); return -1; }
  d.nkind[g] = kind;
  d.nstep[g] = step;
  d.nprob[g] = p;
  d.nlocal[g] = d.pnodes[p]++;
  return g;
}
__device__ int32_t new_layer(Dev &d, int32_t p, int32_t birth_local) {
  const int32_t loc = ++d.lcount[p];
  if (loc >= d.lcap[p]) { atomicCAS(&d.pstatus[p], 0, (int32_t)VLS_ELAYERS); return 0; }
  const int32_t l = d.lbase[p] + loc;
  d.lstate[l] = L_ALIVE;
  d.lbirth[l] = birth_local;
  d.ldeath[l] = -1;
  d.lfwd[l] = 0;
  d.lprob[l] = p;
  return l;
}

// ------------------------------------------------------------------ merge groups
// One thread: the collision rows of a step are few.  `luf` is a union-find parent array over
// global layer ids (-1 = untouched), reset to -1 for every layer it touched before returning.
// The groups of a step are resolved in rounds of at most MAX_TRACES traced layers, in the order
// of their smallest member (the oracle's order): a round skips the ctl[CTL_MSKIP] groups of the
// earlier rounds, takes groups while their traces fit, and asks for another round (H.mround)
// when groups are left.  Groups are disjoint sets of layers, so resolving one does not change
// another's traces, band or values.
__global__ void k_merge_groups(Dev d, int32_t *luf, int32_t *touched, Handles H) {
  if (threadIdx.x != 0) return;
  const int32_t t = d.ctl[CTL_T];
  const int32_t nc = *d.ncoll;
  const int32_t skip = d.ctl[CTL_MSKIP];
  *d.ngroups = 0;
  *d.ntrace = 0;
  if (nc == 0) {
    d.ctl[CTL_MSKIP] = 0;
    if (H.use) cudaGraphSetConditional(H.mround, 0u);
    return;
  }
  int32_t nt = 0;
  for (int32_t c = 0; c < nc; ++c) {
    const int32_t row = d.coll[c];
    const int32_t n = d.onl[row];
    for (int q = 0; q < n; ++q) {
      const int32_t l = d.olay[(int64_t)row * KMAX + q];
      if (luf[l] < 0) { luf[l] = l; touched[nt++] = l; }
    }
    const int32_t l0 = d.olay[(int64_t)row * KMAX];
    for (int q = 1; q < n; ++q) {
      int32_t a = l0, b = d.olay[(int64_t)row * KMAX + q];
      while (luf[a] != a) a = luf[a];
      while (luf[b] != b) b = luf[b];
      if (a != b) {
        if (a < b) luf[b] = a;
        else luf[a] = b;
      }
    }
  }
  // ascending layer order
  for (int32_t i = 1; i < nt; ++i) {
    int32_t x = touched[i], j = i - 1;
    while (j >= 0 && touched[j] > x) { touched[j + 1] = touched[j]; --j; }
    touched[j + 1] = x;
  }
  int32_t ng = 0, ntr = 0, gi = 0;
  bool more = false;
  for (int32_t i = 0; i < nt; ++i) {
    const int32_t r = touched[i];
    int32_t root = r;
    while (luf[root] != root) root = luf[root];
    if (root != r) continue; // groups are opened at their smallest member (the root)
    if (gi++ < skip) continue; // resolved by an earlier round of this step
    const int32_t p = d.lprob[r];
    if (ng >= MAX_TRACES) { more = true; break; }
    int32_t nm = 0;
    for (int32_t j = i; j < nt; ++j) {
      int32_t x = touched[j];
      while (luf[x] != x) x = luf[x];
      if (x == r) {
        if (nm < MAX_GROUP) d.gmem[ng * MAX_GROUP + nm] = touched[j];
        ++nm;
      }
    }
    if (nm > MAX_GROUP) { atomicCAS(&d.pstatus[p], 0, (int32_t)VLS_ELAYERS); continue; }
    if (ntr + nm > MAX_TRACES) { more = true; break; } // the next round takes this group first
    d.gprob[ng] = p;
    d.gnmem[ng] = nm;
    d.gnode[ng] = new_node(d, p, N_MERGE, t);
    d.gnew[ng] = 0; // assigned at finish, after the node (creation order of the oracle)
    for (int32_t j = 0; j < nm; ++j) {
      d.tgroup[ntr] = ng;
      d.tlayer[ntr] = d.gmem[ng * MAX_GROUP + j];
      ++ntr;
    }
    d.pev[3 * p + 0]++;
    ++ng;
  }
  for (int32_t i = 0; i < nt; ++i) luf[touched[i]] = -1;
  *d.ngroups = ng;
  *d.ntrace = ntr;
  // groups failed for size (more than MAX_GROUP layers) count as resolved
  d.ctl[CTL_MSKIP] = more ? gi - 1 : 0;
  if (H.use) cudaGraphSetConditional(H.mround, more ? 1u : 0u);
}

// ------------------------------------------------------------------ isoline trace
// One block per traced layer.  Crossing edges (a, b): psi(a) >= theta > psi(b), an endpoint
// holding the layer; every such edge has an endpoint among this step's frontier rows.
// Successor of (a, b): the other crossing edge of the face holding half-edge a -> b (the
// face on its left); components are cycles of the successor map.  The largest component
// (ties: smallest first edge in (a, b) order) is ordered from its smallest edge.
__global__ void __launch_bounds__(1024) k_trace(Dev d, Params P) {
  const int32_t tb = blockIdx.x;
  if (tb >= *d.ntrace) return;
  const int32_t t = d.ctl[CTL_T], cur = t & 1;
  const int32_t g = d.tgroup[tb], l = d.tlayer[tb], p = d.gprob[g];
  const double th = P.theta;
  unsigned long long *key = d.tkey + (int64_t)tb * TRACE_CAP;
  int32_t *slot = d.tslot + (int64_t)tb * TRACE_CAP;
  int32_t *succ = d.tsucc + (int64_t)tb * TRACE_CAP;
  int32_t *par = d.tpar + (int64_t)tb * TRACE_CAP;
  int32_t *rank = d.trank + (int64_t)tb * 2 * TRACE_CAP;
  int32_t *nxt = d.tnext + (int64_t)tb * 2 * TRACE_CAP;
  int32_t *ord = d.tord + (int64_t)tb * TRACE_CAP;
  __shared__ int32_t n;
  __shared__ unsigned long long best;
  if (threadIdx.x == 0) { n = 0; best = 0ull; }
  __syncthreads();
  // this problem's frontier rows (the isoline of l lies in their closed neighbourhood)
  const int32_t *__restrict__ seg = d.fseg[cur] + d.voff[p];
  const int32_t ns = d.pfront[(size_t)cur * d.P + p];
  for (int32_t j = threadIdx.x; j < ns; j += blockDim.x) {
    const int32_t v = seg[j];
    const double pv = psi_iso(d, v, l);
    const bool hv = holds(d, v, l);
    for (int32_t k = d.rp[v]; k < d.rp[v + 1]; ++k) {
      const int32_t u = d.col[k];
      const double pu = psi_iso(d, u, l);
      const bool hu = holds(d, u, l);
      if (!(hv || hu)) continue;
      int32_t a = -1, b = -1, s = -1;
      if (pv >= th && pu < th) { a = v; b = u; s = k; }
      else if (pu >= th && pv < th && d.fmark[u] != t) { a = u; b = v; s = slot_of(d.rp, d.col, u, v); }
      if (a < 0) continue;
      const int32_t idx = atomicAdd(&n, 1);
      if (idx < TRACE_CAP && VCHK(d.err, s, d.nnz, 201)) {
        key[idx] = ((unsigned long long)(uint32_t)a << 32) | (uint32_t)b;
        slot[idx] = s;
      }
    }
  }
  __syncthreads();
  const int32_t N = n < TRACE_CAP ? n : TRACE_CAP;
  if (n > TRACE_CAP && threadIdx.x == 0) atomicCAS(&d.pstatus[p], 0, (int32_t)VLS_ELAYERS);
  if (N == 0) {
    if (threadIdx.x == 0) d.tlen[tb] = 0;
    return;
  }
  // bitonic sort of (key, slot) over the next power of two
  int32_t M = 1;
  while (M < N) M <<= 1;
  for (int32_t i = N + threadIdx.x; i < M; i += blockDim.x) { key[i] = ~0ull; slot[i] = -1; }
  __syncthreads();
  for (int32_t k = 2; k <= M; k <<= 1)
    for (int32_t j = k >> 1; j > 0; j >>= 1) {
      for (int32_t i = threadIdx.x; i < M; i += blockDim.x) {
        const int32_t ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const unsigned long long a = key[i], b = key[ixj];
          if ((a > b) == up) {
            key[i] = b; key[ixj] = a;
            const int32_t s = slot[i]; slot[i] = slot[ixj]; slot[ixj] = s;
          }
        }
      }
      __syncthreads();
    }
  // drop repeated keys (sorted: keep the first of each run), compacted through scratch
  {
    __shared__ int32_t csum[1024];
    unsigned long long *tk = reinterpret_cast<unsigned long long *>(rank); // 2 * TRACE_CAP int32 = TRACE_CAP u64
    int32_t *ts = nxt;
    const int32_t per = (N + blockDim.x - 1) / blockDim.x;
    const int32_t beg = threadIdx.x * per, end = min(beg + per, N);
    int32_t cnt = 0;
    for (int32_t e = beg; e < end; ++e) cnt += (e == 0 || key[e] != key[e - 1]);
    csum[threadIdx.x] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t run = 0;
      for (int32_t i = 0; i < (int32_t)blockDim.x; ++i) { const int32_t c = csum[i]; csum[i] = run; run += c; }
      n = run;
    }
    __syncthreads();
    int32_t o = csum[threadIdx.x];
    for (int32_t e = beg; e < end; ++e)
      if (e == 0 || key[e] != key[e - 1]) { tk[o] = key[e]; ts[o] = slot[e]; ++o; }
    __syncthreads();
    if (threadIdx.x == 0 && n != N) (void)VCHK(d.err, -1, 0, 205); // records that duplicates were seen
    const int32_t U = n;
    for (int32_t e = threadIdx.x; e < U; e += blockDim.x) { key[e] = tk[e]; slot[e] = ts[e]; }
    __syncthreads();
  }
  const int32_t U = n;
  // successor through the face on the left of a -> b
  for (int32_t e = threadIdx.x; e < U; e += blockDim.x) {
    const int32_t a = (int32_t)(key[e] >> 32), b = (int32_t)(key[e] & 0xffffffffull);
    succ[e] = -1;
    par[e] = e;
    if (!VCHK(d.err, slot[e], d.nnz, 202)) continue;
    const int32_t *tri = d.F + 3 * (int64_t)d.hface[slot[e]];
    int32_t c = -1;
    for (int q = 0; q < 3; ++q)
      if (tri[q] != a && tri[q] != b) c = tri[q];
    if (!VCHK(d.err, c, d.V, 203)) continue;
    unsigned long long want;
    if (psi_iso(d, c, l) >= th) want = ((unsigned long long)(uint32_t)c << 32) | (uint32_t)b;
    else want = ((unsigned long long)(uint32_t)a << 32) | (uint32_t)c;
    int32_t lo = 0, hi = U - 1, j = -1;
    while (lo <= hi) {
      const int32_t m = (lo + hi) >> 1;
      if (key[m] == want) { j = m; break; }
      if (key[m] < want) lo = m + 1;
      else hi = m - 1;
    }
    succ[e] = j;
  }
  __syncthreads();
  for (int32_t e = threadIdx.x; e < U; e += blockDim.x)
    if (succ[e] >= 0) uf_unite(par, e, succ[e]);
  __syncthreads();
  // component labels (root = smallest edge index) into ord[]: writing them back into par[]
  // would race with other threads' path halving, which may re-point an entry at an ancestor
  int32_t *lab = ord;
  for (int32_t e = threadIdx.x; e < U; e += blockDim.x) {
    lab[e] = uf_find(par, e);
    nxt[e] = 0;
    rank[e] = -1;
  }
  __syncthreads();
  // component sizes (nxt as counters), best = (size, smallest root); predecessors in rank[]
  for (int32_t e = threadIdx.x; e < U; e += blockDim.x) {
    atomicAdd(&nxt[lab[e]], 1);
    if (succ[e] >= 0) rank[succ[e]] = e;
  }
  __syncthreads();
  for (int32_t e = threadIdx.x; e < U; e += blockDim.x)
    if (lab[e] == e) {
      const unsigned long long pk = ((unsigned long long)(uint32_t)nxt[e] << 32) | (uint32_t)(0xffffffffu - (uint32_t)e);
      atomicMax(&best, pk);
    }
  __syncthreads();
  // ordered walk from the component's smallest edge along the successors; an open chain is
  // completed backwards from the start (one thread: a loop is a few hundred edges)
  __syncthreads();
  if (threadIdx.x == 0) {
    const int32_t root = (int32_t)(0xffffffffu - (uint32_t)(best & 0xffffffffull));
    const int32_t size = (int32_t)(best >> 32);
    int32_t m = 0, cur = root;
    bool closed = false;
    while (m < size) {
      ord[m++] = cur;
      cur = succ[cur];
      if (cur == root) { closed = true; break; }
      if (cur < 0) break;
    }
    if (!closed) {
      int32_t nb = 0, back = rank[root];
      int32_t *tmp = nxt;
      while (back >= 0 && nb + m < size) { tmp[nb++] = back; back = rank[back]; }
      for (int32_t i = m - 1; i >= 0; --i) ord[nb + i] = ord[i];
      for (int32_t i = 0; i < nb; ++i) ord[i] = tmp[nb - 1 - i];
      m += nb;
    }
    d.tlen[tb] = m;
    d.tcount[tb] = U;
  }
}

// ------------------------------------------------------------------ merge finish
// One block per problem that merges this step (the block of the problem's first group): its
// groups in order, so layer ids, Reeb nodes and handle loops of a problem are created in the same
// order as by the oracle; problems proceed in parallel.
__global__ void __launch_bounds__(1024) k_merge_finish(Dev d, Params P) {
  const int32_t ng = *d.ngroups;
  const int32_t b0 = blockIdx.x;
  if (b0 >= ng) return;
  const int32_t pb = d.gprob[b0];
  for (int32_t h = 0; h < b0; ++h)
    if (d.gprob[h] == pb) return; // an earlier block owns this problem
  const int32_t t = d.ctl[CTL_T], cur = t & 1;
  const int32_t *__restrict__ fv = d.front[cur];
  const int32_t ntr = *d.ntrace;
  const double th = P.theta;
  __shared__ int32_t s_first, s_drop, s_eoff, s_hidx, s_N, s_nodeloc;
  __shared__ double s_pos[3];
  __shared__ int32_t s_cnt;
  for (int32_t g = b0; g < ng; ++g) {
    const int32_t p = d.gprob[g];
    if (p != pb) continue;
    const int32_t nm = d.gnmem[g];
    const int32_t *mem = d.gmem + g * MAX_GROUP;
    if (threadIdx.x == 0) {
      int32_t first = -1;
      for (int32_t i = 0; i < ntr; ++i)
        if (d.tgroup[i] == g) { first = i; break; }
      if (!VCHK(d.err, first, ntr, 210)) first = 0;
      s_first = first;
      int32_t drop = 0;
      for (int32_t i = 0; i < nm; ++i)
        if (d.tlen[first + i] >= d.tlen[first + drop]) drop = i; // most crossing edges, ties -> larger id
      s_drop = drop;
    }
    __syncthreads();
    // node position: mean of the involved narrow bands (pre-merge state)
    {
      double acc[3] = {0.0, 0.0, 0.0};
      int32_t cnt = 0;
      const int32_t *__restrict__ seg = d.fseg[cur] + d.voff[p];
      const int32_t ns = d.pfront[(size_t)cur * d.P + p];
      for (int32_t j = threadIdx.x; j < ns; j += blockDim.x) {
        const int32_t v = seg[j];
        bool inb = false;
        for (int32_t j = 0; j < nm; ++j) inb |= in_band_of(d, v, mem[j]);
        if (inb) {
          for (int c = 0; c < 3; ++c) acc[c] += d.X[3 * (int64_t)v + c];
          ++cnt;
        }
      }
      block_sum3(acc, cnt, s_pos, &s_cnt);
    }
    const int32_t node = d.gnode[g];
    if (threadIdx.x == 0 && node >= 0) {
      for (int c = 0; c < 3; ++c) d.npos[3 * (int64_t)node + c] = s_cnt ? s_pos[c] / (double)s_cnt : 0.0;
      s_nodeloc = d.nlocal[node];
    }
    __syncthreads();
    // handle loops of the members except the dropped one, ascending layer order
    for (int32_t j = 0; j < nm; ++j) {
      if (j == s_drop) continue;
      const int32_t tb = s_first + j;
      const int32_t L = d.tlen[tb];
      const int32_t l = mem[j];
      const unsigned long long *key = d.tkey + (int64_t)tb * TRACE_CAP;
      const int32_t *ord = d.tord + (int64_t)tb * TRACE_CAP;
      if (threadIdx.x == 0) {
        s_hidx = atomicAdd(d.nhand, 1);
        s_eoff = atomicAdd(d.nhedge, L > 0 ? L : 0);
        if (s_hidx >= d.hcap || s_eoff + L > d.ecap) { atomicCAS(&d.pstatus[p], 0, (int32_t)VLS_ELAYERS); s_hidx = -1; }
      }
      __syncthreads();
      if (s_hidx >= 0) {
        for (int32_t q = threadIdx.x; q < L; q += blockDim.x) {
          if (!VCHK(d.err, ord[q], TRACE_CAP, 211)) continue;
          const unsigned long long kk = key[ord[q]];
          const int32_t a = (int32_t)(kk >> 32), b = (int32_t)(kk & 0xffffffffull);
          if (!VCHK(d.err, a, d.V, 212) || !VCHK(d.err, b, d.V, 213)) continue;
          d.hedge[2 * (int64_t)(s_eoff + q)] = a;
          d.hedge[2 * (int64_t)(s_eoff + q) + 1] = b;
          const double pa = psi_iso(d, a, l), pb = psi_iso(d, b, l);
          const double tt = ddiv(dsub(pa, th), dsub(pa, pb));
          for (int c = 0; c < 3; ++c) {
            const double xa = d.X[3 * (int64_t)a + c], xb = d.X[3 * (int64_t)b + c];
            d.hpts[3 * (int64_t)(s_eoff + q) + c] = dadd(xa, dmul(tt, dsub(xb, xa)));
          }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          // collapsed inside-vertex cycle and polyline length, in loop order
          int32_t nv = 0;
          for (int32_t q = 0; q < L; ++q) {
            const int32_t a = d.hedge[2 * (int64_t)(s_eoff + q)];
            if (nv == 0 || d.hverts[s_eoff + nv - 1] != a) d.hverts[s_eoff + nv++] = a;
          }
          while (nv > 1 && d.hverts[s_eoff + nv - 1] == d.hverts[s_eoff]) --nv;
          double len = 0.0;
          for (int32_t q = 0; q < L; ++q) {
            const double *pp = d.hpts + 3 * (int64_t)(s_eoff + q);
            const double *qq = d.hpts + 3 * (int64_t)(s_eoff + (q + 1) % L);
            const double dx = dsub(qq[0], pp[0]), dy = dsub(qq[1], pp[1]), dz = dsub(qq[2], pp[2]);
            len = dadd(len, dsqrt(dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz))));
          }
          const int32_t h = s_hidx;
          d.hprob[h] = p;
          d.hstep[h] = t;
          d.hlayer[h] = l - d.lbase[p];
          d.hnode[h] = s_nodeloc;
          d.hoff[h] = s_eoff;
          d.hn[h] = L;
          d.hvoff[h] = s_eoff;
          d.hvn[h] = nv;
          d.hlen[h] = len;
        }
      }
      __syncthreads();
    }
    // the merged layer, member states, values summed at the collision rows
    if (threadIdx.x == 0) {
      const int32_t N = new_layer(d, p, s_nodeloc);
      s_N = N;
      for (int32_t j = 0; j < nm; ++j) {
        d.lstate[mem[j]] = L_MERGED;
        d.lfwd[mem[j]] = N;
        d.ldeath[mem[j]] = s_nodeloc;
      }
      d.nalive[p] += 1 - nm;
    }
    __syncthreads();
    const int32_t N = s_N;
    const int32_t nc = *d.ncoll;
    for (int32_t c = threadIdx.x; c < nc; c += blockDim.x) {
      const int32_t row = d.coll[c];
      const int32_t l0 = d.olay[(int64_t)row * KMAX];
      bool mine = false;
      for (int32_t j = 0; j < nm; ++j) mine |= (mem[j] == l0);
      if (!mine) continue;
      double acc = 0.0;
      for (int q = 0; q < d.onl[row]; ++q) acc = dadd(acc, d.ophi[(int64_t)row * KMAX + q]);
      const int32_t v = fv[row];
      d.lay[v] = N;
      ph_st_round(d, P, v, acc);
    }
    __syncthreads();
  }
}

// Literal relabel (Sec. 3.1: the merged layers' entries move to the new layer), over the vertex
// ranges of the problems that merged this step only.
__global__ void k_relabel(Dev d) {
  const int32_t ng = *d.ngroups;
  // collision rows are single-layer again once the last round of the step's merge phase is done
  // (a later round still reads the rows of its groups)
  if (d.ctl[CTL_MSKIP] == 0) {
    const int32_t *__restrict__ fv = d.front[d.ctl[CTL_T] & 1];
    const int32_t nc = *d.ncoll;
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) d.multi[fv[d.coll[c]]] = -1;
  }
  for (int32_t g = 0; g < ng; ++g) {
    const int32_t p = d.gprob[g];
    bool seen = false;
    for (int32_t h = 0; h < g; ++h) seen |= d.gprob[h] == p;
    if (seen) continue;
    for (int32_t v = d.voff[p] + blockIdx.x * blockDim.x + threadIdx.x; v < d.voff[p + 1]; v += gridDim.x * blockDim.x) {
      const int32_t l = d.lay[v];
      if (l != 0) {
        const int32_t f = d.lfwd[l];
        if (f != 0) d.lay[v] = f;
      }
    }
  }
}

// ------------------------------------------------------------------ splits / extinctions
__global__ void __launch_bounds__(256) k_split(Dev d) {
  const int32_t p = blockIdx.x;
  if (p >= d.P || d.pdone[p]) return;
  const int32_t t = d.ctl[CTL_T], cur = t & 1;
  // this problem's frontier rows
  const int32_t *__restrict__ seg = d.fseg[cur] + d.voff[p];
  const int32_t ns = d.pfront[(size_t)cur * d.P + p];
  constexpr int MAXC = 64;
  __shared__ int32_t roots[MAXC], child[MAXC];
  __shared__ int32_t s_c, s_nroot, s_nodeloc, s_lc;
  __shared__ double s_pos[3];
  __shared__ int32_t s_cnt;
  if (threadIdx.x == 0) s_lc = d.lcount[p];
  __syncthreads();
  const int32_t lc = s_lc;
  for (int32_t loc = 1; loc <= lc; ++loc) {
    const int32_t l = d.lbase[p] + loc;
    if (d.lstate[l] != L_ALIVE) continue; // uniform across the block
    if (threadIdx.x == 0) {
      s_c = d.lcnt[l];
      d.lcnt[l] = 0;
      s_nroot = 0;
    }
    __syncthreads();
    const int32_t c = s_c;
    if (c == 1) { __syncthreads(); continue; }
    double acc[3] = {0.0, 0.0, 0.0};
    int32_t cnt = 0;
    if (c == 0) {
      // extinction: mean of this step's rows that hold l
      for (int32_t j = threadIdx.x; j < ns; j += blockDim.x)
        if (d.lay[seg[j]] == l) {
          for (int q = 0; q < 3; ++q) acc[q] += d.X[3 * (int64_t)seg[j] + q];
          ++cnt;
        }
      block_sum3(acc, cnt, s_pos, &s_cnt);
      if (threadIdx.x == 0) {
        const int32_t node = new_node(d, p, N_END, t);
        if (node >= 0) {
          for (int q = 0; q < 3; ++q) d.npos[3 * (int64_t)node + q] = s_cnt ? s_pos[q] / (double)s_cnt : 0.0;
          d.ldeath[l] = d.nlocal[node];
        }
        d.lstate[l] = L_ENDED;
        d.nalive[p] -= 1;
        d.pev[3 * p + 2]++;
      }
      __syncthreads();
      continue;
    }
    // split: collect the component roots (smallest vertex of each component)
    for (int32_t j = threadIdx.x; j < ns; j += blockDim.x) {
      const int32_t v = seg[j];
      if (d.lay[v] != l) continue;
      if (!ph_band(d, v)) continue;
      for (int q = 0; q < 3; ++q) acc[q] += d.X[3 * (int64_t)v + q];
      ++cnt;
      if (VCHK(d.err, d.uf[v], d.V, 221) && d.uf[v] == v) {
        const int32_t k = atomicAdd(&s_nroot, 1);
        if (k < MAXC) roots[k] = v;
      }
    }
    block_sum3(acc, cnt, s_pos, &s_cnt);
    if (threadIdx.x == 0) {
      const int32_t nr = s_nroot < MAXC ? s_nroot : MAXC;
      if (s_nroot > MAXC) atomicCAS(&d.pstatus[p], 0, (int32_t)VLS_ELAYERS);
      for (int32_t i = 1; i < nr; ++i) {
        int32_t x = roots[i], j = i - 1;
        while (j >= 0 && roots[j] > x) { roots[j + 1] = roots[j]; --j; }
        roots[j + 1] = x;
      }
      const int32_t node = new_node(d, p, N_SPLIT, t);
      s_nodeloc = node >= 0 ? d.nlocal[node] : -1;
      if (node >= 0)
        for (int q = 0; q < 3; ++q) d.npos[3 * (int64_t)node + q] = s_cnt ? s_pos[q] / (double)s_cnt : 0.0;
      d.lstate[l] = L_DEAD;
      d.ldeath[l] = s_nodeloc;
      for (int32_t i = 0; i < nr; ++i) child[i] = new_layer(d, p, s_nodeloc);
      d.nalive[p] += nr - 1;
      s_nroot = nr;
      d.pev[3 * p + 1]++;
    }
    __syncthreads();
    const int32_t nr = s_nroot;
    for (int32_t j = threadIdx.x; j < ns; j += blockDim.x) {
      const int32_t v = seg[j];
      if (d.lay[v] != l) continue;
      if (!ph_band(d, v)) continue;
      const int32_t r = uf_find(d.uf, v);
      if (!VCHK(d.err, r, d.V, 220)) continue;
      for (int32_t k = 0; k < nr; ++k)
        if (roots[k] == r) { d.lay[v] = child[k]; break; }
    }
    __syncthreads();
  }
}

// The round loop of a merge phase is entered with its condition set: a handle's default value is
// applied when the whole graph is launched, not each time the IF body runs.
__global__ void k_mround_start(Handles H) {
  if (threadIdx.x == 0 && H.use) cudaGraphSetConditional(H.mround, 1u);
}

}  // namespace

// IF(merge) body: WHILE(groups left) { groups -> traces (one block each) -> finish -> relabel }
cudaError_t add_merge_nodes(Batch &b, cudaGraph_t gif, const cudaGraphNode_t *dep) {
  Dev &d = b.d;
  int32_t *luf = d.lcnt + b.Lcap;                  // [Lcap] layer union-find scratch (init -1)
  int32_t *touched = d.lcnt + 2 * (size_t)b.Lcap;  // [Lcap]
  cudaGraphNode_t s0, w, n0, n1, n2, n3;
  Handles H{};
  H.use = 1;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphConditionalHandleCreate(&H.mround, gif, 1u, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = add_kernel(&s0, gif, dep, dep ? 1 : 0, k_mround_start, dim3(1), dim3(32), H);
  if (e == cudaSuccess) {
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = H.mround;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&w, gif, &s0, nullptr, 1, &np);
    if (e == cudaSuccess) g = np.conditional.phGraph_out[0];
  }
  if (e == cudaSuccess) e = add_kernel(&n0, g, nullptr, 0, k_merge_groups, dim3(1), dim3(32), d, luf, touched, H);
  if (e == cudaSuccess) e = add_kernel(&n1, g, &n0, 1, k_trace, dim3(MAX_TRACES), dim3(1024), d, b.prm);
  if (e == cudaSuccess) e = add_kernel(&n2, g, &n1, 1, k_merge_finish, dim3(MAX_TRACES), dim3(1024), d, b.prm);
  if (e == cudaSuccess) e = add_kernel(&n3, g, &n2, 1, k_relabel, dim3(b.cfg[KK_RELABEL].grid), dim3(b.cfg[KK_RELABEL].threads), d);
  return e;
}

// IF(split / extinction) body
cudaError_t add_split_nodes(Batch &b, cudaGraph_t g) {
  cudaGraphNode_t n0;
  return add_kernel(&n0, g, nullptr, 0, k_split, dim3(b.P), dim3(256), b.d);
}

void configure_events(Batch &b) { b.cfg[KK_RELABEL] = wave_cfg(b, k_relabel, 256); }

cudaError_t merge_phase_host(Batch &b) {
  Dev &d = b.d;
  cudaStream_t st = b.st;
  int32_t *luf = d.lcnt + b.Lcap;
  int32_t *touched = d.lcnt + 2 * (size_t)b.Lcap;
  Handles H{};
  H.use = 0;
  for (;;) {
    long ps = b.prof.begin(st, KK_MERGE_GROUPS);
    k_merge_groups<<<1, 32, 0, st>>>(d, luf, touched, H); VLS_LAUNCH(b);
    b.prof.end(st, ps);
    ps = b.prof.begin(st, KK_TRACE);
    k_trace<<<MAX_TRACES, 1024, 0, st>>>(d, b.prm); VLS_LAUNCH(b);
    b.prof.end(st, ps);
    ps = b.prof.begin(st, KK_MERGE_FINISH);
    k_merge_finish<<<MAX_TRACES, 1024, 0, st>>>(d, b.prm); VLS_LAUNCH(b);
    b.prof.end(st, ps);
    ps = b.prof.begin(st, KK_RELABEL);
    k_relabel<<<b.cfg[KK_RELABEL].grid, b.cfg[KK_RELABEL].threads, 0, st>>>(d); VLS_LAUNCH(b);
    b.prof.end(st, ps);
    // another round while groups of this step are left (rare: more traces than MAX_TRACES)
    int32_t skip = 0;
    cudaError_t e = cudaMemcpyAsync(&skip, d.ctl + CTL_MSKIP, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    b.d2h += (int64_t)sizeof(int32_t);
    if (e != cudaSuccess) return e;
    if (skip == 0) break;
  }
  return cudaGetLastError();
}

cudaError_t split_phase_host(Batch &b) {
  const long ps = b.prof.begin(b.st, KK_SPLIT);
  k_split<<<b.P, 256, 0, b.st>>>(b.d); VLS_LAUNCH(b);
  b.prof.end(b.st, ps);
  return cudaGetLastError();
}

}  // namespace vls
