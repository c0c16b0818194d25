// initial.cu -- the initial pass (Sec. 3.1): per step
//   update   Eq. (2) explicit Euler step at every frontier row (Jacobi: reads the old state,
//            writes a per-row output), clamp, snap, column normalisation;
//   apply    scatter the rows into the state, collect rows where several layers meet
//            (merge candidates, Sec. 3.1), record cover steps;
//   events   merges, then band labelling and splits / extinctions (events.cu);
//   frontier next frontier = vertices of the closed neighbourhood of this step's rows whose
//            own closed neighbourhood holds the base and at least one live layer (only
//            those can change: all rates of Eq. (2) vanish elsewhere);
//   epilogue per-problem termination, step limit, step records.
// A frontier row is one thread: the Laplacian of each layer is a sequential sum over the
// row in CSR order (diagonal last), the same rounding order as the FP64 oracle.
#include "vls_batch.cuh"

namespace vls {

namespace {

__device__ __forceinline__ int32_t append(int32_t *counter) { return atomicAdd(counter, 1); }

// ------------------------------------------------------------------- update
__global__ void __launch_bounds__(256) k_update(Dev d, Params P, const int32_t *__restrict__ fv,
                                                const int32_t *__restrict__ fp, const int32_t *nF_ptr) {
  const int32_t nF = *nF_ptr;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nF; i += gridDim.x * blockDim.x) {
    const int32_t p = fp[i];
    if (d.pdone[p]) { d.onl[i] = -1; continue; }
    const int32_t v = fv[i];
    if (!VCHK(d.err, v, d.V, 101)) { d.onl[i] = -1; continue; }
    const int32_t b = d.rp[v], e = d.rp[v + 1];
    if (!VCHK(d.err, e, d.nnz + 1, 102) || !VCHK(d.err, b, e + 1, 103)) { d.onl[i] = -1; continue; }
    const int32_t lv = d.lay[v];
    if (!VCHK(d.err, lv, d.Lcap, 104)) { d.onl[i] = -1; continue; }
    const double xv = d.phi[v];
    int32_t o = 0;
    if (lv != 0 && d.lstate[lv] == L_ALIVE) o = lv;
    // layers present in the closed neighbourhood, base presence
    int32_t ls[KMAX];
    int nl = 0;
    bool hb = false, ovf = false;
    for (int32_t k = b - 1; k < e; ++k) {
      const int32_t u = (k < b) ? v : d.col[k];
      if (!VCHK(d.err, u, d.V, 105)) continue;
      const int32_t lu = d.lay[u];
      if (lu == 0) { hb = true; continue; }
      if (!VCHK(d.err, lu, d.Lcap, 106)) continue;
      if (frozen_state(d.lstate[lu])) continue; // a plateau reads as the row's own layer
      if (dsub(1.0, d.phi[u]) > 0.0) hb = true;
      bool dup = false;
      for (int q = 0; q < nl; ++q) dup |= (ls[q] == lu);
      if (!dup) {
        if (nl == KMAX) ovf = true;
        else {
          int q = nl++;
          while (q > 0 && ls[q - 1] > lu) { ls[q] = ls[q - 1]; --q; }
          ls[q] = lu;
        }
      }
    }
    if (ovf) {
      atomicCAS(&d.pstatus[p], 0, (int32_t)VLS_ESLOTS);
      d.onl[i] = -1;
      continue;
    }
    if (!hb || nl == 0) { d.onl[i] = -1; continue; }
    const double Lv = ddiv(P.s, (double)(e - b));
    const double xb = dsub(1.0, lv != 0 ? xv : 0.0);
    double x[KMAX], lap[KMAX], out[KMAX];
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
      if (q < nl) {
        const int32_t l = ls[q];
        double acc = 0.0;
        for (int32_t k = b; k < e; ++k) {
          const int32_t u = d.col[k];
          const int32_t lu = d.lay[u];
          double psi = 0.0;
          if (lu == l) psi = d.phi[u];
          else if (lu != 0 && frozen_state(d.lstate[lu])) psi = (o != 0 && l == o) ? 1.0 : 0.0;
          acc = dadd(acc, dmul(Lv, psi));
        }
        x[q] = (lv == l) ? xv : 0.0;
        acc = dadd(acc, dmul(-P.s, x[q]));
        lap[q] = acc;
      }
    }
    double accb = 0.0;
    for (int32_t k = b; k < e; ++k) {
      const int32_t u = d.col[k];
      const int32_t lu = d.lay[u];
      const double bu = (lu == 0) ? 1.0 : dsub(1.0, d.phi[u]);
      accb = dadd(accb, dmul(Lv, bu));
    }
    accb = dadd(accb, dmul(-P.s, xb));
    if (!vertex_update(P, nl, x, lap, xb, accb, out)) {
#pragma unroll
      for (int q = 0; q < KMAX; ++q)
        if (q < nl) out[q] = x[q];
    }
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < KMAX; ++q)
      if (q < nl && out[q] > 0.0) {
        d.olay[(int64_t)i * KMAX + cnt] = ls[q];
        d.ophi[(int64_t)i * KMAX + cnt] = out[q];
        ++cnt;
      }
    d.onl[i] = cnt;
  }
}

// ------------------------------------------------------------------- apply
__global__ void k_apply(Dev d, const int32_t *__restrict__ fv, const int32_t *__restrict__ fp,
                        const int32_t *nF_ptr, int32_t t) {
  const int32_t nF = *nF_ptr;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nF; i += gridDim.x * blockDim.x) {
    const int32_t c = d.onl[i];
    if (c < 0) continue;
    const int32_t v = fv[i];
    if (c == 0) {
      d.lay[v] = 0;
      d.phi[v] = 0.0;
    } else {
      d.lay[v] = d.olay[(int64_t)i * KMAX];
      d.phi[v] = d.ophi[(int64_t)i * KMAX];
      if (d.cover[v] < 0) d.cover[v] = t;
    }
    if (c >= 2) {
      d.multi[v] = i;
      const int32_t s = append(d.ncoll);
      if (VCHK(d.err, s, d.V, 110)) d.coll[s] = i;
      d.pmerge[fp[i]] = 1;
    }
  }
}

// ------------------------------------------------------------------- band labelling
__device__ __forceinline__ bool is_band(const Dev &d, int32_t v, int32_t &l) {
  l = d.lay[v];
  if (l == 0 || d.lstate[l] != L_ALIVE) return false;
  const double x = d.phi[v];
  return x > 0.0 && x < 1.0;
}

__global__ void k_band_init(Dev d, const int32_t *__restrict__ fv, const int32_t *__restrict__ fp,
                            const int32_t *nF_ptr) {
  const int32_t nF = *nF_ptr;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nF; i += gridDim.x * blockDim.x) {
    if (d.pdone[fp[i]]) continue;
    const int32_t v = fv[i];
    int32_t l;
    if (is_band(d, v, l)) d.uf[v] = v;
  }
}

__global__ void k_band_hook(Dev d, const int32_t *__restrict__ fv, const int32_t *__restrict__ fp,
                            const int32_t *nF_ptr, int32_t t) {
  const int32_t nF = *nF_ptr;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nF; i += gridDim.x * blockDim.x) {
    if (d.pdone[fp[i]]) continue;
    const int32_t v = fv[i];
    int32_t l;
    if (!is_band(d, v, l)) continue;
    for (int32_t k = d.rp[v]; k < d.rp[v + 1]; ++k) {
      const int32_t u = d.col[k];
      if (!VCHK(d.err, u, d.V, 130)) continue;
      if (u >= v || d.fmark[u] != t) continue; // band vertices are frontier rows of this step
      int32_t lu;
      if (is_band(d, u, lu) && lu == l) uf_unite(d.uf, u, v);
    }
  }
}

__global__ void k_band_count(Dev d, const int32_t *__restrict__ fv, const int32_t *__restrict__ fp,
                             const int32_t *nF_ptr) {
  const int32_t nF = *nF_ptr;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nF; i += gridDim.x * blockDim.x) {
    if (d.pdone[fp[i]]) continue;
    const int32_t v = fv[i];
    int32_t l;
    if (!is_band(d, v, l)) continue;
    if (uf_find(d.uf, v) == v) atomicAdd(&d.lcnt[l], 1);
  }
}

// ------------------------------------------------------------------- next frontier
__device__ __forceinline__ bool in_frontier(const Dev &d, int32_t u) {
  const int32_t lu = d.lay[u];
  if (lu != 0 && frozen_state(d.lstate[lu])) return false;
  bool hb = false, hl = false;
  const int32_t b = d.rp[u], e = d.rp[u + 1];
  for (int32_t k = b - 1; k < e && !(hb && hl); ++k) {
    const int32_t w = (k < b) ? u : d.col[k];
    const int32_t lw = d.lay[w];
    if (lw == 0) { hb = true; continue; }
    if (frozen_state(d.lstate[lw])) continue;
    hl = true;
    if (dsub(1.0, d.phi[w]) > 0.0) hb = true;
  }
  return hb && hl;
}

// F_t (cur) -> F_{t+1} (nxt).  `tnext` is the id of the step the new list belongs to.
__global__ void k_frontier(Dev d, const int32_t *__restrict__ fv, const int32_t *__restrict__ fp,
                           const int32_t *nF_ptr, int32_t *__restrict__ nv_out, int32_t *__restrict__ np_out,
                           int32_t *nN_ptr, int32_t *pcount_next, int32_t tnext, int32_t record) {
  const int32_t nF = *nF_ptr;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nF; i += gridDim.x * blockDim.x) {
    const int32_t p = fp[i];
    if (d.pdone[p]) continue;
    const int32_t v = fv[i];
    if (record) {
      int32_t l;
      if (is_band(d, v, l)) {
        atomicAdd(&d.rband[p], 1);
        const uint64_t key = ((uint64_t)(uint32_t)(v - d.voff[p]) << 32) | (uint32_t)(l - d.lbase[p]);
        atomicAdd(&d.rhash[p], (unsigned long long)mix64(key));
      }
    }
    const int32_t b = d.rp[v], e = d.rp[v + 1];
    for (int32_t k = b - 1; k < e; ++k) {
      const int32_t u = (k < b) ? v : d.col[k];
      if (!VCHK(d.err, u, d.V, 120)) continue;
      if (atomicExch(&d.stamp[u], tnext) == tnext) continue;
      if (!in_frontier(d, u)) continue;
      const int32_t s = append(nN_ptr);
      if (!VCHK(d.err, s, d.V, 121)) continue;
      nv_out[s] = u;
      np_out[s] = p;
      d.fmark[u] = tnext;
      atomicAdd(&pcount_next[p], 1);
    }
  }
}

// ------------------------------------------------------------------- epilogue
__global__ void k_epilogue(Dev d, int32_t *pcount_cur, int32_t *pcount_next, int32_t t, int32_t max_steps,
                           int32_t *active, int32_t *nF_cur) {
  __shared__ int32_t nact;
  if (threadIdx.x == 0) nact = 0;
  __syncthreads();
  for (int32_t p = threadIdx.x; p < d.P; p += blockDim.x) {
    if (!d.pdone[p]) {
      d.psteps[p] = t;
      d.pupd[p] += pcount_cur[p];
      if (d.record && t - 1 < d.rcap) {
        long long *r = d.rec + ((int64_t)p * d.rcap + (t - 1)) * 4;
        const unsigned long long h = d.rhash[p];
        r[0] = pcount_cur[p];
        r[1] = d.rband[p];
        r[2] = (long long)(h & 0xffffffffull);
        r[3] = (long long)(h >> 32);
      }
      d.rband[p] = 0;
      d.rhash[p] = 0ull;
      if (d.pstatus[p] != 0) d.pdone[p] = 1;
      else if (pcount_next[p] == 0) d.pdone[p] = 1;
      else if (t >= max_steps) { d.pstatus[p] = VLS_EMAXSTEPS; d.pdone[p] = 1; }
      if (!d.pdone[p]) atomicAdd(&nact, 1);
    }
    pcount_cur[p] = 0;
    d.pmerge[p] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *active = nact;
    *nF_cur = 0; // the list just consumed is reused two steps later
    *d.ncoll = 0;
  }
}

// ------------------------------------------------------------------- init
// Seed region: the closed 1-ring of the seed vertex gets layer 1 with value 1 (Sec. 2: a
// region is initialised to 1 inside and 0 outside; the column sum is already 1).
__global__ void k_init(Dev d, int32_t *fv0, int32_t *fp0, int32_t *nF0) {
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < d.P; p += gridDim.x * blockDim.x) {
    if (d.pstatus[p] != 0) { d.pdone[p] = 1; continue; }
    const int32_t s = d.voff[p] + d.seed[p];
    const int32_t L1 = d.lbase[p] + 1;
    d.lstate[L1] = L_ALIVE;
    d.lbirth[L1] = 0;
    d.ldeath[L1] = -1;
    d.lprob[L1] = p;
    d.lcount[p] = 1;
    const int32_t node = atomicAdd(d.nnodes, 1);
    d.nkind[node] = N_SEED;
    d.nstep[node] = 0;
    d.nprob[node] = p;
    d.nlocal[node] = 0;
    for (int c = 0; c < 3; ++c) d.npos[3 * (int64_t)node + c] = d.X[3 * (int64_t)s + c];
    d.pnodes[p] = 1;
    for (int32_t k = d.rp[s] - 1; k < d.rp[s + 1]; ++k) {
      const int32_t u = (k < d.rp[s]) ? s : d.col[k];
      if (!VCHK(d.err, u, d.V, 140)) continue;
      d.lay[u] = L1;
      d.phi[u] = 1.0;
      d.cover[u] = 0;
      const int32_t q = atomicAdd(nF0, 1);
      fv0[q] = u;
      fp0[q] = p;
    }
  }
}

// A finished problem must have covered everything with value 1 and have no live layer.
__global__ void k_final_vertices(Dev d, int32_t *pstall) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < d.V; v += gridDim.x * blockDim.x)
    if (d.lay[v] == 0 || dsub(1.0, d.phi[v]) > 0.0) pstall[prob_of_vertex(d.voff, d.P, v)] = 1;
}
__global__ void k_final_layers(Dev d, int32_t *pstall) {
  for (int32_t p = blockIdx.x; p < d.P; p += gridDim.x)
    for (int32_t l = threadIdx.x + 1; l <= d.lcount[p]; l += blockDim.x)
      if (d.lstate[d.lbase[p] + l] == L_ALIVE) pstall[p] = 1;
}
__global__ void k_final_status(Dev d, const int32_t *pstall) {
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < d.P; p += gridDim.x * blockDim.x)
    if (d.pstatus[p] == 0 && pstall[p]) d.pstatus[p] = VLS_ESTALL;
}

}  // namespace

// The frontier list buffers: index 0/1 alternate; list c holds F_t for t % 2 == c.
cudaError_t init_state(Batch &b) {
  Dev &d = b.d;
  cudaStream_t st = b.st;
  k_init<<<(b.P + 127) / 128, 128, 0, st>>>(d, d.front[0], d.front[0] + b.V, d.nfront + 0); VLS_LAUNCH(b);
  // F_1 from the seed regions (treated as the rows of step 0)
  int32_t *pc = d.pfront;
  k_frontier<<<b.grid, b.threads, 0, st>>>(d, d.front[0], d.front[0] + b.V, d.nfront + 0, d.front[1],
                                            d.front[1] + b.V, d.nfront + 1, pc + b.P, 1, 0); VLS_LAUNCH(b);
  cudaMemsetAsync(d.nfront + 0, 0, sizeof(int32_t), st);
  return cudaGetLastError();
}

cudaError_t initial_step(Batch &b, int t) {
  Dev &d = b.d;
  cudaStream_t st = b.st;
  const int cur = t & 1, nxt = cur ^ 1;
  int32_t *fv = d.front[cur], *fp = d.front[cur] + b.V;
  int32_t *nF = d.nfront + cur;
  int32_t *pcur = d.pfront + (size_t)cur * b.P, *pnxt = d.pfront + (size_t)nxt * b.P;
  const long ps = b.prof.begin(st, 0);
  k_update<<<b.grid, b.threads, 0, st>>>(d, b.prm, fv, fp, nF); VLS_LAUNCH(b);
  b.prof.end(st, ps);
  k_apply<<<b.grid, b.threads, 0, st>>>(d, fv, fp, nF, t); VLS_LAUNCH(b);
  cudaError_t e = merge_phase(b, t, cur);
  if (e != cudaSuccess) return e;
  k_band_init<<<b.grid, b.threads, 0, st>>>(d, fv, fp, nF); VLS_LAUNCH(b);
  k_band_hook<<<b.grid, b.threads, 0, st>>>(d, fv, fp, nF, t); VLS_LAUNCH(b);
  k_band_count<<<b.grid, b.threads, 0, st>>>(d, fv, fp, nF); VLS_LAUNCH(b);
  e = split_phase(b, t, cur);
  if (e != cudaSuccess) return e;
  k_frontier<<<b.grid, b.threads, 0, st>>>(d, fv, fp, nF, d.front[nxt], d.front[nxt] + b.V, d.nfront + nxt, pnxt,
                                            t + 1, d.record); VLS_LAUNCH(b);
  k_epilogue<<<1, 256, 0, st>>>(d, pcur, pnxt, t, b.opt.max_steps, d.err + 1, nF); VLS_LAUNCH(b);
  return cudaGetLastError();
}

cudaError_t final_checks(Batch &b) {
  Dev &d = b.d;
  int32_t *pstall = d.pev + 3 * b.P; // spare P ints after the event counters
  cudaMemsetAsync(pstall, 0, sizeof(int32_t) * b.P, b.st);
  k_final_vertices<<<b.sm_count * 4, 256, 0, b.st>>>(d, pstall); VLS_LAUNCH(b);
  k_final_layers<<<b.P < 1024 ? b.P : 1024, 128, 0, b.st>>>(d, pstall); VLS_LAUNCH(b);
  k_final_status<<<(b.P + 255) / 256, 256, 0, b.st>>>(d, pstall); VLS_LAUNCH(b);
  return cudaGetLastError();
}

}  // namespace vls
