// noalloc.cu -- one tunnel pass for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running where the device allocator is off
// limits (inside a pre-sized memory pool or an allocation-free region of a larger
// application) or where every device byte is budgeted up front.  vls_tunnel_pass_noalloc()
// serves them: the caller passes device inputs and outputs, and every byte of scratch the
// pass needs lives in g_noalloc_scratch, a fixed array of this library.  A device reserves the
// array when this translation unit's CUDA module is loaded on it -- with lazy module loading
// (the CUDA default) at the first call on that device -- and holds it until the process exits.
//
// The pass is the same computation as a tunnel pass of vls_detect (same operator, update,
// frontier rule, stop rule, trace and closure), run by a single thread block.
#include <mutex>

#include "vls_batch.cuh"

namespace vls {
namespace {

constexpr int64_t NA_MAX_V = 262144;       // vertices
constexpr int64_t NA_MAX_F = 3 * NA_MAX_V; // faces
constexpr int64_t NA_MAX_E = 65536;        // crossing edges of the handle loop
constexpr int NA_THREADS = 1024;
constexpr int8_t NF_SRC = 1, NF_TGT = 2, NF_VIS = 4;

constexpr size_t na_align(size_t x) { return (x + 255) & ~size_t(255); }
// byte offsets of the scratch regions
constexpr size_t NA_RP = 0;
constexpr size_t NA_CNT = NA_RP + na_align(sizeof(int32_t) * (NA_MAX_V + 1));
constexpr size_t NA_COL = NA_CNT + na_align(sizeof(int32_t) * NA_MAX_V);
constexpr size_t NA_FLAG = NA_COL + na_align(sizeof(int32_t) * 3 * NA_MAX_F);
constexpr size_t NA_PHI = NA_FLAG + na_align(sizeof(int8_t) * NA_MAX_V);
constexpr size_t NA_ONEW = NA_PHI + na_align(sizeof(double) * NA_MAX_V);
constexpr size_t NA_T = NA_ONEW + na_align(sizeof(double) * NA_MAX_V);
constexpr size_t NA_STAMP = NA_T + na_align(sizeof(int32_t) * NA_MAX_V);
constexpr size_t NA_F0 = NA_STAMP + na_align(sizeof(int32_t) * NA_MAX_V);
constexpr size_t NA_F1 = NA_F0 + na_align(sizeof(int32_t) * NA_MAX_V);
constexpr size_t NA_CUT = NA_F1 + na_align(sizeof(int32_t) * NA_MAX_V);
constexpr size_t NA_PATH = NA_CUT + na_align(sizeof(int32_t) * 2 * NA_MAX_E);
constexpr size_t NA_BYTES = NA_PATH + na_align(sizeof(int32_t) * NA_MAX_V);

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

struct NA {
  int32_t *rp, *cnt, *col, *T, *stamp, *fv[2], *cut, *path;
  int8_t *flag;
  double *phi, *onew;
};

__device__ __forceinline__ int32_t na_slot(const NA &s, int32_t u, int32_t w) {
  int32_t lo = s.rp[u], hi = s.rp[u + 1] - 1;
  while (lo <= hi) {
    const int32_t m = (lo + hi) >> 1;
    const int32_t c = s.col[m];
    if (c == w) return m;
    if (c < w) lo = m + 1;
    else hi = m - 1;
  }
  return -1;
}
__device__ __forceinline__ bool na_cut(const NA &s, int32_t ncut, int32_t k) {
  int32_t lo = 0, hi = ncut - 1;
  while (lo <= hi) {
    const int32_t m = (lo + hi) >> 1;
    if (s.cut[m] == k) return true;
    if (s.cut[m] < k) lo = m + 1;
    else hi = m - 1;
  }
  return false;
}
__device__ __forceinline__ bool na_kept(const NA &s, const int32_t *cover, int32_t step, int32_t ncut, int32_t v,
                                        int32_t u, int32_t k) {
  const int32_t c = cover[u];
  if (c < 0 || c > step) return false;
  const int8_t fv = s.flag[v], fu = s.flag[u];
  if (((fv & NF_SRC) && (fu & NF_TGT)) || ((fv & NF_TGT) && (fu & NF_SRC))) return !na_cut(s, ncut, k);
  return true;
}
__device__ bool na_in_frontier(const NA &s, const int32_t *cover, int32_t step, int32_t ncut, int32_t u) {
  const int32_t c = cover[u];
  if (c < 0 || c > step || (s.flag[u] & NF_SRC)) return false;
  bool lay = val_pos(s.phi[u]), bas = val_lt1(s.phi[u]);
  for (int32_t k = s.rp[u]; k < s.rp[u + 1] && !(lay && bas); ++k) {
    const int32_t w = s.col[k];
    if (!na_kept(s, cover, step, ncut, u, w, k)) continue;
    if (val_pos(s.phi[w])) lay = true;
    if (val_lt1(s.phi[w])) bas = true;
  }
  return lay && bas;
}

// block-wide exclusive scan of cnt[0..n) into rp[0..n] (rp[n] = total)
__device__ void na_scan(const int32_t *cnt, int32_t *rp, int32_t n) {
  __shared__ int32_t part[NA_THREADS];
  const int32_t per = (n + blockDim.x - 1) / blockDim.x;
  const int32_t beg = threadIdx.x * per, end = min(beg + per, n);
  int32_t s = 0;
  for (int32_t i = beg; i < end; ++i) s += cnt[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t run = 0;
    for (int32_t i = 0; i < (int32_t)blockDim.x; ++i) { const int32_t x = part[i]; part[i] = run; run += x; }
    rp[n] = run;
  }
  __syncthreads();
  int32_t o = part[threadIdx.x];
  for (int32_t i = beg; i < end; ++i) { rp[i] = o; o += cnt[i]; }
  __syncthreads();
}

__global__ void __launch_bounds__(NA_THREADS) k_tunnel_noalloc(unsigned char *scratch, const int32_t *F, int32_t nf,
                                                                int32_t nv, const int32_t *cover, int32_t handle_step,
                                                                const int32_t *edges, int32_t ne, Params P,
                                                                int32_t max_steps, int32_t *out_verts,
                                                                int32_t *out_info) {
  NA s;
  s.rp = reinterpret_cast<int32_t *>(scratch + NA_RP);
  s.cnt = reinterpret_cast<int32_t *>(scratch + NA_CNT);
  s.col = reinterpret_cast<int32_t *>(scratch + NA_COL);
  s.flag = reinterpret_cast<int8_t *>(scratch + NA_FLAG);
  s.phi = reinterpret_cast<double *>(scratch + NA_PHI);
  s.onew = reinterpret_cast<double *>(scratch + NA_ONEW);
  s.T = reinterpret_cast<int32_t *>(scratch + NA_T);
  s.stamp = reinterpret_cast<int32_t *>(scratch + NA_STAMP);
  s.fv[0] = reinterpret_cast<int32_t *>(scratch + NA_F0);
  s.fv[1] = reinterpret_cast<int32_t *>(scratch + NA_F1);
  s.cut = reinterpret_cast<int32_t *>(scratch + NA_CUT);
  s.path = reinterpret_cast<int32_t *>(scratch + NA_PATH);
  __shared__ int32_t nfr[2], bstar, status, stop, bad;
  const int tid = threadIdx.x, nth = blockDim.x;
  // inputs are checked before any scratch write indexed by them
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int64_t i = tid; i < 3 * (int64_t)nf; i += nth)
    if (F[i] < 0 || F[i] >= nv) bad = 1;
  for (int32_t i = tid; i < 2 * ne; i += nth)
    if (edges[i] < 0 || edges[i] >= nv) bad = 1;
  __syncthreads();
  if (bad) {
    if (tid == 0) { out_info[0] = VLS_EINVAL; out_info[1] = 0; out_info[2] = -1; out_info[3] = 0; }
    return;
  }
  // ---- CSR of the half-edges (ascending columns); scratch keeps the previous call's data,
  // so everything read below is written first
  for (int32_t v = tid; v < nv; v += nth) s.cnt[v] = 0;
  __syncthreads();
  for (int64_t i = tid; i < 3 * (int64_t)nf; i += nth) atomicAdd(&s.cnt[F[i]], 1);
  __syncthreads();
  na_scan(s.cnt, s.rp, nv);
  // a row longer than the operator table (LV_MAX neighbours) is rejected, as vls_detect does
  for (int32_t v = tid; v < nv; v += nth)
    if (s.rp[v + 1] - s.rp[v] > LV_MAX) bad = 1;
  for (int32_t v = tid; v < nv; v += nth) s.cnt[v] = 0;
  __syncthreads();
  if (bad) {
    if (tid == 0) { out_info[0] = VLS_EINVAL; out_info[1] = 0; out_info[2] = -1; out_info[3] = 0; }
    return;
  }
  for (int64_t i = tid; i < 3 * (int64_t)nf; i += nth) {
    const int64_t f = i / 3;
    const int32_t v = F[i], nx = F[3 * f + (i - 3 * f + 1) % 3];
    s.col[s.rp[v] + atomicAdd(&s.cnt[v], 1)] = nx;
  }
  __syncthreads();
  for (int32_t v = tid; v < nv; v += nth)
    for (int32_t i = s.rp[v] + 1; i < s.rp[v + 1]; ++i) {
      const int32_t c = s.col[i];
      int32_t j = i - 1;
      while (j >= s.rp[v] && s.col[j] > c) { s.col[j + 1] = s.col[j]; --j; }
      s.col[j + 1] = c;
    }
  // The pass runs on the area covered when the handle was found; when the handle loop
  // separates that area (the far side is never reached), it runs again on the whole surface.
  int32_t step = handle_step;
  const int32_t ncut = 2 * ne;
  for (int attempt = 0; attempt < 2; ++attempt) {
  // ---- pass state: sources held at 1, targets, cut half-edges
  for (int32_t v = tid; v < nv; v += nth) {
    s.flag[v] = 0;
    s.phi[v] = 0.0;
    s.T[v] = -1;
    s.stamp[v] = 0;
  }
  if (tid == 0) { nfr[0] = 0; nfr[1] = 0; bstar = 0x7fffffff; status = -1; stop = 0; }
  __syncthreads();
  for (int32_t i = tid; i < ne; i += nth) {
    const int32_t a = edges[2 * i], b = edges[2 * i + 1];
    s.flag[a] = NF_SRC;
    s.flag[b] = NF_TGT;
    s.phi[a] = 1.0;
    s.T[a] = 0;
  }
  __syncthreads();
  for (int32_t i = tid; i < ne; i += nth) {
    const int32_t a = edges[2 * i], b = edges[2 * i + 1];
    s.cut[2 * i] = na_slot(s, a, b);
    s.cut[2 * i + 1] = na_slot(s, b, a);
    s.fv[0][atomicAdd(&nfr[0], 1)] = a;
  }
  __syncthreads();
  if (tid == 0)
    for (int32_t i = 1; i < ncut; ++i) {
      const int32_t x = s.cut[i];
      int32_t j = i - 1;
      while (j >= 0 && s.cut[j] > x) { s.cut[j + 1] = s.cut[j]; --j; }
      s.cut[j + 1] = x;
    }
  __syncthreads();
  // ---- steps: F_tau in list tau & 1 (F_0 = sources, F_1 from their kept neighbourhoods)
  for (int32_t tau = 0;; ++tau) {
    const int cur = tau & 1, nxt = cur ^ 1;
    if (tau > 0) {
      const int32_t n = nfr[cur];
      for (int32_t i = tid; i < n; i += nth) {
        const int32_t v = s.fv[cur][i];
        int32_t dh = 0;
        for (int32_t k = s.rp[v]; k < s.rp[v + 1]; ++k) dh += na_kept(s, cover, step, ncut, v, s.col[k], k);
        const double Lv = dh > 0 ? P.lv[dh] : 0.0; // dh <= degree <= LV_MAX (checked above)
        const double diag = dh > 0 ? -P.s : 0.0;
        const double x = s.phi[v];
        double acc = 0.0, accb = 0.0;
        for (int32_t k = s.rp[v]; k < s.rp[v + 1]; ++k) {
          const int32_t u = s.col[k];
          if (na_kept(s, cover, step, ncut, v, u, k) && val_pos(s.phi[u])) acc = dadd(acc, dmul(Lv, s.phi[u]));
        }
        acc = dadd(acc, dmul(diag, x));
        for (int32_t k = s.rp[v]; k < s.rp[v + 1]; ++k) {
          const int32_t u = s.col[k];
          if (na_kept(s, cover, step, ncut, v, u, k) && val_lt1(s.phi[u]))
            accb = dadd(accb, dmul(Lv, dsub(1.0, s.phi[u])));
        }
        const double xb = dsub(1.0, x);
        accb = dadd(accb, dmul(diag, xb));
        double out;
        if (!vertex_update(P, 1, &x, &acc, xb, accb, &out)) out = x;
        s.onew[i] = out;
      }
      __syncthreads();
      for (int32_t i = tid; i < n; i += nth) {
        const int32_t v = s.fv[cur][i];
        s.phi[v] = s.onew[i];
        if (s.T[v] < 0 && s.phi[v] >= P.theta) {
          s.T[v] = tau;
          if (s.flag[v] & NF_TGT) atomicMin(&bstar, v);
        }
      }
      __syncthreads();
      if (bstar != 0x7fffffff) {
        if (tid == 0) { status = VLS_OK; stop = tau; }
        break;
      }
    }
    // next frontier from the closed kept neighbourhoods of this step's rows
    if (tid == 0) nfr[nxt] = 0;
    __syncthreads();
    const int32_t n = nfr[cur];
    for (int32_t i = tid; i < n; i += nth) {
      const int32_t v = s.fv[cur][i];
      for (int32_t k = s.rp[v] - 1; k < s.rp[v + 1]; ++k) {
        const int32_t u = (k < s.rp[v]) ? v : s.col[k];
        if (k >= s.rp[v] && !na_kept(s, cover, step, ncut, v, u, k)) continue;
        if (atomicExch(&s.stamp[u], tau + 1) == tau + 1) continue;
        if (na_in_frontier(s, cover, step, ncut, u)) s.fv[nxt][atomicAdd(&nfr[nxt], 1)] = u;
      }
    }
    __syncthreads();
    if (tau > 0 && nfr[nxt] == 0) {
      if (tid == 0) { status = VLS_ELOOPFAIL; stop = tau; }
      break;
    }
    if (tau >= max_steps) {
      if (tid == 0) { status = VLS_EMAXSTEPS; stop = tau; }
      break;
    }
  }
  __syncthreads();
  if (status != VLS_ELOOPFAIL || bstar != 0x7fffffff || ne == 0) break;
  step = INT32_MAX;
  __syncthreads();
  }
  if (tid != 0) return;
  out_info[0] = status;
  out_info[1] = stop;
  out_info[2] = status == VLS_OK ? bstar : (status == -1 ? 0 : -1);
  out_info[3] = 0;
  if (status != VLS_OK) return;
  // depth-first descent on (arrival raised, arrival, id) over kept edges with steps back from
  // dead ends, then closure along the loop
  int32_t np = 0, x = bstar;
  s.path[np++] = x;
  s.flag[x] |= NF_VIS;
  while (s.T[x] != 0) {
    const int32_t tx = s.T[x];
    int32_t best = -1, tb = 0, bup = 0;
    for (int32_t k = s.rp[x]; k < s.rp[x + 1]; ++k) {
      const int32_t u = s.col[k];
      if (!na_kept(s, cover, step, ncut, x, u, k)) continue;
      const int32_t tu = s.T[u];
      if (tu < 0 || (s.flag[u] & NF_VIS)) continue;
      const int32_t up = tu > tx ? 1 : 0;
      if (best < 0 || up < bup || (up == bup && (tu < tb || (tu == tb && u < best)))) {
        best = u;
        tb = tu;
        bup = up;
      }
    }
    if (best < 0) {
      if (np <= 1) { out_info[0] = VLS_ELOOPFAIL; return; }
      --np;
      x = s.path[np - 1];
      continue;
    }
    if (np >= nv) { out_info[0] = VLS_ELOOPFAIL; return; }
    s.flag[best] |= NF_VIS;
    s.path[np++] = best;
    x = best;
  }
  int64_t bd = -1, bj = -1;
  int dir = 1;
  for (int32_t i = 0; i < ne; ++i) {
    if (edges[2 * i + 1] != bstar) continue;
    for (int32_t j = 0; j < ne; ++j) {
      if (edges[2 * j] != x) continue;
      const int64_t fwd = ((int64_t)(i - j) % ne + ne) % ne, bwd = ((int64_t)(j - i) % ne + ne) % ne;
      const int64_t dd = fwd <= bwd ? fwd : bwd;
      if (bd < 0 || dd < bd) { bd = dd; bj = j; dir = fwd <= bwd ? 1 : -1; }
    }
  }
  int32_t nc = 0;
  for (int32_t i = 0; i < np; ++i) out_verts[nc++] = s.path[i];
  for (int64_t k = 1; k <= bd; ++k) {
    const int64_t ix = ((bj + dir * k) % ne + ne) % ne;
    const int32_t a = edges[2 * ix];
    if (nc < nv && out_verts[nc - 1] != a) out_verts[nc++] = a;
  }
  while (nc > 1 && out_verts[nc - 1] == out_verts[0]) --nc;
  out_info[3] = nc;
}

std::mutex g_na_mutex;
void *g_na_ptr[64] = {};  // per-device address of g_noalloc_scratch

}  // namespace
}  // namespace vls

using namespace vls;

extern "C" vls_status vls_tunnel_pass_noalloc(const int32_t *F, int64_t nf, int64_t nv, const int32_t *cover,
                                              int32_t handle_step, const int32_t *edges, int64_t n_edges,
                                              const vls_options *o, void *cuda_stream, int32_t *out_verts,
                                              int32_t *out_info) {
  if (!F || !cover || !edges || !out_verts || !out_info || nf < 4 || nv < 4 || n_edges < 1) return VLS_EINVAL;
  if (nv > NA_MAX_V || nf > NA_MAX_F || n_edges > NA_MAX_E) return VLS_ETOOLARGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return VLS_ECUDA;
  void *ptr = nullptr;
  {
    // once per device, with that device current: the device address of the scratch array
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return VLS_ECUDA;
      g_na_ptr[dev] = p;
    }
    ptr = g_na_ptr[dev];
  }
  vls_options opt;
  if (o) opt = *o;
  else vls_default_options(&opt);
  double c[4];
  vls_constants(&opt, c);
  Params P{};
  P.mu = opt.mu;
  P.e = opt.e;
  P.w = opt.w;
  P.ah = opt.a * opt.a / 2.0;
  P.dt = c[2];
  P.s = c[3];
  P.eps0 = opt.eps0;
  P.one_m_eps = 1.0 - opt.eps0;
  P.theta = opt.theta_iso;
  P.lv[0] = 0.0;
  for (int k = 1; k <= LV_MAX; ++k) P.lv[k] = P.s / (double)k;
  P.mun[0] = 0.0;
  for (int k = 1; k <= KMAX + 1; ++k) P.mun[k] = P.mu / (double)k;
  k_tunnel_noalloc<<<1, NA_THREADS, 0, (cudaStream_t)cuda_stream>>>(
      static_cast<unsigned char *>(ptr), F, (int32_t)nf, (int32_t)nv, cover, handle_step, edges, (int32_t)n_edges, P,
      opt.max_pass_steps, out_verts, out_info);
  return cudaGetLastError() == cudaSuccess ? VLS_OK : VLS_ECUDA;
}
