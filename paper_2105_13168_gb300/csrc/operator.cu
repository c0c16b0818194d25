// operator.cu -- mesh validation and operator construction on the device (step a0).
//
// The operator is the uniform scaled Laplacian L_vu = s / d_v (u ~ v), L_vv = -s, a reading
// of the paper's "standard linear finite element approximation" (Sec. 2, "Implementation
// details") that needs only the connectivity: its values are recomputed in registers from
// the row length, so the operator in memory is the CSR pattern alone (rp, col) plus, per
// half-edge, the face holding it (hface), which the isoline tracer walks.
//
// Validation (per problem, first failure wins in this order): index range / degenerate face
// -> EINVAL; a directed half-edge used twice -> ENONORIENTABLE; a half-edge without twin ->
// ENOTMANIFOLD; per vertex in ascending order: no incident face -> EDISCONNECTED, fan not a
// single cycle -> ENOTMANIFOLD; more than one connected component -> EDISCONNECTED.
#include <climits>

#include "vls_batch.cuh"

namespace vls {

namespace {

constexpr int SCAN_T = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t x, int32_t *warp_sums, int32_t *total) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int32_t w = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
    int32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    warp_sums[lane] = wi - w;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  int32_t r = incl - x + warp_sums[wid];
  __syncthreads();
  return r;
}

// tile sums of in[0..n)
__global__ void k_scan_tiles(const int32_t *in, int64_t n, int32_t *tile_sums) {
  __shared__ int32_t ws[32];
  __shared__ int32_t tot;
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int32_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
    if (i < n) s += in[i];
  }
  block_exclusive_scan(s, ws, &tot);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}
// exclusive scan of the tile sums in place (one block, sequential chunks)
__global__ void k_scan_sums(int32_t *tile_sums, int64_t ntiles) {
  __shared__ int32_t ws[32];
  __shared__ int32_t tot;
  int32_t carry = 0;
  for (int64_t b = 0; b < ntiles; b += blockDim.x) {
    int64_t i = b + threadIdx.x;
    int32_t x = i < ntiles ? tile_sums[i] : 0;
    int32_t e = block_exclusive_scan(x, ws, &tot);
    if (i < ntiles) tile_sums[i] = e + carry;
    carry += tot;
    __syncthreads();
  }
}
// out[i] = exclusive prefix of in; out[n] = total
__global__ void k_scan_apply(const int32_t *in, int64_t n, const int32_t *tile_sums, int32_t *out) {
  __shared__ int32_t ws[32];
  __shared__ int32_t tot;
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int32_t v[SCAN_ITEMS], s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
    v[k] = i < n ? in[i] : 0;
    s += v[k];
  }
  int32_t e = block_exclusive_scan(s, ws, &tot) + tile_sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
    if (i < n) out[i] = e;
    e += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = e;
}

// stage layout per problem: [0] EINVAL, [1] ENONORIENTABLE, [2] ENOTMANIFOLD (twin),
// [3] min(v * 16 + code) of per-vertex failures, [4] component roots
__global__ void k_faces(Dev d, int32_t *stage) {
  int64_t nf = d.NF;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    // problem of the face
    int32_t lo = 0, hi = d.P - 1;
    while (lo < hi) {
      int32_t m = (lo + hi + 1) >> 1;
      if (d.foff[m] <= f) lo = m;
      else hi = m - 1;
    }
    int32_t p = lo;
    int32_t nvp = d.voff[p + 1] - d.voff[p];
    int32_t *t = const_cast<int32_t *>(d.F) + 3 * f;
    int32_t a = t[0], b = t[1], c = t[2];
    bool bad = a < 0 || a >= nvp || b < 0 || b >= nvp || c < 0 || c >= nvp || a == b || b == c || a == c;
    if (bad) {
      stage[5 * p + 0] = 1;
      // keep indices in range so later kernels stay in bounds; the problem will not run
      a = 0; b = nvp > 1 ? 1 : 0; c = nvp > 2 ? 2 : 0;
    }
    t[0] = a + d.voff[p];
    t[1] = b + d.voff[p];
    t[2] = c + d.voff[p];
  }
}

__global__ void k_degree(Dev d, int32_t *deg) {
  int64_t n3 = 3 * (int64_t)d.NF;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&deg[d.F[i]], 1);
}

__global__ void k_fill(Dev d, int32_t *fillc) {
  int64_t n3 = 3 * (int64_t)d.NF;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t f = i / 3;
    int k = (int)(i - 3 * f);
    int32_t v = d.F[i], nx = d.F[3 * f + (k + 1) % 3];
    int32_t slot = d.rp[v] + atomicAdd(&fillc[v], 1);
    d.col[slot] = nx;
    d.hface[slot] = (int32_t)f;
  }
}

// sort each row by column (rows are short: insertion sort), flag duplicates
__global__ void k_sort_rows(Dev d, int32_t *stage) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < d.V; v += gridDim.x * blockDim.x) {
    int32_t b = d.rp[v], e = d.rp[v + 1];
    for (int32_t i = b + 1; i < e; ++i) {
      int32_t c = d.col[i], h = d.hface[i];
      int32_t j = i - 1;
      while (j >= b && d.col[j] > c) {
        d.col[j + 1] = d.col[j];
        d.hface[j + 1] = d.hface[j];
        --j;
      }
      d.col[j + 1] = c;
      d.hface[j + 1] = h;
    }
    for (int32_t i = b + 1; i < e; ++i)
      if (d.col[i] == d.col[i - 1]) {
        int32_t p = prob_of_vertex(d.voff, d.P, v);
        stage[5 * p + 1] = 1;
      }
  }
}

__global__ void k_twin_fan(Dev d, int32_t *stage) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < d.V; v += gridDim.x * blockDim.x) {
    int32_t b = d.rp[v], e = d.rp[v + 1];
    int32_t p = prob_of_vertex(d.voff, d.P, v);
    int32_t deg = e - b;
    int32_t vloc = v - d.voff[p];
    if (deg == 0) {
      atomicMin(&stage[5 * p + 3], vloc * 16 + VLS_EDISCONNECTED);
      continue;
    }
    bool twin_ok = true;
    for (int32_t k = b; k < e; ++k)
      if (slot_of(d.rp, d.col, d.col[k], v) < 0) twin_ok = false;
    if (!twin_ok) {
      stage[5 * p + 2] = 1;
      continue;
    }
    // fan: next neighbour = third vertex of the face holding v -> cur
    int32_t start = d.col[b], cur = start, steps = 0;
    do {
      int32_t k = slot_of(d.rp, d.col, v, cur);
      if (k < 0) { steps = -1; break; }
      const int32_t *t = d.F + 3 * (int64_t)d.hface[k];
      int32_t nxt = -1;
      for (int q = 0; q < 3; ++q)
        if (t[q] != v && t[q] != cur) nxt = t[q];
      cur = nxt;
      ++steps;
    } while (cur != start && cur >= 0 && steps <= deg);
    if (steps != deg) atomicMin(&stage[5 * p + 3], vloc * 16 + VLS_ENOTMANIFOLD);
  }
}

__global__ void k_conn_init(Dev d) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < d.V; v += gridDim.x * blockDim.x) d.uf[v] = v;
}
__global__ void k_conn_unite(Dev d) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < d.V; v += gridDim.x * blockDim.x)
    for (int32_t k = d.rp[v]; k < d.rp[v + 1]; ++k) {
      int32_t u = d.col[k];
      if (u < v) uf_unite(d.uf, u, v);
    }
}
__global__ void k_conn_count(Dev d, int32_t *stage) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < d.V; v += gridDim.x * blockDim.x)
    if (d.uf[v] == v) atomicAdd(&stage[5 * prob_of_vertex(d.voff, d.P, v) + 4], 1);
}

__global__ void k_stage_init(int32_t *stage, int32_t P) {
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    stage[5 * p + 0] = 0;
    stage[5 * p + 1] = 0;
    stage[5 * p + 2] = 0;
    stage[5 * p + 3] = INT_MAX;
    stage[5 * p + 4] = 0;
  }
}

}  // namespace

cudaError_t build_operator(Batch &b, int32_t *stage) {
  Dev &d = b.d;
  cudaStream_t st = b.st;
  int g = b.sm_count * 4, t = 256;
  k_stage_init<<<(b.P + 255) / 256, 256, 0, st>>>(stage, b.P); VLS_LAUNCH(b);
  k_faces<<<g, t, 0, st>>>(d, stage); VLS_LAUNCH(b);
  // degrees into rp[0..V) via a scratch (onl is V-sized and free at this point)
  int32_t *deg = d.onl;
  cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)b.V, st);
  k_degree<<<g, t, 0, st>>>(d, deg); VLS_LAUNCH(b);
  int64_t ntiles = ((int64_t)b.V + SCAN_TILE - 1) / SCAN_TILE;
  int32_t *tiles = d.stamp;  // V-sized scratch, reinitialised later
  k_scan_tiles<<<(unsigned)ntiles, SCAN_T, 0, st>>>(deg, b.V, tiles); VLS_LAUNCH(b);
  k_scan_sums<<<1, SCAN_T, 0, st>>>(tiles, ntiles); VLS_LAUNCH(b);
  k_scan_apply<<<(unsigned)ntiles, SCAN_T, 0, st>>>(deg, b.V, tiles, d.rp); VLS_LAUNCH(b);
  cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)b.V, st);
  k_fill<<<g, t, 0, st>>>(d, deg); VLS_LAUNCH(b);
  k_sort_rows<<<g, t, 0, st>>>(d, stage); VLS_LAUNCH(b);
  k_twin_fan<<<g, t, 0, st>>>(d, stage); VLS_LAUNCH(b);
  k_conn_init<<<g, t, 0, st>>>(d); VLS_LAUNCH(b);
  k_conn_unite<<<g, t, 0, st>>>(d); VLS_LAUNCH(b);
  k_conn_count<<<g, t, 0, st>>>(d, stage); VLS_LAUNCH(b);
  return cudaGetLastError();
}

}  // namespace vls
