// tunnel.cu -- tunnel passes (Sec. 3.2), one per handle loop, all passes of a batch in the
// same launches (Sec. 4: many single-layer passes run concurrently).
//
// Pass q of handle h (problem p, found at step t_h):
//   domain   vertices covered by step t_h (the area the initial pass had reached, Sec. 3.2)
//   cut      the handle loop's crossing edges are removed (the loop is the border)
//   operator uniform scaled Laplacian of the cut, restricted graph (rows renormalised over the
//            kept edges: s / d_h(v) off the diagonal, -s on it)
//   field    one dense layer (Sec. 4: the base is 1 - phi), phi = 1 held on the inside
//            endpoints of the loop's crossing edges, Eq. (2) with n = 2 elsewhere
//   stop     when an outside endpoint first reaches theta_iso; b* = the smallest such vertex
//   trace    from b*, repeatedly the unvisited kept neighbour with the least (arrival, id)
//            whose arrival step is not larger, down to a source; the cycle is closed along
//            the handle loop by the shorter way to a crossing edge ending at b*.
//   stream   (streamlines on) the PL steepest-descent path of the arrival time from b* to a
//            source, closed the same way (k_tstream below).
// Only rows whose closed neighbourhood holds both phases change, so each step updates the
// frontier rows only (exact).
#include <math_constants.h>

#include <type_traits>

#include "vls_batch.cuh"

namespace vls {

namespace {

constexpr int8_t F_SRC = 1, F_TGT = 2, F_VIS = 4;
// frontier rows per warp of the pass kernels: the passes' frontiers (every pass of a chunk at once)
// are large, where one row per lane is fastest (measured: 19 us per update launch on the tube chain
// against 23 and 35 us with 16 and 8 rows per warp)
constexpr int32_t PASS_RPW = 32;

struct PassRow {
  int32_t q, p, base, voff, step;
};

__device__ __forceinline__ bool in_dom(const Dev &d, int32_t u, int32_t step) {
  const int32_t c = d.cover[u];
  return c >= 0 && c <= step;
}
// grp-edge slot k (v -> u) is cut in pass q
__device__ __forceinline__ bool is_cut(const TDev &T, int32_t q, int32_t k) {
  const int32_t *c = T.cut + T.pcoff[q];
  int32_t lo = 0, hi = T.pcn[q] - 1;
  while (lo <= hi) {
    const int32_t m = (lo + hi) >> 1;
    if (c[m] == k) return true;
    if (c[m] < k) lo = m + 1;
    else hi = m - 1;
  }
  return false;
}
__device__ __forceinline__ bool kept(const Dev &d, const TDev &T, int32_t q, int32_t step, int32_t base, int32_t voff,
                                     int8_t fv, int32_t u, int32_t k) {
  if (!in_dom(d, u, step)) return false;
  const int8_t fu = T.flag[base + (u - voff)];
  if (((fv & F_SRC) && (fu & F_TGT)) || ((fv & F_TGT) && (fu & F_SRC))) return !is_cut(T, q, k);
  return true;
}

template <class TV> __device__ __forceinline__ const TV *tph_arr(const TDev &T);
template <> __device__ __forceinline__ const double *tph_arr<double>(const TDev &T) { return T.phi; }
template <> __device__ __forceinline__ const float *tph_arr<float>(const TDev &T) { return T.phif; }
template <> __device__ __forceinline__ const __nv_bfloat16 *tph_arr<__nv_bfloat16>(const TDev &T) { return T.phih; }
__device__ __forceinline__ double tph_ld(const TDev &T, int32_t i) {
  return T.phih ? to_f64(T.phih[i]) : T.phif ? (double)T.phif[i] : T.phi[i];
}
// a row output (exactly representable in float in the FP32 form) into the pass state
__device__ __forceinline__ void tph_st(const TDev &T, int32_t i, double x) {
  if (T.phih) T.phih[i] = __double2bfloat16(x);
  else if (T.phif) T.phif[i] = (float)x;
  else T.phi[i] = x;
}

// Block-cooperative bitonic sort (ascending) of a[0, n2), n2 a power of two; a is shared or
// block-private global memory (__syncthreads orders both).  Every thread of the block calls it.
__device__ void block_bitonic_sort(int32_t *a, int32_t n2) {
  for (int32_t k = 2; k <= n2; k <<= 1)
    for (int32_t j = k >> 1; j > 0; j >>= 1) {
      for (int32_t i = threadIdx.x; i < n2; i += blockDim.x) {
        const int32_t ixj = i ^ j;
        if (ixj > i) {
          const int32_t x = a[i], y = a[ixj];
          if ((x > y) == ((i & k) == 0)) {
            a[i] = y;
            a[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
}
constexpr int32_t TINIT_SMEM_SORT = 4096; // cut slots sorted in shared memory up to this many

// per pass: flags, sources at 1, cut slots sorted, F_0 = sources
__global__ void __launch_bounds__(256) k_tinit(Dev d, TDev T, int32_t *fv0, int32_t *fq0, int32_t *nF0) {
  __shared__ int32_t sk[TINIT_SMEM_SORT];
  const int32_t q = blockIdx.x;
  if (q >= T.NP) return;
  const int32_t p = T.pprob[q];
  const int32_t base = T.pbase[q], voff = d.voff[p];
  const int32_t eo = T.heoff[q], L = T.hen[q];
  int32_t *cut = const_cast<int32_t *>(T.cut) + T.pcoff[q];
  const int32_t nvp = d.voff[p + 1] - voff;
  (void)nvp; // used by the checked build's guards
  for (int32_t i = threadIdx.x; i < L; i += blockDim.x) {
    const int32_t a = T.xedge[2 * (int64_t)(eo + i)], b = T.xedge[2 * (int64_t)(eo + i) + 1];
    if (!VCHK(T.err, a - voff, nvp, 301) || !VCHK(T.err, b - voff, nvp, 302)) continue;
    T.flag[base + (a - voff)] = F_SRC;
    T.flag[base + (b - voff)] = F_TGT;
    tph_st(T, base + (a - voff), 1.0);
    T.T[base + (a - voff)] = 0;
    if (T.tfa) T.tfa[base + (a - voff)] = 0.0;
    cut[2 * i] = slot_of(d.rp, d.col, a, b);
    cut[2 * i + 1] = slot_of(d.rp, d.col, b, a);
    const int32_t s = atomicAdd(nF0, 1);
    if (!VCHK(T.err, s, T.PV, 303)) continue;
    fv0[s] = a;
    fq0[s] = q;
  }
  __syncthreads();
  // sort the 2L cut slots (padded with INT32_MAX to a power of two): in shared memory, or for a
  // long loop in the pass's own stretch of the trace scratch (nvp entries, unused until the
  // trace); a loop too long even for that (never seen) keeps a one-thread insertion sort
  const int32_t n = 2 * L;
  int32_t n2 = 1;
  while (n2 < n) n2 <<= 1;
  int32_t *buf = n2 <= TINIT_SMEM_SORT ? sk : (n2 <= nvp ? T.path + base : nullptr);
  if (buf != nullptr) {
    for (int32_t i = threadIdx.x; i < n2; i += blockDim.x) buf[i] = i < n ? cut[i] : INT32_MAX;
    __syncthreads();
    block_bitonic_sort(buf, n2);
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) cut[i] = buf[i];
  } else if (threadIdx.x == 0) {
    for (int32_t i = 1; i < n; ++i) {
      int32_t x = cut[i], j = i - 1;
      while (j >= 0 && cut[j] > x) { cut[j + 1] = cut[j]; --j; }
      cut[j + 1] = x;
    }
  }
}

// Kept neighbours of a row of pass q, gathered before use: ids, then cover steps, flags and
// values (MAXD bounds the row length of one instantiation).
template <int MAXD, class TV>
__device__ __forceinline__ int gather_kept(const Dev &d, const TDev &T, int32_t q, int32_t step, int32_t base,
                                          int32_t voff, int8_t fl, int32_t v, int32_t b, int32_t deg, uint64_t &kp,
                                          TV *nx, int &nsrc) {
  const TV *__restrict__ ph = tph_arr<TV>(T);
  int32_t nu[MAXD];
  kp = 0;
  nsrc = 0;
#pragma unroll
  for (int j = 0; j < MAXD; ++j) nu[j] = (j < deg) ? d.col[b + j] : v;
#pragma unroll
  for (int j = 0; j < MAXD; ++j) {
    const int32_t c = (j < deg) ? d.cover[nu[j]] : -1;
    const int8_t f = (j < deg) ? T.flag[base + (nu[j] - voff)] : (int8_t)0;
    nx[j] = (j < deg) ? ph[base + (nu[j] - voff)] : TV(0.0f);
    bool k = j < deg && c >= 0 && c <= step;
    if (k && (((fl & F_SRC) && (f & F_TGT)) || ((fl & F_TGT) && (f & F_SRC)))) k = !is_cut(T, q, b + j);
    if (k) kp |= 1ull << j;
    nsrc += (k && (f & F_SRC)) ? 1 : 0;
  }
  return __popcll(kp);
}

// FP64 pass row (Eq. (2) with n = 2: the pass layer and its base) from the stored inputs
// (FP32 values are widened exactly).
template <int MAXD, class TV>
__device__ __forceinline__ double trow_f64(const Params &P, uint64_t kp, int dh, int nsrc, const TV *nx, TV xs,
                                           double2 &mass, bool *unc = nullptr) {
  const double Lv = dh > 0 ? P.lv[dh] : 0.0;
  const double diag = dh > 0 ? -P.s : 0.0;
  const double x = to_f64(xs);
  double acc = 0.0, accb = 0.0;
  // terms are >= 0 and the sums start at +0: zero terms are skipped (bit-identical)
#pragma unroll
  for (int j = 0; j < MAXD; ++j)
    if (((kp >> j) & 1ull) && val_pos(nx[j])) acc = dadd(acc, dmul(Lv, to_f64(nx[j])));
  acc = dadd(acc, dmul(diag, x));
#pragma unroll
  for (int j = 0; j < MAXD; ++j)
    if (((kp >> j) & 1ull) && val_lt1(nx[j])) accb = dadd(accb, dmul(Lv, dsub(1.0, to_f64(nx[j]))));
  const double xb = dsub(1.0, x);
  // mass check: m_v (L base)_v less the flux into the sources (held at 1, base 0; never rows), and
  // the magnitude of its terms
  mass = make_double2(0.0, dadd(dmul(P.mv[dh], accb), dmul((double)dh, xb)));
  accb = dadd(accb, dmul(diag, xb));
  mass.x = dmul(P.mv[dh], accb) + (double)nsrc * xb;
  double out;
  if (!vertex_update(P, 1, &x, &acc, xb, accb, &out, unc)) out = x;
  return out;
}

// FP32 pass row (values stored as float or bfloat16); false when a decision lies within the
// recheck margin.
template <int MAXD, class TN>
__device__ __forceinline__ bool trow_f32(const Params &P, uint64_t kp, int dh, int nsrc, const TN *nx, TN xs,
                                         double &out, double2 &mass, bool &unc) {
  if (dh == 0) return false;
  const float Lv = P.f_lv[dh];
  const float x = to_f32(xs);
  float acc = 0.f, accb = 0.f;
#pragma unroll
  for (int j = 0; j < MAXD; ++j)
    if ((kp >> j) & 1ull) {
      const float xj = to_f32(nx[j]);
      acc = fmaf(Lv, xj, acc);
      accb = fmaf(Lv, 1.f - xj, accb);
    }
  const float xb = 1.f - x;
  const float lapb = fmaf(-P.f_s, xb, accb);
  // mass check (FP64 from the FP32 sums), as in the FP64 row
  mass = make_double2(P.mv[dh] * (double)lapb + (double)nsrc * (double)xb,
                      P.mv[dh] * (double)accb + (double)dh * (double)xb);
  float y;
  if (!vertex_update_f32(P, x, fmaf(-P.f_s, x, acc), xb, lapb, y, unc)) return false;
  out = round_keep<TN>((double)y, P.theta); // exact for float storage
  return true;
}

// FP32 / BF16 forms: the FP64 redo of a pass row from copies of its gathered inputs, rounded to
// the stored type keeping every threshold's side; out of line (rare) so that the hot row keeps
// few registers.
template <int MAXD, class TV>
__device__ __noinline__ double trow_redo(const Params &P, uint64_t kp, int dh, int nsrc, const TV *nx, TV x,
                                         double2 &mass, bool &unc) {
  return round_keep<TV>(trow_f64<MAXD, TV>(P, kp, dh, nsrc, nx, x, mass, &unc), P.theta);
}

// Returns bit 0: redone in FP64; bit 2: a decision within the drift bound of its threshold.
template <int MAXD, class TV>
__device__ __forceinline__ int tupdate_row(const Dev &d, const TDev &T, const Params &P, int32_t i, int32_t q,
                                           int32_t v, double2 &mass) {
  const int32_t p = T.pprob[q], base = T.pbase[q], voff = d.voff[p], step = T.pstep[q];
  const int32_t idx = base + (v - voff);
  if (!VCHK(T.err, idx, T.PV, 310)) { T.onew[i] = 0.0; return 0; }
  const int8_t fl = T.flag[idx];
  const int32_t b = d.rp[v], deg = d.rp[v + 1] - b;
  uint64_t kp;
  TV nx[MAXD];
  int nsrc;
  const int dh = gather_kept<MAXD, TV>(d, T, q, step, base, voff, fl, v, b, deg, kp, nx, nsrc);
  const TV x = tph_arr<TV>(T)[idx];
  double out;
  bool redo = false, unc = false;
  if constexpr (!std::is_same<TV, double>::value) {
    if (!trow_f32<MAXD>(P, kp, dh, nsrc, nx, x, out, mass, unc)) {
      TV cx[MAXD];
#pragma unroll
      for (int j = 0; j < MAXD; ++j) cx[j] = nx[j];
      unc = false;
      out = trow_redo<MAXD, TV>(P, kp, dh, nsrc, cx, x, mass, unc);
      redo = true;
    }
  } else {
    out = trow_f64<MAXD, TV>(P, kp, dh, nsrc, nx, x, mass);
  }
  T.onew[i] = out;
  return (redo ? 1 : 0) | (unc ? 4 : 0);
}

template <class TV>
__device__ __noinline__ int tupdate_row_wide(const Dev &d, const TDev &T, const Params &P, int32_t i, int32_t q,
                                             int32_t v, double2 &mass) {
  return tupdate_row<64, TV>(d, T, P, i, q, v, mass);
}

template <class TV>
__device__ __forceinline__ void tupdate_rows(const Dev &d, const TDev &T, const Params &P) {
  const int32_t cur = __ldcg(T.ctl + CTL_TAU) & 1;
  const int32_t *__restrict__ fv = T.fv[cur];
  const int32_t *__restrict__ fq = T.fq[cur];
  const int32_t nF = __ldcg(T.nf + cur);
  uint32_t redo = 0;
  const int32_t R = PASS_RPW, lane = (int32_t)(threadIdx.x & 31);
  VLS_WARP_LOOP(w, R, nF) { // one row per lane of the first R lanes, then the warp's mass sums
    const int32_t i = w * R + lane;
    int32_t q = -1;
    double2 mass = make_double2(0.0, 0.0);
    int oc = 0;
    if (lane < R && i < nF) {
      const int32_t v = fv[i];
      q = fq[i];
      const int32_t deg = d.rp[v + 1] - d.rp[v];
      if (deg <= 12) oc = tupdate_row<12, TV>(d, T, P, i, q, v, mass);
      else if (deg <= 64) oc = tupdate_row_wide<TV>(d, T, P, i, q, v, mass);
      else T.onew[i] = tph_ld(T, T.pbase[q] + (v - d.voff[T.pprob[q]]));
      redo += oc & 1;
    }
    mass_sums(T.qmass, T.qslots, q, lane, mass);
    if constexpr (!std::is_same<TV, double>::value) count_keyed(T.qunc, q, (oc & 4) != 0);
  }
  if constexpr (!std::is_same<TV, double>::value) {
    redo = __reduce_add_sync(0xffffffffu, redo);
    if ((threadIdx.x & 31) == 0 && redo) atomicAdd(&d.nrecheck[1], (unsigned long long)redo);
  }
}

// One instantiation per stored value type, so that each form gets its own register budget.
template <class TV> __global__ void __launch_bounds__(256, VLS_UPDATE_MINB) k_tupdate(Dev d, TDev T, Params P) {
  pdl_enter();
  tupdate_rows<TV>(d, T, P);
}

__device__ __forceinline__ void tapply_phase(const Dev &d, const TDev &T, double theta) {
  const int32_t tau = __ldcg(T.ctl + CTL_TAU), cur = tau & 1;
  const int32_t *__restrict__ fv = T.fv[cur];
  const int32_t *__restrict__ fq = T.fq[cur];
  const int32_t nF = __ldcg(T.nf + cur);
  FOR_ROWS_R(i, nF, PASS_RPW) {
    const int32_t q = fq[i], v = fv[i];
    const int32_t p = T.pprob[q];
    const int32_t idx = T.pbase[q] + (v - d.voff[p]);
    if (!VCHK(T.err, idx, T.PV, 320)) continue;
    const double x = T.onew[i];
    if (T.T[idx] < 0 && x >= theta) {
      // arrival time: theta is crossed within this step, linearly in time between the old value
      // and the new one
      if (T.tfa) {
        const double old = tph_ld(T, idx);
        T.tfa[idx] = dadd((double)(tau - 1), ddiv(dsub(theta, old), dsub(x, old)));
      }
      T.T[idx] = tau;
      if (T.flag[idx] & F_TGT) atomicMin(&T.qbstar[q], v - d.voff[p]);
    }
    tph_st(T, idx, x);
  }
}
__global__ void k_tapply(Dev d, TDev T, double theta) {
  pdl_enter();
  tapply_phase(d, T, theta);
}

// u joins pass q's frontier iff it is in the domain, not a source, and its kept closed
// neighbourhood holds both phases (a value > 0 and a value < 1).  tgives(x): bit 0 the layer
// (x > 0), bit 1 the base (x < 1).  As in the initial pass, u qualifies iff tgives(u) = 3 or
// some kept neighbour w has tgives(u) | tgives(w) = 3, and every such pair has an endpoint in
// the current frontier (a pair outside it kept its values and qualified one step earlier), so
// the next frontier is found from the pairs (v, u), v in the frontier, u kept from v.
template <class TV> __device__ __forceinline__ uint32_t tgives(TV x) {
  return (val_pos(x) ? 1u : 0u) | (val_lt1(x) ? 2u : 0u);
}
__device__ __forceinline__ uint32_t tgives_at(const TDev &T, int32_t i) {
  return T.phih ? tgives(T.phih[i]) : T.phif ? tgives(T.phif[i]) : tgives(T.phi[i]);
}

// GL-lane groups per row, lane j takes the row's neighbour j (rows longer than GL loop).
// Returns true in the threads that appended to the next frontier (the epilogue reads its counts).
__device__ __forceinline__ bool tfrontier_phase(const Dev &d, const TDev &T) {
  const int32_t tau = __ldcg(T.ctl + CTL_TAU), cur = tau & 1, nxt = cur ^ 1, tnext = tau + 1;
  const int32_t *__restrict__ fv = T.fv[cur];
  const int32_t *__restrict__ fq = T.fq[cur];
  const int32_t nF = __ldcg(T.nf + cur);
  int32_t *__restrict__ nv_out = T.fv[nxt];
  int32_t *__restrict__ nq_out = T.fq[nxt];
  int32_t *nN_ptr = T.nf + nxt;
  int32_t *qcnt_next = T.qcnt + (size_t)nxt * T.NP;
  const int32_t lane = group_lane();
  const unsigned grp = group_mask();
  bool wrote = false;
  auto add = [&](int32_t u, int32_t iu, int32_t q) {
    wrote = true;
    if (atomicExch(&T.stamp[iu], tnext) == tnext) return;
    const int32_t s = warp_append(nN_ptr, qcnt_next, q);
    if (!VCHK(T.err, s, T.PV, 331)) return;
    nv_out[s] = u;
    nq_out[s] = q;
  };
  FOR_ROWS_G(i, nF) {
    const int32_t q = fq[i];
    if (__ldcg(T.qdone + q) || __ldcg(T.qbstar + q) != 0x7fffffff) continue;
    const int32_t v = fv[i];
    const int32_t p = T.pprob[q], base = T.pbase[q], voff = d.voff[p], step = T.pstep[q];
    const int32_t iv = base + (v - voff);
    if (!VCHK(T.err, iv, T.PV, 330)) continue;
    const int8_t fl = T.flag[iv];
    const uint32_t gv = tgives_at(T, iv);
    const int32_t b = d.rp[v], e = d.rp[v + 1];
    bool join = gv == 3u;
    for (int32_t k0 = b; k0 < e; k0 += GL) {
      const int32_t k = k0 + lane;
      if (k >= e) continue;
      const int32_t u = d.col[k];
      if (!kept(d, T, q, step, base, voff, fl, u, k)) continue;
      const int32_t iu = base + (u - voff);
      if (!VCHK(T.err, iu, T.PV, 332)) continue;
      const uint32_t gu = tgives_at(T, iu);
      if ((gv | gu) != 3u) continue;
      join = true;
      if (!(T.flag[iu] & F_SRC)) add(u, iu, q);
    }
    join = __any_sync(grp, join) && !(fl & F_SRC);
    if (lane == 0 && join) add(v, iv, q);
  }
  return wrote;
}


// One block: pass bookkeeping, then the step counter advances; the WHILE node stops when no
// pass is running (or at the hard step bound).
__device__ __forceinline__ void tepilogue_phase(const Dev &d, const TDev &T, const Handles &H, int32_t max_steps) {
  __shared__ int32_t nact;
  const int32_t tau = __ldcg(T.ctl + CTL_TAU), cur = tau & 1, nxt = cur ^ 1;
  int32_t *cnt_cur = T.qcnt + (size_t)cur * T.NP;
  int32_t *cnt_next = T.qcnt + (size_t)nxt * T.NP;
  if (threadIdx.x == 0) nact = 0;
  __syncthreads();
  for (int32_t q = threadIdx.x; q < T.NP; q += blockDim.x) {
    if (!__ldcg(T.qdone + q)) {
      T.qsteps[q] = tau;
      T.qupd[q] += __ldcg(cnt_cur + q);
      if (__ldcg(T.qbstar + q) != 0x7fffffff) { T.qdone[q] = 1; T.qstatus[q] = VLS_OK; }
      else if (__ldcg(cnt_next + q) == 0) { T.qdone[q] = 1; T.qstatus[q] = VLS_ELOOPFAIL; }
      else if (tau >= max_steps) { T.qdone[q] = 1; T.qstatus[q] = VLS_EMAXSTEPS; }
      if (!T.qdone[q]) atomicAdd(&nact, 1);
      T.qmres[q] = fmax(T.qmres[q], mass_fold(T.qmass, T.qslots, q));
    }
    cnt_cur[q] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T.ctl[CTL_TACTIVE] = nact;
    T.nf[cur] = 0;
    T.ctl[CTL_TAU] = tau + 1;
    if (H.use && (nact == 0 || tau >= T.ctl[CTL_TLIMIT])) cudaGraphSetConditional(H.loop, 0u);
  }
}

// The next frontier of every pass, then (epi = 1) the step's epilogue in the last block to finish.
__global__ void __launch_bounds__(256) k_tfrontier(Dev d, TDev T, Handles H, int32_t max_steps, int32_t epi) {
  pdl_enter();
  const bool wrote = tfrontier_phase(d, T);
  if (!epi) return;
  if (wrote) __threadfence(); // the epilogue reads the next frontier's counts
  if (last_block_fenced(T.ctl + CTL_DONE_TFRONT)) tepilogue_phase(d, T, H, max_steps);
}

// one thread per pass: greedy descent on (arrival, id), then closure along the loop
__global__ void k_ttrace(Dev d, TDev T) {
  for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < T.NP; q += gridDim.x * blockDim.x) {
    if (T.qstatus[q] != VLS_OK) continue;
    const int32_t p = T.pprob[q], base = T.pbase[q], voff = d.voff[p], step = T.pstep[q];
    int32_t *path = T.path + base;
    const int32_t nvp = d.voff[p + 1] - voff;
    (void)nvp; // used by the checked build's guards
    int32_t np = 0;
    if (!VCHK(T.err, T.qbstar[q], nvp, 340)) { T.qstatus[q] = VLS_ELOOPFAIL; continue; }
    int32_t x = voff + T.qbstar[q];
    path[np++] = x;
    T.flag[base + (x - voff)] |= F_VIS;
    bool fail = false;
    // depth first: the unvisited reached neighbour of least (arrival raised, arrival, id); from a
    // dead end, step back along the path
    while (T.T[base + (x - voff)] != 0) {
      const int32_t tx = T.T[base + (x - voff)];
      const int8_t fx = T.flag[base + (x - voff)];
      int32_t best = -1, tb = 0, bup = 0;
      for (int32_t k = d.rp[x]; k < d.rp[x + 1]; ++k) {
        const int32_t u = d.col[k];
        if (!kept(d, T, q, step, base, voff, fx, u, k)) continue;
        const int32_t iu = base + (u - voff);
        const int32_t tu = T.T[iu];
        if (tu < 0 || (T.flag[iu] & F_VIS)) continue;
        const int32_t up = tu > tx ? 1 : 0;
        if (best < 0 || up < bup || (up == bup && (tu < tb || (tu == tb && u < best)))) {
          best = u;
          tb = tu;
          bup = up;
        }
      }
      if (best < 0) {
        if (np <= 1) { fail = true; break; }
        --np;
        x = path[np - 1];
        continue;
      }
      if (!VCHK(T.err, np, nvp, 341)) { fail = true; break; }
      T.flag[base + (best - voff)] |= F_VIS;
      path[np++] = best;
      x = best;
    }
    if (fail) { T.qstatus[q] = VLS_ELOOPFAIL; continue; }
    // close along the handle loop: crossing edge i ending at b*, loop position j of the source reached
    const int32_t eo = T.heoff[q], m = T.hen[q];
    const int32_t bstar = path[0];
    int64_t bd = -1, bj = -1;
    int dir = 1;
    for (int32_t i = 0; i < m; ++i) {
      if (T.xedge[2 * (int64_t)(eo + i) + 1] != bstar) continue;
      for (int32_t j = 0; j < m; ++j) {
        if (T.xedge[2 * (int64_t)(eo + j)] != x) continue;
        const int64_t fwd = ((int64_t)(i - j) % m + m) % m, bwd = ((int64_t)(j - i) % m + m) % m;
        const int64_t dd = fwd <= bwd ? fwd : bwd;
        if (bd < 0 || dd < bd) { bd = dd; bj = j; dir = fwd <= bwd ? 1 : -1; }
      }
    }
    const int32_t off = atomicAdd(T.ntverts, np + (int32_t)(bd > 0 ? bd : 0));
    if (off + np + bd > T.tvcap) { T.qstatus[q] = VLS_ELAYERS; continue; }
    int32_t nc = 0;
    for (int32_t i = 0; i < np; ++i) T.tverts[off + nc++] = path[i] - voff;
    for (int64_t s = 1; s <= bd; ++s) {
      const int64_t ix = ((bj + dir * s) % m + m) % m;
      const int32_t a = T.xedge[2 * (int64_t)(eo + ix)] - voff;
      if (T.tverts[off + nc - 1] != a) T.tverts[off + nc++] = a;
    }
    while (nc > 1 && T.tverts[off + nc - 1] == T.tverts[off]) --nc;
    T.tvoff[q] = off;
    T.tvn[q] = nc;
  }
}

// ---- PL streamline (Sec. 3.2: the loop is traced back from the first point reached against the
// gradient of the arrival time).  The arrival time tfa is the step at which theta was crossed, with
// the fraction of that step found by linear interpolation in time (sources 0; unreached vertices
// have T < 0), interpolated linearly over the faces of the cut, restricted domain.  A face is
// usable when its three vertices are reached and none of its edges is cut.  In a face with corners
// (p0, p1, p2) the gradient is g = al e1 + be e2 (e1 = p1 - p0, e2 = p2 - p0), from the Gram
// system of e1, e2.  At a vertex the path enters the steepest (largest |g|, first in CSR order on
// ties) usable face around it whose corner there holds -g, and crosses it to the opposite edge;
// with none it follows the steepest descending kept edge.  On an edge it enters the face beyond if
// that face is usable and -g points into it, and leaves it where the ray meets its boundary; else
// it runs along the edge to its lower end (smaller arrival, then smaller id).  It ends at a source;
// a vertex with no descent left fails.  Points: the start, every edge crossing, every vertex
// passed; at most min(SL_MAX, nv / 4 + 64) with the closure for a mesh of nv vertices (the host lays
// out one region of that many points per pass).  Every product, sum and quotient is rounded on its
// own.
constexpr int32_t SL_MAX = 16384;

// CSR slot of u -> w: the row's columns compared all at once (one memory level for rows of up to 16)
__device__ __forceinline__ int32_t slot_scan(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t u,
                                             int32_t w) {
  const int32_t b = rp[u], e = rp[u + 1];
  if (e - b > 16) return slot_of(rp, col, u, w);
  int32_t k = -1;
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (b + j < e && col[b + j] == w) k = b + j;
  return k;
}

struct SlPass {
  const Dev &d;
  const TDev &T;
  int32_t q, base, voff;
  __device__ bool reached(int32_t v) const { return T.T[base + (v - voff)] >= 0; }
  __device__ double tf(int32_t v) const { return T.tfa[base + (v - voff)]; }
  __device__ bool cut(int32_t a, int32_t b, int32_t k) const {
    const int8_t fa = T.flag[base + (a - voff)], fb = T.flag[base + (b - voff)];
    if (((fa & F_SRC) && (fb & F_TGT)) || ((fa & F_TGT) && (fb & F_SRC))) return is_cut(T, q, k);
    return false;
  }
  // every vertex reached and no edge cut; only an edge between a source and a target can be cut,
  // so its slot is looked up only then (edges of a face always have slots in a validated mesh)
  __device__ bool usable(int32_t f) const {
    const int32_t *t = d.F + 3 * (int64_t)f;
    const int32_t a0 = t[0], a1 = t[1], a2 = t[2];
    const int32_t i0 = base + (a0 - voff), i1 = base + (a1 - voff), i2 = base + (a2 - voff);
    if (T.T[i0] < 0 || T.T[i1] < 0 || T.T[i2] < 0) return false;
    const int8_t f0 = T.flag[i0], f1 = T.flag[i1], f2 = T.flag[i2];
    if (((f0 | f1 | f2) & (F_SRC | F_TGT)) == 0) return true;
    const int32_t vv[3] = {a0, a1, a2};
    const int8_t ff[3] = {f0, f1, f2};
    for (int j = 0; j < 3; ++j) {
      const int jn = j == 2 ? 0 : j + 1;
      if (((ff[j] & F_SRC) && (ff[jn] & F_TGT)) || ((ff[j] & F_TGT) && (ff[jn] & F_SRC))) {
        const int32_t k = slot_scan(d.rp, d.col, vv[j], vv[jn]);
        if (k < 0 || is_cut(T, q, k)) return false;
      }
    }
    return true;
  }
  __device__ int32_t third(int32_t f, int32_t a, int32_t b) const {
    const int32_t *t = d.F + 3 * (int64_t)f;
    return (t[0] != a && t[0] != b) ? t[0] : (t[1] != a && t[1] != b) ? t[1] : t[2];
  }
  // gradient coefficients and |g|^2 of the arrival time on the face (p0, p1, p2)
  __device__ bool grad(int32_t p0, int32_t p1, int32_t p2, double &al, double &be, double &n2) const {
    const double *x0 = d.X + 3 * (int64_t)p0, *x1 = d.X + 3 * (int64_t)p1, *x2 = d.X + 3 * (int64_t)p2;
    double e1[3], e2[3];
    for (int j = 0; j < 3; ++j) {
      e1[j] = dsub(x1[j], x0[j]);
      e2[j] = dsub(x2[j], x0[j]);
    }
    const double g11 = dadd(dadd(dmul(e1[0], e1[0]), dmul(e1[1], e1[1])), dmul(e1[2], e1[2]));
    const double g12 = dadd(dadd(dmul(e1[0], e2[0]), dmul(e1[1], e2[1])), dmul(e1[2], e2[2]));
    const double g22 = dadd(dadd(dmul(e2[0], e2[0]), dmul(e2[1], e2[1])), dmul(e2[2], e2[2]));
    const double det = dsub(dmul(g11, g22), dmul(g12, g12));
    if (!(det > 0.0)) return false;
    const double t0 = tf(p0), d1 = dsub(tf(p1), t0), d2 = dsub(tf(p2), t0);
    al = ddiv(dsub(dmul(g22, d1), dmul(g12, d2)), det);
    be = ddiv(dsub(dmul(g11, d2), dmul(g12, d1)), det);
    n2 = dadd(dadd(dmul(dmul(al, al), g11), dmul(dmul(dadd(al, al), be), g12)), dmul(dmul(be, be), g22));
    return true;
  }
};

// point writer of a warp that traces in lock-step: every lane counts, lane 0 stores; at most lim
// points
struct SlOut {
  double *out;
  int32_t n, lim;
  bool writer;
  __device__ bool push(const double p[3]) {
    if (n >= lim) return false;
    if (writer) {
      out[3 * (int64_t)n] = p[0];
      out[3 * (int64_t)n + 1] = p[1];
      out[3 * (int64_t)n + 2] = p[2];
    }
    ++n;
    return true;
  }
  __device__ bool push_v(const Dev &d, int32_t v) { return push(d.X + 3 * (int64_t)v); }
};

// the trace from start; returns VLS_OK with the source reached in xs, or VLS_ELOOPFAIL
// (all lanes of a warp, in lock-step; lane = the caller's lane)
__device__ int32_t sl_trace(const SlPass &S, int32_t start, SlOut &o, int32_t &xs, int32_t lane) {
  const Dev &d = S.d;
  int32_t v = start, ex = -1, ey = -1;
  double mu = 0.0;
  bool at_vertex = true;
  o.push_v(d, v);
  for (int32_t it = 0; it < 4 * SL_MAX; ++it) {
    if (at_vertex) {
      if (S.T.T[S.base + (v - S.voff)] == 0) {
        xs = v;
        return VLS_OK;
      }
      // the faces around v, one half-edge per lane: each lane keeps its first steepest face, then the
      // warp takes the steepest, the smallest slot on ties (the first in CSR order)
      double best = -1.0, bal = 0.0, bbe = 0.0;
      int32_t bu = -1, bw = -1, bk = INT32_MAX;
      const int32_t kb = d.rp[v], ke = d.rp[v + 1];
      for (int32_t k0 = kb; k0 < ke; k0 += 32) {
        const int32_t k = k0 + lane;
        if (k >= ke) continue;
        const int32_t u = d.col[k], f = d.hface[k], w = S.third(f, v, u);
        double al, be, n2;
        if (!S.usable(f) || !S.grad(v, u, w, al, be, n2)) continue;
        if (!(al <= 0.0 && be <= 0.0 && (al < 0.0 || be < 0.0))) continue; // -g not into this corner
        if (n2 > best) {
          best = n2;
          bal = al;
          bbe = be;
          bu = u;
          bw = w;
          bk = k;
        }
      }
      {
        double wb = best;
        int32_t wk = bk;
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
          const double ob = __shfl_xor_sync(0xffffffffu, wb, o2);
          const int32_t ok = __shfl_xor_sync(0xffffffffu, wk, o2);
          if (ob > wb || (ob == wb && ok < wk)) {
            wb = ob;
            wk = ok;
          }
        }
        const int owner = wk == INT32_MAX ? 0 : (wk - kb) & 31;
        bal = __shfl_sync(0xffffffffu, bal, owner);
        bbe = __shfl_sync(0xffffffffu, bbe, owner);
        bu = __shfl_sync(0xffffffffu, bu, owner);
        bw = __shfl_sync(0xffffffffu, bw, owner);
        if (wk == INT32_MAX) bu = -1;
      }
      if (bu >= 0) {
        const double lam = ddiv(bbe, dadd(bal, bbe)); // where the ray meets edge u -> w, from u
        if (lam <= 0.0) {
          v = bu;
          if (!o.push_v(d, v)) break;
          continue;
        }
        if (lam >= 1.0) {
          v = bw;
          if (!o.push_v(d, v)) break;
          continue;
        }
        double p[3];
        const double *xu = d.X + 3 * (int64_t)bu, *xw = d.X + 3 * (int64_t)bw;
        for (int j = 0; j < 3; ++j) p[j] = dadd(xu[j], dmul(lam, dsub(xw[j], xu[j])));
        if (!o.push(p)) break;
        ex = bw;
        ey = bu;
        mu = dsub(1.0, lam); // into the face left of w -> u
        at_vertex = false;
        continue;
      }
      // the steepest descending kept edge, one half-edge per lane as above (ties: the first)
      double bs = 0.0;
      int32_t bn = -1, bk2 = INT32_MAX;
      const double *xv = d.X + 3 * (int64_t)v;
      for (int32_t k0 = kb; k0 < ke; k0 += 32) {
        const int32_t k = k0 + lane;
        if (k >= ke) continue;
        const int32_t u = d.col[k];
        if (S.cut(v, u, k) || !S.reached(u)) continue;
        const double *xu = d.X + 3 * (int64_t)u;
        const double dx = dsub(xu[0], xv[0]), dy = dsub(xu[1], xv[1]), dz = dsub(xu[2], xv[2]);
        const double sl = ddiv(dsub(S.tf(v), S.tf(u)), dsqrt(dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz))));
        if (sl > bs) {
          bs = sl;
          bn = u;
          bk2 = k;
        }
      }
      for (int o2 = 16; o2 > 0; o2 >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, bs, o2);
        const int32_t ok = __shfl_xor_sync(0xffffffffu, bk2, o2);
        if (ob > bs || (ob == bs && ok < bk2)) {
          bs = ob;
          bk2 = ok;
        }
      }
      bn = bk2 == INT32_MAX ? -1 : d.col[bk2];
      if (bn < 0) break; // no descent left
      v = bn;
      if (!o.push_v(d, v)) break;
      continue;
    }
    // on edge ex -> ey at mu from ex, entering the face left of it
    const int32_t k = slot_scan(d.rp, d.col, ex, ey);
    const int32_t f = k >= 0 ? d.hface[k] : -1, z = f >= 0 ? S.third(f, ex, ey) : -1;
    double al = 0.0, be = 0.0, n2 = 0.0;
    if (f < 0 || !S.usable(f) || !S.grad(ex, ey, z, al, be, n2) || !(be < 0.0)) {
      const double ta = S.tf(ex), tb = S.tf(ey);
      v = (ta < tb || (ta == tb && ex < ey)) ? ex : ey; // along the edge to its lower end
      at_vertex = true;
      if (!o.push_v(d, v)) break;
      continue;
    }
    // ray (u, w) = (mu - s al, -s be) in the frame (e1, e2) of the face (ex, ey, z)
    const double su = al > 0.0 ? ddiv(mu, al) : CUDART_INF;
    const double suw = dadd(al, be) < 0.0 ? ddiv(dsub(mu, 1.0), dadd(al, be)) : CUDART_INF;
    double p[3];
    if (su <= suw) { // leaves through the edge from ex to z
      const double w = -dmul(su, be);
      if (w >= 1.0) {
        v = z;
        at_vertex = true;
        if (!o.push_v(d, v)) break;
        continue;
      }
      if (w <= 0.0) {
        v = ex;
        at_vertex = true;
        if (!o.push_v(d, v)) break;
        continue;
      }
      const double *xa = d.X + 3 * (int64_t)ex, *xz = d.X + 3 * (int64_t)z;
      for (int j = 0; j < 3; ++j) p[j] = dadd(xa[j], dmul(w, dsub(xz[j], xa[j])));
      ey = z;
      mu = w; // into the face left of ex -> z
    } else { // leaves through the edge from ey to z
      const double w = -dmul(suw, be);
      if (w >= 1.0) {
        v = z;
        at_vertex = true;
        if (!o.push_v(d, v)) break;
        continue;
      }
      if (w <= 0.0) {
        v = ey;
        at_vertex = true;
        if (!o.push_v(d, v)) break;
        continue;
      }
      const double *xb = d.X + 3 * (int64_t)ey, *xz = d.X + 3 * (int64_t)z;
      for (int j = 0; j < 3; ++j) p[j] = dadd(xb[j], dmul(w, dsub(xz[j], xb[j])));
      ex = z;
      mu = dsub(1.0, w); // into the face left of z -> ey
    }
    if (!o.push(p)) break;
  }
  return VLS_ELOOPFAIL;
}

// closure along the border, as the vertex trace is closed: from the source reached, the shorter
// way along the border edges to one ending at the start
__device__ int32_t sl_close(const Dev &d, const TDev &T, int32_t q, int32_t bstar, int32_t xs, SlOut &o) {
  const int32_t eo = T.heoff[q], m = T.hen[q];
  int64_t bd = -1, bj = -1;
  int dir = 1;
  for (int32_t i = 0; i < m; ++i) {
    if (T.xedge[2 * (int64_t)(eo + i) + 1] != bstar) continue;
    for (int32_t j = 0; j < m; ++j) {
      if (T.xedge[2 * (int64_t)(eo + j)] != xs) continue;
      const int64_t fwd = ((int64_t)(i - j) % m + m) % m, bwd = ((int64_t)(j - i) % m + m) % m;
      const int64_t dd = fwd <= bwd ? fwd : bwd;
      if (bd < 0 || dd < bd) {
        bd = dd;
        bj = j;
        dir = fwd <= bwd ? 1 : -1;
      }
    }
  }
  if (bd < 0) return VLS_ELOOPFAIL;
  int32_t last = xs;
  for (int64_t s = 1; s <= bd; ++s) {
    const int64_t ix = ((bj + dir * s) % m + m) % m;
    const int32_t a = T.xedge[2 * (int64_t)(eo + ix)];
    if (a == last) continue;
    if (!o.push_v(d, a)) return VLS_ELAYERS;
    last = a;
  }
  return VLS_OK;
}

// one warp per pass whose vertex trace succeeded (the lanes share the vertex steps): the trace into
// the pass's region of the point pool (sroff), its status, point count and the closed polyline's
// length
constexpr int STREAM_WARPS = 4;
__global__ void __launch_bounds__(32 * STREAM_WARPS) k_tstream(Dev d, TDev T) {
  const int32_t q = blockIdx.x * STREAM_WARPS + (int32_t)(threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (q >= T.NP) return;
  if (T.qstatus[q] != VLS_OK) {
    if (lane == 0) {
      T.sst[q] = -1;
      T.sn[q] = 0;
    }
    return;
  }
  const int32_t p = T.pprob[q];
  const SlPass S{d, T, q, T.pbase[q], d.voff[p]};
  const int32_t start = S.voff + T.qbstar[q];
  double *P = T.sreg + 3 * (int64_t)T.sroff[q];
  SlOut o{P, 0, T.sroff[q + 1] - T.sroff[q], lane == 0};
  int32_t xs = -1;
  int32_t st = sl_trace(S, start, o, xs, lane);
  if (st == VLS_OK) st = sl_close(d, T, q, start, xs, o);
  __syncwarp();
  if (lane != 0) return;
  T.sst[q] = st;
  T.sn[q] = st == VLS_OK ? o.n : 0;
  if (st != VLS_OK) return;
  double len = 0.0;
  for (int32_t i = 0; i < o.n; ++i) {
    const double *a = P + 3 * (int64_t)i, *b = P + 3 * (int64_t)(i + 1 == o.n ? 0 : i + 1);
    const double dx = dsub(b[0], a[0]), dy = dsub(b[1], a[1]), dz = dsub(b[2], a[2]);
    len = dadd(len, dsqrt(dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz))));
  }
  T.slen[q] = len;
}

// one warp: offsets of the traced streamlines in the compact pool, in pass order; *nspts = points
__global__ void k_tstream_scan(TDev T) {
  const int32_t lane = threadIdx.x;
  int64_t run = 0;
  for (int32_t b0 = 0; b0 < T.NP; b0 += 32) {
    const int32_t q = b0 + lane;
    const int64_t c = q < T.NP && T.sst[q] == VLS_OK ? T.sn[q] : 0;
    int64_t inc = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (q < T.NP) T.soff[q] = (int32_t)(run + inc - c);
    run += __shfl_sync(0xffffffffu, inc, 31);
  }
  if (lane == 0) *T.nspts = (int32_t)run;
}

// one block per pass: its points from its region into the compact pool (whose capacity is the
// regions' total, so every traced streamline fits)
__global__ void k_tstream_compact(TDev T) {
  const int32_t q = blockIdx.x;
  if (q >= T.NP || T.sst[q] != VLS_OK) return;
  const double *src = T.sreg + 3 * (int64_t)T.sroff[q];
  double *dst = T.spts + 3 * (int64_t)T.soff[q];
  const int32_t n3 = 3 * T.sn[q];
  for (int32_t i = threadIdx.x; i < n3; i += blockDim.x) dst[i] = src[i];
}

__global__ void k_tctl_set(int32_t *ctl, int32_t idx, int32_t v) { ctl[idx] = v; }

}  // namespace

void configure_tunnel(Batch &b) {
  b.cfg[KK_TUPDATE] = b.opt.precision == VLS_BF16_RECHECK   ? row_cfg(b, k_tupdate<__nv_bfloat16>, KK_TUPDATE, 128)
                      : b.opt.precision == VLS_FP32_RECHECK ? row_cfg(b, k_tupdate<float>, KK_TUPDATE, 128)
                                                            : row_cfg(b, k_tupdate<double>, KK_TUPDATE, 128);
  b.cfg[KK_TAPPLY] = row_cfg(b, k_tapply, KK_TAPPLY, 128);
  b.cfg[KK_TFRONTIER] = row_cfg(b, k_tfrontier, KK_TFRONTIER, 256);
}

// Runs the passes of T (laid out by the host) on stream st: init, F_1, then one graph launch
// WHILE(passes running) { update; apply; next frontier; epilogue }, then the traces.  The step
// counter after the loop is copied to *tau_dst (host memory, pinned: the copy is asynchronous).  In
// the graph mode the instantiated graph goes to *ge_out; destroy it once st has run it.  With
// host-driven steps (b.host_loop) the call waits for the passes.
cudaError_t run_tunnels(Batch &b, const TDev &T, cudaStream_t st, int32_t *tau_dst, cudaGraphExec_t *ge_out) {
  Dev &d = b.d;
  *ge_out = nullptr;
  k_tinit<<<T.NP, 256, 0, st>>>(d, T, T.fv[0], T.fq[0], T.nf + 0); VLS_LAUNCH(b);
  k_tctl_set<<<1, 1, 0, st>>>(T.ctl, CTL_TAU, 0); VLS_LAUNCH(b);
  {
    Handles H0{};
    H0.use = 0;
    k_tfrontier<<<b.cfg[KK_TFRONTIER].grid, b.cfg[KK_TFRONTIER].threads, 0, st>>>(d, T, H0, b.opt.max_pass_steps, 0); VLS_LAUNCH(b);
  }
  cudaMemsetAsync(T.nf + 0, 0, sizeof(int32_t), st);
  k_tctl_set<<<1, 1, 0, st>>>(T.ctl, CTL_TAU, 1); VLS_LAUNCH(b);
  cudaError_t e = cudaSuccess;
  if (b.host_loop) {
    Handles H{};
    H.use = 0;
    const int sync_every = b.opt.sync_interval > 0 ? b.opt.sync_interval : 16;
    for (int32_t tau = 1;; ++tau) {
      long ps = b.prof.begin(st, KK_TUPDATE);
      if (T.phih) k_tupdate<__nv_bfloat16><<<b.cfg[KK_TUPDATE].grid, b.cfg[KK_TUPDATE].threads, 0, st>>>(d, T, b.prm);
      else if (T.phif) k_tupdate<float><<<b.cfg[KK_TUPDATE].grid, b.cfg[KK_TUPDATE].threads, 0, st>>>(d, T, b.prm);
      else k_tupdate<double><<<b.cfg[KK_TUPDATE].grid, b.cfg[KK_TUPDATE].threads, 0, st>>>(d, T, b.prm);
      VLS_LAUNCH(b);
      b.prof.end(st, ps);
      ps = b.prof.begin(st, KK_TAPPLY);
      k_tapply<<<b.cfg[KK_TAPPLY].grid, b.cfg[KK_TAPPLY].threads, 0, st>>>(d, T, b.prm.theta); VLS_LAUNCH(b);
      b.prof.end(st, ps);
      ps = b.prof.begin(st, KK_TFRONTIER);
      k_tfrontier<<<b.cfg[KK_TFRONTIER].grid, b.cfg[KK_TFRONTIER].threads, 0, st>>>(d, T, H, b.opt.max_pass_steps, 1); VLS_LAUNCH(b);
      b.prof.end(st, ps);
      if (tau % sync_every == 0) {
        int32_t act = 0;
        e = cudaMemcpyAsync(&act, T.ctl + CTL_TACTIVE, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        b.d2h += (int64_t)sizeof(int32_t);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        if (act == 0) break;
      }
    }
  } else {
    cudaGraph_t g = nullptr, body = nullptr;
    cudaGraphNode_t w, n0, n1, n2;
    Handles H{};
    H.use = 1;
    e = cudaGraphCreate(&g, 0);
    if (e == cudaSuccess) e = add_conditional(&w, g, nullptr, 0, cudaGraphCondTypeWhile, 1u, &H.loop, &body);
    if (e == cudaSuccess) e = add_kernel(&n0, body, nullptr, 0, T.phih ? k_tupdate<__nv_bfloat16> : T.phif ? k_tupdate<float> : k_tupdate<double>, dim3(b.cfg[KK_TUPDATE].grid), dim3(b.cfg[KK_TUPDATE].threads), d, T, b.prm);
    if (e == cudaSuccess) e = add_kernel(&n1, body, nullptr, 0, k_tapply, dim3(b.cfg[KK_TAPPLY].grid), dim3(b.cfg[KK_TAPPLY].threads), d, T, b.prm.theta);
    if (e == cudaSuccess) e = add_programmatic_edge(body, n0, n1);
    if (e == cudaSuccess)
      e = add_kernel(&n2, body, nullptr, 0, k_tfrontier, dim3(b.cfg[KK_TFRONTIER].grid), dim3(b.cfg[KK_TFRONTIER].threads), d, T, H,
                     b.opt.max_pass_steps, 1);
    if (e == cudaSuccess) e = add_programmatic_edge(body, n1, n2);
    cudaGraphExec_t ge = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, st);
    if (g) cudaGraphDestroy(g);
    *ge_out = ge;
    if (e != cudaSuccess) return e;
  }
  k_ttrace<<<(T.NP + 127) / 128, 128, 0, st>>>(d, T); VLS_LAUNCH(b);
  if (T.tfa) {
    k_tstream<<<(T.NP + STREAM_WARPS - 1) / STREAM_WARPS, 32 * STREAM_WARPS, 0, st>>>(d, T); VLS_LAUNCH(b);
    k_tstream_scan<<<1, 32, 0, st>>>(T); VLS_LAUNCH(b);
    k_tstream_compact<<<T.NP, 128, 0, st>>>(T); VLS_LAUNCH(b);
  }
  e = cudaMemcpyAsync(tau_dst, T.ctl + CTL_TAU, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  b.d2h += (int64_t)sizeof(int32_t);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace vls
