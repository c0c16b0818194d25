// initial.cu -- the initial pass (Sec. 3.1): per step
//   update   Eq. (2) explicit Euler step at every frontier row (Jacobi: reads the old state,
//            writes a per-row output), clamp, snap, column normalisation;
//   apply    the rows' new states go into the state: by the band count (below) on ordinary
//            steps, the band phases reading them from the update's vertex-indexed output
//            (nlay, nph); first of all, in the merge phase's body, on a step where several
//            layers meet at a row (merge candidates, Sec. 3.1), which also collects those rows;
//            cover steps are recorded with the scatter;
//   events   merges, then band labelling and splits / extinctions (events.cu);
//   frontier next frontier = vertices of the closed neighbourhood of this step's rows whose
//            own closed neighbourhood holds the base and at least one live layer (only
//            those can change: all rates of Eq. (2) vanish elsewhere);
//   epilogue per-problem termination, step limit, step records.
// A frontier row is one thread: the Laplacian of each layer is a sequential sum over the
// row in CSR order (diagonal last), the same rounding order as the FP64 oracle.
#include <type_traits>

#include "vls_batch.cuh"

namespace vls {

namespace {

__device__ __forceinline__ int32_t append(int32_t *counter) { return atomicAdd(counter, 1); }

// ------------------------------------------------------------------- update
// Neighbour states of a row are gathered into registers first (all loads of one level issued
// together: columns, then layer ids and values, then layer states), so a row costs a few
// memory latencies instead of one per neighbour and pass.  MAXD bounds the row length
// handled by one instantiation (16: registers; 64: local memory, rare).  TV is the stored
// value type: double (FP64 form) or float (FP32 form).

// FP64 row: Laplacian of every present layer and of the base, then Eq. (2).  Values of the
// FP32 form are widened exactly, so the row is the FP64 step from the stored inputs.
template <int MAXD, class TV>
__device__ __forceinline__ void row_f64(const Params &P, int nl, const int32_t *ls, int32_t lv, int32_t o, TV xv,
                                        const int32_t *nlay, const TV *nx, int32_t deg, double *out, double2 &mass,
                                        bool *unc = nullptr) {
  const double Lv = P.lv[deg];
  const double xvd = to_f64(xv);
  const double xb = dsub(1.0, lv != 0 ? xvd : 0.0);
  double x[KMAX], lap[KMAX];
#pragma unroll 1
  for (int q = 0; q < nl; ++q) {
    const int32_t l = ls[q];
    const double plat = (o != 0 && l == o) ? 1.0 : 0.0; // a plateau reads as the row's layer
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < MAXD; ++j) {
      if (j < deg) {
        const double psi = nlay[j] == l ? to_f64(nx[j]) : (nlay[j] < 0 ? plat : 0.0);
        // terms are >= 0 and acc starts at +0: skipping a zero term leaves acc bit-identical
        if (val_pos(psi)) acc = dadd(acc, dmul(Lv, psi));
      }
    }
    x[q] = (lv == l) ? xvd : 0.0;
    acc = dadd(acc, dmul(-P.s, x[q]));
    lap[q] = acc;
  }
  double accb = 0.0;
#pragma unroll
  for (int j = 0; j < MAXD; ++j)
    if (j < deg) {
      if (nlay[j] == 0) accb = dadd(accb, Lv);                                         // Lv * 1.0
      else if (val_lt1(nx[j])) accb = dadd(accb, dmul(Lv, dsub(1.0, to_f64(nx[j])))); // zero terms skipped
    }
  // mass check: m_v (L base)_v less the flux into frozen neighbours (never rows), and the
  // magnitude of its terms, sum_u base(u) + d base(v)
  double fzb = 0.0; // base held by frozen neighbours (a dead plateau holds none)
  int nfz = 0;
#pragma unroll
  for (int j = 0; j < MAXD; ++j)
    if (j < deg && nlay[j] < 0) {
      ++nfz;
      if (val_lt1(nx[j])) fzb += 1.0 - to_f64(nx[j]);
    }
  const double bnd = fzb - (double)nfz * xb;
  mass = make_double2(0.0, dadd(dmul(P.mv[deg], accb), dmul((double)deg, xb)));
  accb = dadd(accb, dmul(-P.s, xb));
  mass.x = dmul(P.mv[deg], accb) - bnd;
  if (!vertex_update(P, nl, x, lap, xb, accb, out, unc)) {
#pragma unroll
    for (int q = 0; q < KMAX; ++q)
      if (q < nl) out[q] = x[q];
  }
}

// FP32 row of the common case (one layer l and the base, Eq. (2) with n = 2).  Returns false
// when a decision of the step lies within the recheck margin (the row is then redone in FP64).
template <int MAXD, class TN>
__device__ __forceinline__ bool row_f32(const Params &P, int32_t l, int32_t lv, int32_t o, TN xvs,
                                        const int32_t *nlay, const TN *nx, int32_t deg, double &out,
                                        double2 &mass, bool &unc) {
  const float Lv = P.f_lv[deg];
  const float plat = (o != 0 && l == o) ? 1.f : 0.f;
  const float xv = to_f32(xvs);
  float acc = 0.f, accb = 0.f;
#pragma unroll
  for (int j = 0; j < MAXD; ++j)
    if (j < deg) {
      const float xj = to_f32(nx[j]);
      const float psi = nlay[j] == l ? xj : (nlay[j] < 0 ? plat : 0.f);
      acc = fmaf(Lv, psi, acc);
      accb = fmaf(Lv, nlay[j] == 0 ? 1.f : 1.f - xj, accb);
    }
  const float x = (lv == l) ? xv : 0.f;
  const float xb = 1.f - (lv != 0 ? xv : 0.f);
  const float lap = fmaf(-P.f_s, x, acc);
  const float lapb = fmaf(-P.f_s, xb, accb);
  // mass check (FP64 from the FP32 sums): m_v (L base)_v less the flux into frozen neighbours,
  // and the magnitude of its terms
  float fzb = 0.f; // base held by frozen neighbours (a dead plateau holds none: exact 0)
  int nfz = 0;
#pragma unroll
  for (int j = 0; j < MAXD; ++j)
    if (j < deg && nlay[j] < 0) {
      ++nfz;
      fzb += 1.f - to_f32(nx[j]);
    }
  const double bnd = (double)fzb - (double)nfz * (double)xb;
  mass = make_double2(P.mv[deg] * (double)lapb - bnd, P.mv[deg] * (double)accb + (double)deg * (double)xb);
  float y;
  if (!vertex_update_f32(P, x, lap, xb, lapb, y, unc)) return false;
  out = round_keep<TN>((double)y, P.theta); // exact for float storage
  return true;
}

// FP32 / BF16 forms: the FP64 redo of a row from its gathered inputs (rounded to the stored type
// keeping every threshold's side), out of line so that the hot row keeps few registers.  Rare: a
// collision or a decision within the margin.
template <int MAXD, class TN>
__device__ __noinline__ void row_redo(const Params &P, int nl, const int32_t *ls, int32_t lv, int32_t o, TN xv,
                                      const int32_t *nlay, const TN *nx, int32_t deg, double *out, double2 &mass,
                                      bool &unc) {
  row_f64<MAXD, TN>(P, nl, ls, lv, o, xv, nlay, nx, deg, out, mass, &unc);
  for (int q = 0; q < nl; ++q) out[q] = round_keep<TN>(out[q], P.theta);
}

// One frontier row.  FP32 form: the common case (one layer and the base) in FP32, a row that
// needs FP64 (several layers, or a decision within the margin) redone out of line from the same
// gathered inputs (FAST = true), or all in FP64 and rounded keeping every threshold's side
// (FAST = false: the out-of-line path of rows longer than the register path).  FP64 form: the
// FP64 row.
// Row outcome bits: redone in FP64, a decision within the drift bound of its threshold (uncertified).
enum RowOutcome : int { ROW_DONE = 0, ROW_REDONE = 1, ROW_UNCERT = 4 };

template <int MAXD, class TV, bool FAST>
__device__ __forceinline__ int update_row(const Dev &d, const Params &P, int32_t i, int32_t p, int32_t v, int32_t b,
                                          int32_t deg, double2 &mass) {
  const TV *__restrict__ ph = ph_arr<TV>(d);
  // nlay[j]: layer of neighbour j, 0 for the base only, -1 for a frozen plateau
  int32_t nlay[MAXD];
  TV nx[MAXD];
  {
    int32_t nu[MAXD];
#pragma unroll
    for (int j = 0; j < MAXD; ++j) nu[j] = (j < deg) ? d.col[b + j] : v;
#pragma unroll
    for (int j = 0; j < MAXD; ++j) {
      nlay[j] = (j < deg) ? d.lay[nu[j]] : 0;
      nx[j] = (j < deg) ? ph[nu[j]] : TV(0.0f);
    }
  }
  const int32_t lv = d.lay[v];
  const TV xv = ph[v];
#pragma unroll
  for (int j = 0; j < MAXD; ++j)
    if (j < deg && nlay[j] != 0 && frozen_state(d.lstate[nlay[j]])) nlay[j] = -1;
  const int32_t sv = lv != 0 ? d.lstate[lv] : 0;
  const int32_t o = (lv != 0 && sv == L_ALIVE) ? lv : 0;
  // layers present in the closed neighbourhood (ascending), base presence
  int32_t ls[KMAX];
  int nl = 0;
  bool hb = false, ovf = false;
  auto see = [&](int32_t lu, TV xu, int32_t su) {
    if (lu == 0) { hb = true; return; }
    if (frozen_state(su)) return; // a plateau reads as the row's own layer
    if (val_lt1(xu)) hb = true;
    bool dup = false;
    for (int q = 0; q < nl; ++q) dup |= (ls[q] == lu);
    if (dup) return;
    if (nl == KMAX) { ovf = true; return; }
    int q = nl++;
    while (q > 0 && ls[q - 1] > lu) { ls[q] = ls[q - 1]; --q; }
    ls[q] = lu;
  };
  see(lv, xv, sv);
#pragma unroll
  for (int j = 0; j < MAXD; ++j)
    if (j < deg) see(nlay[j] < 0 ? 1 : nlay[j], nx[j], nlay[j] < 0 ? (int32_t)L_DEAD : (int32_t)L_ALIVE);
  if (ovf) {
    atomicCAS(&d.pstatus[p], 0, (int32_t)VLS_ESLOTS);
    d.onl[i] = -1;
    row_new(d, v, lv, (double)xv);
    return ROW_DONE;
  }
  if (!hb || nl == 0) {
    d.onl[i] = -1;
    row_new(d, v, lv, (double)xv);
    return ROW_DONE;
  }
  double out[KMAX];
  int outcome = ROW_DONE;
  bool unc = false;
  if constexpr (!std::is_same<TV, double>::value && FAST) {
    // FP32 / BF16 forms: one layer in FP32; several layers (a collision: merge arithmetic
    // follows) and rows near a decision are redone in FP64 from copies of the gathered inputs
    // (only the copies live in local memory)
    if (nl != 1 || !row_f32<MAXD>(P, ls[0], lv, o, xv, nlay, nx, deg, out[0], mass, unc)) {
      int32_t cl[MAXD], cls[KMAX];
      TV cx[MAXD];
      double co[KMAX];
#pragma unroll
      for (int j = 0; j < MAXD; ++j) { cl[j] = nlay[j]; cx[j] = nx[j]; }
#pragma unroll
      for (int q = 0; q < KMAX; ++q) cls[q] = ls[q];
      unc = false;
      row_redo<MAXD>(P, nl, cls, lv, o, xv, cl, cx, deg, co, mass, unc);
#pragma unroll
      for (int q = 0; q < KMAX; ++q) out[q] = co[q];
      outcome = ROW_REDONE;
    }
  } else if constexpr (!std::is_same<TV, double>::value) {
    row_f64<MAXD, TV>(P, nl, ls, lv, o, xv, nlay, nx, deg, out, mass, &unc);
#pragma unroll
    for (int q = 0; q < KMAX; ++q)
      if (q < nl) out[q] = round_keep<TV>(out[q], P.theta);
    outcome = ROW_REDONE;
  } else {
    row_f64<MAXD, TV>(P, nl, ls, lv, o, xv, nlay, nx, deg, out, mass);
  }
  int cnt = 0;
  int32_t l1 = 0;
  double x1 = 0.0;
#pragma unroll
  for (int q = 0; q < KMAX; ++q)
    if (q < nl && out[q] > 0.0) {
      d.olay[(int64_t)i * KMAX + cnt] = ls[q];
      d.ophi[(int64_t)i * KMAX + cnt] = out[q];
      if (cnt == 0) {
        l1 = ls[q];
        x1 = out[q];
      }
      ++cnt;
    }
  d.onl[i] = cnt;
  row_new(d, v, l1, x1);
  if (cnt >= 2) { // several layers at the row: the merge phase runs (read by the update's last block)
    d.ctl[CTL_MERGE] = 1;
    __threadfence();
  }
  return outcome | (unc ? ROW_UNCERT : 0);
}

// Rows longer than the register path: out of line.
constexpr int ROW_REG = 12; // longest row of the register path (mesh degrees are 3..10)
template <class TV>
__device__ __noinline__ int update_row_wide(const Dev &d, const Params &P, int32_t i, int32_t p, int32_t v, int32_t b,
                                            int32_t deg, double2 &mass) {
  return update_row<64, TV, false>(d, P, i, p, v, b, deg, mass);
}
// Rows the common-case path leaves (several layers, a frozen neighbour, a decision near its
// threshold in the FP32 / BF16 forms): the general row, out of line.
template <class TV>
__device__ __noinline__ int update_row_general(const Dev &d, const Params &P, int32_t i, int32_t p, int32_t v,
                                               int32_t b, int32_t deg, double2 &mass) {
  return update_row<ROW_REG, TV, true>(d, P, i, p, v, b, deg, mass);
}

// FP64 row of the common case below (one live layer l0 and the base, no frozen neighbour): the
// operations of the general row for this case, in the same order.
template <class TV>
__device__ __forceinline__ double row_one_f64(const Params &P, int32_t l0, int32_t lv, TV xv, const int32_t *nlay,
                                              const TV *nx, int32_t deg, double2 &mass, bool *unc = nullptr) {
  const double Lv = P.lv[deg];
  const double xvd = to_f64(xv);
  const double xb = dsub(1.0, lv != 0 ? xvd : 0.0);
  double acc = 0.0, accb = 0.0;
#pragma unroll
  for (int j = 0; j < ROW_REG; ++j)
    if (j < deg) {
      const double psi = nlay[j] == l0 ? to_f64(nx[j]) : 0.0;
      if (val_pos(psi)) acc = dadd(acc, dmul(Lv, psi)); // zero terms skipped, as in the general row
    }
  const double x = lv == l0 ? xvd : 0.0;
  acc = dadd(acc, dmul(-P.s, x));
#pragma unroll
  for (int j = 0; j < ROW_REG; ++j)
    if (j < deg) {
      if (nlay[j] == 0) accb = dadd(accb, Lv);
      else if (val_lt1(nx[j])) accb = dadd(accb, dmul(Lv, dsub(1.0, to_f64(nx[j]))));
    }
  mass = make_double2(0.0, dadd(dmul(P.mv[deg], accb), dmul((double)deg, xb)));
  accb = dadd(accb, dmul(-P.s, xb));
  mass.x = dmul(P.mv[deg], accb);
  double out;
  if (!vertex_update(P, 1, &x, &acc, xb, accb, &out, unc)) out = x;
  return out;
}
// FP32 / BF16 forms: the FP64 redo of a common-case row from its gathered inputs, rounded to the
// stored type keeping every threshold's side; out of line (rare: a decision within the margin).
template <class TV>
__device__ __noinline__ double row_one_redo(const Params &P, int32_t l0, int32_t lv, TV xv, const int32_t *nlay,
                                            const TV *nx, int32_t deg, double2 &mass, bool &unc) {
  return round_keep<TV>(row_one_f64<TV>(P, l0, lv, xv, nlay, nx, deg, mass, &unc), P.theta);
}

// The common case, kept short: every non-base entry of the closed neighbourhood belongs to one
// live layer l0 (no collision, no frozen plateau next to the row), so Eq. (2) has n = 2 and the
// layer's state is read once instead of once per neighbour.  The arithmetic is exactly that of
// the general row for this case.  Returns ROW_GENERAL, having written nothing, for any other row.
constexpr int ROW_GENERAL = 2;
template <class TV>
__device__ __forceinline__ int update_row_fast(const Dev &d, const Params &P, int32_t i, int32_t v, int32_t b,
                                               int32_t deg, double2 &mass) {
  const TV *__restrict__ ph = ph_arr<TV>(d);
  int32_t nu[ROW_REG], nlay[ROW_REG];
  TV nx[ROW_REG];
#pragma unroll
  for (int j = 0; j < ROW_REG; ++j) nu[j] = (j < deg) ? d.col[b + j] : v;
  const int32_t lv = d.lay[v];
  const TV xv = ph[v];
#pragma unroll
  for (int j = 0; j < ROW_REG; ++j) {
    nlay[j] = (j < deg) ? d.lay[nu[j]] : 0;
    nx[j] = (j < deg) ? ph[nu[j]] : TV(0.0f);
  }
  int32_t l0 = lv;
  bool one = true, hb = lv == 0 || val_lt1(xv);
#pragma unroll
  for (int j = 0; j < ROW_REG; ++j)
    if (j < deg) {
      const int32_t lu = nlay[j];
      if (lu == 0) hb = true;
      else {
        if (l0 == 0) l0 = lu;
        one &= lu == l0;
        hb |= val_lt1(nx[j]);
      }
    }
  if (!one) return ROW_GENERAL;
  if (l0 == 0) { // the base alone: nothing changes
    d.onl[i] = -1;
    row_new(d, v, lv, (double)xv);
    return ROW_DONE;
  }
  if (d.lstate[l0] != L_ALIVE) return ROW_GENERAL;
  if (!hb) { // no base in the neighbourhood: nothing changes
    d.onl[i] = -1;
    row_new(d, v, lv, (double)xv);
    return ROW_DONE;
  }
  double out;
  int outcome = ROW_DONE;
  bool unc = false;
  if constexpr (std::is_same<TV, double>::value) {
    out = row_one_f64<TV>(P, l0, lv, xv, nlay, nx, deg, mass);
  } else if (!row_f32<ROW_REG>(P, l0, lv, lv, xv, nlay, nx, deg, out, mass, unc)) {
    int32_t cl[ROW_REG];
    TV cx[ROW_REG];
#pragma unroll
    for (int j = 0; j < ROW_REG; ++j) { cl[j] = nlay[j]; cx[j] = nx[j]; }
    unc = false;
    out = row_one_redo<TV>(P, l0, lv, xv, cl, cx, deg, mass, unc);
    outcome = ROW_REDONE;
  }
  if (unc) outcome |= ROW_UNCERT;
  if (out > 0.0) {
    d.olay[(int64_t)i * KMAX] = l0;
    d.ophi[(int64_t)i * KMAX] = out;
    d.onl[i] = 1;
    row_new(d, v, l0, out);
  } else {
    d.onl[i] = 0;
    row_new(d, v, 0, 0.0);
  }
  return outcome;
}

template <class TV>
__device__ __forceinline__ int update_one(const Dev &d, const Params &P, const int32_t *fv, int32_t i, int32_t p,
                                          double2 &mass) {
  if (__ldcg(d.pdone + p)) { d.onl[i] = -1; return ROW_DONE; } // nothing reads a finished problem's rows
  const int32_t v = fv[i];
  if (!VCHK(d.err, v, d.V, 101)) { d.onl[i] = -1; return ROW_DONE; }
  d.uf[v] = v; // the band labelling starts from singletons (only band rows are ever united)
  const int32_t b = d.rp[v], e = d.rp[v + 1];
  if (!VCHK(d.err, e, d.nnz + 1, 102) || !VCHK(d.err, b, e + 1, 103)) { d.onl[i] = -1; return ROW_DONE; }
  const int32_t deg = e - b;
  if (deg <= ROW_REG) {
    const int oc = update_row_fast<TV>(d, P, i, v, b, deg, mass);
    return oc != ROW_GENERAL ? oc : update_row_general<TV>(d, P, i, p, v, b, deg, mass);
  }
  if (deg <= 64) return update_row_wide<TV>(d, P, i, p, v, b, deg, mass);
  atomicCAS(&d.pstatus[p], 0, (int32_t)VLS_EINVAL);
  d.onl[i] = -1;
  row_new(d, v, d.lay[v], ph_ld(d, v));
  return ROW_DONE;
}

template <class TV>
__device__ __forceinline__ void update_rows(const Dev &d, const Params &P) {
  const int32_t cur = __ldcg(d.ctl + CTL_T) & 1;
  const int32_t *__restrict__ fv = d.front[cur];
  const int32_t *__restrict__ fp = d.front[cur] + d.V;
  const int32_t nF = __ldcg(d.nfront + cur);
  uint32_t redo = 0;
  const int32_t lane = (int32_t)(threadIdx.x & 31);
  const int32_t R = d.rpw;
  VLS_WARP_LOOP(w, R, nF) { // one row per lane of the first R lanes (as FOR_ROWS_R), then the warp's mass sums
    const int32_t i = w * R + lane;
    int32_t p = -1;
    double2 mass = make_double2(0.0, 0.0);
    bool unc = false;
    if (lane < R && i < nF) {
      p = fp[i];
      const int oc = update_one<TV>(d, P, fv, i, p, mass);
      redo += (oc & ROW_REDONE) != 0;
      unc = (oc & ROW_UNCERT) != 0;
    }
    mass_sums(d.pmass, d.mslots, p, lane, mass);
    if constexpr (!std::is_same<TV, double>::value) {
      count_keyed(d.punc, p, unc);
      count_keyed(d.runc, p, unc);
    }
  }
  if constexpr (!std::is_same<TV, double>::value) {
    redo = __reduce_add_sync(0xffffffffu, redo);
    if ((threadIdx.x & 31) == 0 && redo) atomicAdd(&d.nrecheck[0], (unsigned long long)redo);
  }
}

// One instantiation per stored value type, so that each form gets its own register budget.  The
// last block decides whether the merge phase (with the scatter first) runs this step.
template <class TV>
__global__ void __launch_bounds__(256, VLS_UPDATE_MINB) k_update(Dev d, Params P, Handles H) {
  update_rows<TV>(d, P);
  if (last_block_done_fenced(d.ctl + CTL_DONE_APPLY)) {
    const int32_t m = __ldcg(d.ctl + CTL_MERGE);
    if (H.use) cudaGraphSetConditional(H.merge, m ? 1u : 0u);
    if (m) d.ctl[CTL_NMERGE]++;
    d.ctl[CTL_MERGE] = 0;
    d.ctl[CTL_APPLIED] = m ? 1 : 0;
  }
}

// ------------------------------------------------------------------- apply
// A merge step (first node of the merge phase's body): every row into the state, and the rows
// where several layers meet collected for the merge phase.  On other steps the band count does
// the scatter (apply returns at once: it is launched every step only in the host-driven loop).
__device__ __forceinline__ void apply_phase(const Dev &d) {
  const int32_t t = __ldcg(d.ctl + CTL_T), cur = t & 1;
  const int32_t *__restrict__ fv = d.front[cur];
  const int32_t *__restrict__ fp = d.front[cur] + d.V;
  const int32_t nF = __ldcg(d.nfront + cur);
  if (!__ldcg(d.ctl + CTL_APPLIED)) return;
  FOR_ROWS_R(i, nF, d.rpw) {
    const int32_t v = fv[i];
    const int32_t c = d.onl[i];
    if (c < 0) continue;
    if (c == 0) {
      d.lay[v] = 0;
      ph_st(d, v, 0.0);
    } else {
      d.lay[v] = d.olay[(int64_t)i * KMAX];
      ph_st(d, v, d.ophi[(int64_t)i * KMAX]);
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
__global__ void k_apply(Dev d) { apply_phase(d); }

// ------------------------------------------------------------------- band labelling
__device__ __forceinline__ bool is_band(const Dev &d, int32_t v, int32_t &l) {
  l = d.lay[v];
  if (l == 0 || d.lstate[l] != L_ALIVE) return false;
  return ph_band(d, v);
}
// the same on this step's new state of a frontier row (before the scatter)
__device__ __forceinline__ bool is_band_new(const Dev &d, int32_t v, int32_t &l, bool applied) {
  if (applied) return is_band(d, v, l);
  l = d.nlay[v];
  if (l == 0 || d.lstate[l] != L_ALIVE) return false;
  return nph_band(d, v);
}

__device__ __forceinline__ void hook_phase(const Dev &d) {
  const int32_t t = __ldcg(d.ctl + CTL_T), cur = t & 1;
  const int32_t *__restrict__ fv = d.front[cur];
  const int32_t *__restrict__ fp = d.front[cur] + d.V;
  const int32_t nF = __ldcg(d.nfront + cur);
  const int32_t lane = group_lane();
  const bool applied = __ldcg(d.ctl + CTL_APPLIED) != 0;
  // GL lanes per band row, one neighbour each: a neighbour joins the row's band component iff
  // it is a frontier row of this step (band vertices are) holding the same live layer strictly
  // between 0 and 1 in its new state; the smaller id of each such pair unites
  FOR_ROWS_G(i, nF) {
    if (__ldcg(d.pdone + fp[i])) continue;
    const int32_t v = fv[i];
    int32_t l;
    if (!is_band_new(d, v, l, applied)) continue;
    const int32_t b = d.rp[v], e = d.rp[v + 1];
    for (int32_t k = b + lane; k < e; k += GL) {
      const int32_t u = d.col[k];
      if (!VCHK(d.err, u, d.V, 130)) continue;
      const int32_t fm = d.fmark[u], lu = applied ? d.lay[u] : d.nlay[u];
      const bool bu = applied ? ph_band(d, u) : nph_band(d, u);
      if (u < v && fm == t && lu == l && bu) uf_unite(d.uf, u, v);
    }
  }
}
__global__ void k_band_hook(Dev d) {
  pdl_enter();
  hook_phase(d);
}

// The other union-find variant: one thread per band row unites the row with each qualifying
// neighbour in turn (neighbour states gathered first).
__global__ void k_band_hook_row(Dev d) {
  pdl_enter();
  const int32_t t = __ldcg(d.ctl + CTL_T), cur = t & 1;
  const int32_t *__restrict__ fv = d.front[cur];
  const int32_t *__restrict__ fp = d.front[cur] + d.V;
  const int32_t nF = __ldcg(d.nfront + cur);
  const bool applied = __ldcg(d.ctl + CTL_APPLIED) != 0;
  FOR_ROWS_R(i, nF, d.rpw) {
    if (__ldcg(d.pdone + fp[i])) continue;
    const int32_t v = fv[i];
    int32_t l;
    if (!is_band_new(d, v, l, applied)) continue;
    const int32_t b = d.rp[v], deg = d.rp[v + 1] - b;
    if (deg <= 16) {
      int32_t nu[16], nm[16], nl[16];
      bool nb[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) nu[j] = (j < deg) ? d.col[b + j] : v;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const bool ok = j < deg && nu[j] < v;
        nm[j] = ok ? d.fmark[nu[j]] : -1;
        nl[j] = ok ? (applied ? d.lay[nu[j]] : d.nlay[nu[j]]) : 0;
        nb[j] = ok && (applied ? ph_band(d, nu[j]) : nph_band(d, nu[j]));
      }
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (nm[j] == t && nl[j] == l && nb[j]) uf_unite(d.uf, nu[j], v);
    } else {
      for (int32_t k = b; k < b + deg; ++k) {
        const int32_t u = d.col[k];
        if (!VCHK(d.err, u, d.V, 131)) continue;
        if (u >= v || d.fmark[u] != t) continue;
        int32_t lu;
        if (is_band_new(d, u, lu, applied) && lu == l) uf_unite(d.uf, u, v);
      }
    }
  }
}

// Component roots per layer.  A layer reaching two roots, or a problem with a live layer
// that has no root (no band left), sends the step through the split phase.
// Also the scatter of the step's rows into (lay, phi) and their cover steps, unless a merge step
// did it before the band phases.
__device__ __forceinline__ void count_phase(const Dev &d) {
  const int32_t t = __ldcg(d.ctl + CTL_T), cur = t & 1;
  const int32_t *__restrict__ fv = d.front[cur];
  const int32_t *__restrict__ fp = d.front[cur] + d.V;
  const int32_t nF = __ldcg(d.nfront + cur);
  const bool applied = __ldcg(d.ctl + CTL_APPLIED) != 0;
  FOR_ROWS_R(i, nF, d.rpw) {
    const int32_t p = fp[i];
    if (__ldcg(d.pdone + p)) continue;
    const int32_t v = fv[i];
    int32_t l;
    const bool band = is_band_new(d, v, l, applied);
    if (!applied) {
      row_scatter(d, v);
      if (d.nlay[v] != 0 && d.cover[v] < 0) d.cover[v] = t;
    }
    if (!band) continue;
    if (__ldcg(d.uf + v) == v) { // hooking is complete: roots are exactly the self-parents
      const int32_t old = atomicAdd(&d.lcnt[l], 1);
      if (old == 0) atomicAdd(&d.nbl[p], 1);
      else if (old == 1) d.ctl[CTL_SPLIT] = 1;
      __threadfence(); // read by the last block
    }
  }
}
__global__ void k_band_count(Dev d, Handles H) {
  pdl_enter();
  count_phase(d);
  if (last_block_done_fenced(d.ctl + CTL_DONE_COUNT)) {
    int32_t s = __ldcg(d.ctl + CTL_SPLIT);
    for (int32_t p = 0; p < d.P && !s; ++p)
      if (!d.pdone[p] && __ldcg(d.nbl + p) != d.nalive[p]) s = 1;
    if (H.use) cudaGraphSetConditional(H.split, s ? 1u : 0u);
    if (s) d.ctl[CTL_NSPLIT]++;
    d.ctl[CTL_SPLIT] = 0;
  }
}

// ------------------------------------------------------------------- next frontier
// F_{t+1} = the vertices, not frozen, whose closed neighbourhood holds the base and a live
// layer (only those can change: all rates of Eq. (2) vanish elsewhere).  gives(w) is what w
// contributes to such a test: bit 0 the base (no layer, or a live layer below 1), bit 1 a
// live layer; a frozen plateau contributes nothing.  A vertex u qualifies iff gives(u) = 3 or
// some neighbour w has gives(u) | gives(w) = 3, and every such pair has an endpoint in F_t:
// a pair with neither endpoint in F_t kept its values through step t, so it qualified at the
// end of step t - 1 already and put both endpoints into F_t (events only take contributions
// away: a split freezes a plateau, an extinction ends a layer, a merge relabels live layers).
// So F_{t+1} is found from the pairs (v, u), v in F_t, u a neighbour of v: O(degree) per row.
__device__ __forceinline__ uint32_t gives(const Dev &d, int32_t w) {
  const int32_t l = d.lay[w];
  const bool lt1 = ph_lt1(d, w);
  if (l == 0) return 1u;
  if (frozen_state(d.lstate[l])) return 0u;
  return lt1 ? 3u : 2u;
}

// F_t -> F_{t+1}: a group of GL lanes per row, lane j takes the row's neighbour j (rows longer
// than GL loop); the row itself joins when it qualifies on its own or through any pair.  Also
// clears the per-layer root counts of this step (each band root resets its layer's counter) and
// accumulates the step record.
// Returns true in the threads that wrote something the step's epilogue reads (list counts, step
// records).
__device__ __forceinline__ bool frontier_phase(const Dev &d) {
  const int32_t t = __ldcg(d.ctl + CTL_T), cur = t & 1, nxt = cur ^ 1, tnext = t + 1;
  const int32_t *__restrict__ fv = d.front[cur];
  const int32_t *__restrict__ fp = d.front[cur] + d.V;
  const int32_t nF = __ldcg(d.nfront + cur);
  int32_t *__restrict__ nv_out = d.front[nxt];
  int32_t *__restrict__ np_out = d.front[nxt] + d.V;
  int32_t *nN_ptr = d.nfront + nxt;
  int32_t *pcount_next = d.pfront + (size_t)nxt * d.P;
  const int32_t lane = group_lane();
  const unsigned grp = group_mask();
  int32_t *__restrict__ seg_out = d.fseg[nxt];
  bool wrote = false;
  auto add = [&](int32_t u, int32_t p) {
    wrote = true;
    if (atomicExch(&d.stamp[u], tnext) == tnext) return;
    int32_t ks;
    const int32_t s = warp_append(nN_ptr, pcount_next, p, &ks);
    if (!VCHK(d.err, s, d.V, 121)) return;
    nv_out[s] = u;
    np_out[s] = p;
    d.fmark[u] = tnext;
    const int32_t j = d.voff[p] + ks;
    if (VCHK(d.err, j, d.voff[p + 1], 122)) seg_out[j] = u;
  };
  FOR_ROWS_G(i, nF) {
    const int32_t p = fp[i];
    if (__ldcg(d.pdone + p)) continue;
    const int32_t v = fv[i];
    if (lane == 0) {
      int32_t l;
      if (is_band(d, v, l)) {
        if (d.uf[v] == v) d.lcnt[l] = 0;
        if (d.record) {
          wrote = true;
          atomicAdd(&d.rband[p], 1);
          const uint64_t key = ((uint64_t)(uint32_t)(v - d.voff[p]) << 32) | (uint32_t)(l - d.lbase[p]);
          atomicAdd(&d.rhash[p], (unsigned long long)mix64(key));
        }
      }
    }
    const uint32_t gv = gives(d, v);
    const int32_t b = d.rp[v], e = d.rp[v + 1];
    bool join = gv == 3u;
    for (int32_t k0 = b; k0 < e; k0 += GL) {
      const int32_t k = k0 + lane;
      if (k >= e) continue;
      const int32_t u = d.col[k];
      if (!VCHK(d.err, u, d.V, 120)) continue;
      const uint32_t gu = gives(d, u);
      if ((gv | gu) != 3u) continue;
      join = true;
      if (gu != 0u) add(u, p);
    }
    join = __any_sync(grp, join) && gv != 0u;
    if (lane == 0 && join) add(v, p);
  }
  return wrote;
}

// ------------------------------------------------------------------- epilogue
// One block: per-problem bookkeeping, then the step counter advances; the WHILE node stops
// when no problem is running (or at the hard step bound).
__device__ __forceinline__ void epilogue_phase(const Dev &d, const Handles &H, int32_t max_steps) {
  __shared__ int32_t nact;
  const int32_t t = __ldcg(d.ctl + CTL_T), cur = t & 1, nxt = cur ^ 1;
  int32_t *pcount_cur = d.pfront + (size_t)cur * d.P;
  int32_t *pcount_next = d.pfront + (size_t)nxt * d.P;
  if (threadIdx.x == 0) nact = 0;
  __syncthreads();
  for (int32_t p = threadIdx.x; p < d.P; p += blockDim.x) {
    if (!__ldcg(d.pdone + p)) {
      d.psteps[p] = t;
      d.pupd[p] += __ldcg(pcount_cur + p);
      if (d.record && t - 1 < d.rcap) {
        long long *r = d.rec + ((int64_t)p * d.rcap + (t - 1)) * 5;
        const unsigned long long h = __ldcg(d.rhash + p);
        r[0] = __ldcg(pcount_cur + p);
        r[1] = __ldcg(d.rband + p);
        r[2] = (long long)(h & 0xffffffffull);
        r[3] = (long long)(h >> 32);
        r[4] = __ldcg(d.runc + p);
      }
      d.runc[p] = 0;
      d.rband[p] = 0;
      d.rhash[p] = 0ull;
      {
        // mass check of this step's diffusion: the base's Laplacian weighted by the lumped
        // masses, less the flux into frozen neighbours, sums to zero over the rows that can
        // change (every other non-frozen vertex next to a row holds that row's base value); the
        // FP64 residual relative to the terms' magnitude
        d.pmres[p] = fmax(d.pmres[p], mass_fold(d.pmass, d.mslots, p));
      }
      if (__ldcg(d.pstatus + p) != 0) d.pdone[p] = 1;
      else if (__ldcg(pcount_next + p) == 0) d.pdone[p] = 1;
      else if (t >= max_steps) { d.pstatus[p] = VLS_EMAXSTEPS; d.pdone[p] = 1; }
      if (!d.pdone[p]) atomicAdd(&nact, 1);
    }
    pcount_cur[p] = 0;
    d.pmerge[p] = 0;
    d.nbl[p] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    d.ctl[CTL_ACTIVE] = nact;
    d.nfront[cur] = 0; // the list just consumed is reused two steps later
    *d.ncoll = 0;
    d.ctl[CTL_APPLIED] = 0;
    d.ctl[CTL_T] = t + 1;
    if (H.use && (nact == 0 || t >= d.ctl[CTL_LIMIT])) cudaGraphSetConditional(H.loop, 0u);
  }
}
// The next frontier, then (epi = 1) the step's epilogue in the last block to finish.
__global__ void __launch_bounds__(256) k_frontier(Dev d, Handles H, int32_t max_steps, int32_t epi) {
  const bool wrote = frontier_phase(d);
  if (!epi) return;
  if (wrote) __threadfence(); // the epilogue reads the list counts and step records
  if (last_block_fenced(d.ctl + CTL_DONE_FRONT)) epilogue_phase(d, H, max_steps);
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
    d.nalive[p] = 1;
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
      ph_st(d, u, 1.0);
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
    if (d.lay[v] == 0 || ph_lt1(d, v)) pstall[prob_of_vertex(d.voff, d.P, v)] = 1;
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

__global__ void k_ctl_set(int32_t *ctl, int32_t idx, int32_t v) { ctl[idx] = v; }

}  // namespace

// The frontier lists alternate: list (t & 1) holds F_t.  The seed regions form F_0 and the
// frontier kernel run at t = 0 builds F_1.
cudaError_t init_state(Batch &b) {
  Dev &d = b.d;
  cudaStream_t st = b.st;
  k_init<<<(b.P + 127) / 128, 128, 0, st>>>(d, d.front[0], d.front[0] + b.V, d.nfront + 0); VLS_LAUNCH(b);
  {
    Handles H{};
    H.use = 0;
    k_frontier<<<b.cfg[KK_FRONTIER].grid, b.cfg[KK_FRONTIER].threads, 0, st>>>(d, H, b.opt.max_steps, 0); VLS_LAUNCH(b);
  }
  cudaMemsetAsync(d.nfront + 0, 0, sizeof(int32_t), st);
  k_ctl_set<<<1, 1, 0, st>>>(d.ctl, CTL_T, 1); VLS_LAUNCH(b);
  return cudaGetLastError();
}

// The initial pass as one graph: WHILE(problems running) { update; IF(merge) { apply; ... };
// band hook; band count (and the scatter); IF(split / extinction) {...}; next frontier; epilogue }.
cudaError_t build_initial_graph(Batch &b, cudaGraph_t *out) {
  cudaGraph_t g = nullptr, body = nullptr, mbody = nullptr, sbody = nullptr;
  cudaGraphNode_t w, n_upd, n_app, n_if_m, n_hook, n_cnt, n_if_s, n_fr;
  Handles H{};
  H.use = 1;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  auto G = [&](int k) { return dim3(b.cfg[k].grid); };
  auto T = [&](int k) { return dim3(b.cfg[k].threads); };
#define GK(x)                         \
  do {                                \
    e = (x);                          \
    if (e != cudaSuccess) goto fail;  \
  } while (0)
  GK(add_conditional(&w, g, nullptr, 0, cudaGraphCondTypeWhile, 1u, &H.loop, &body));
  GK(cudaGraphConditionalHandleCreate(&H.merge, body, 0u, cudaGraphCondAssignDefault));
  GK(cudaGraphConditionalHandleCreate(&H.split, body, 0u, cudaGraphCondAssignDefault));
  GK(add_kernel(&n_upd, body, nullptr, 0, b.d.phih ? k_update<__nv_bfloat16> : b.d.phif ? k_update<float> : k_update<double>,
                G(KK_UPDATE), T(KK_UPDATE),
                b.d, b.prm, H));
  {
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = H.merge;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    GK(cudaGraphAddNode(&n_if_m, body, &n_upd, nullptr, 1, &np));
    mbody = np.conditional.phGraph_out[0];
    GK(add_kernel(&n_app, mbody, nullptr, 0, k_apply, G(KK_APPLY), T(KK_APPLY), b.d));
    GK(add_merge_nodes(b, mbody, &n_app));
  }
  GK(add_kernel(&n_hook, body, &n_if_m, 1, b.hook_variant == 1 ? k_band_hook_row : k_band_hook, G(KK_HOOK), T(KK_HOOK),
                b.d));
  GK(add_kernel(&n_cnt, body, nullptr, 0, k_band_count, G(KK_COUNT), T(KK_COUNT), b.d, H));
  GK(add_programmatic_edge(body, n_hook, n_cnt));
  {
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = H.split;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    GK(cudaGraphAddNode(&n_if_s, body, &n_cnt, nullptr, 1, &np));
    sbody = np.conditional.phGraph_out[0];
    GK(add_split_nodes(b, sbody));
  }
  GK(add_kernel(&n_fr, body, &n_if_s, 1, k_frontier, G(KK_FRONTIER), T(KK_FRONTIER), b.d, H, b.opt.max_steps, 1));
#undef GK
  *out = g;
  return cudaSuccess;
fail:
  cudaGraphDestroy(g);
  return e;
}

// Debug path: the same kernels launched one step at a time from the host (the event phases
// run every step; their kernels return at once when nothing happened).
cudaError_t initial_step_host(Batch &b) {
  Dev &d = b.d;
  cudaStream_t st = b.st;
  Handles H{};
  H.use = 0;
  long ps = b.prof.begin(st, KK_UPDATE);
  if (d.phih) k_update<__nv_bfloat16><<<b.cfg[KK_UPDATE].grid, b.cfg[KK_UPDATE].threads, 0, st>>>(d, b.prm, H);
  else if (d.phif) k_update<float><<<b.cfg[KK_UPDATE].grid, b.cfg[KK_UPDATE].threads, 0, st>>>(d, b.prm, H);
  else k_update<double><<<b.cfg[KK_UPDATE].grid, b.cfg[KK_UPDATE].threads, 0, st>>>(d, b.prm, H);
  VLS_LAUNCH(b);
  b.prof.end(st, ps);
  ps = b.prof.begin(st, KK_APPLY);
  k_apply<<<b.cfg[KK_APPLY].grid, b.cfg[KK_APPLY].threads, 0, st>>>(d); VLS_LAUNCH(b);
  b.prof.end(st, ps);
  cudaError_t e = merge_phase_host(b);
  if (e != cudaSuccess) return e;
  ps = b.prof.begin(st, KK_HOOK);
  if (b.hook_variant == 1) k_band_hook_row<<<b.cfg[KK_HOOK].grid, b.cfg[KK_HOOK].threads, 0, st>>>(d);
  else k_band_hook<<<b.cfg[KK_HOOK].grid, b.cfg[KK_HOOK].threads, 0, st>>>(d);
  VLS_LAUNCH(b);
  b.prof.end(st, ps);
  ps = b.prof.begin(st, KK_COUNT);
  k_band_count<<<b.cfg[KK_COUNT].grid, b.cfg[KK_COUNT].threads, 0, st>>>(d, H); VLS_LAUNCH(b);
  b.prof.end(st, ps);
  e = split_phase_host(b);
  if (e != cudaSuccess) return e;
  ps = b.prof.begin(st, KK_FRONTIER);
  k_frontier<<<b.cfg[KK_FRONTIER].grid, b.cfg[KK_FRONTIER].threads, 0, st>>>(d, H, b.opt.max_steps, 1); VLS_LAUNCH(b);
  b.prof.end(st, ps);
  return cudaGetLastError();
}

void configure_initial(Batch &b) {
  // one thread per frontier row
  b.cfg[KK_UPDATE] = b.opt.precision == VLS_BF16_RECHECK   ? row_cfg(b, k_update<__nv_bfloat16>, KK_UPDATE, 128)
                     : b.opt.precision == VLS_FP32_RECHECK ? row_cfg(b, k_update<float>, KK_UPDATE, 128)
                                                           : row_cfg(b, k_update<double>, KK_UPDATE, 128);
  b.cfg[KK_APPLY] = row_cfg(b, k_apply, KK_APPLY, 128);
  b.cfg[KK_HOOK] = b.hook_variant == 1 ? row_cfg(b, k_band_hook_row, KK_HOOK, 128) : row_cfg(b, k_band_hook, KK_HOOK, 256);
  b.cfg[KK_COUNT] = row_cfg(b, k_band_count, KK_COUNT, 128);
  b.cfg[KK_FRONTIER] = row_cfg(b, k_frontier, KK_FRONTIER, 256); // GL lanes per row
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
