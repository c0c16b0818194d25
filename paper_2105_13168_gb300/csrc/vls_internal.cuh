// vls_internal.cuh -- device-side data layout and helpers of the GB300 loop-shrinking library.
//
// Layout (one "batch" = P problems; problem = (mesh, seed vertex)):
//   The batch is a disjoint union graph: problem p owns vertices [voff[p], voff[p+1]) and
//   faces [foff[p], foff[p+1]) with global vertex ids, so every frontier kernel works on
//   global ids and needs the problem id only for rare events.  Meshes shared by several
//   seeds are replicated (state is per problem anyway).
//   Per vertex (structure-of-arrays, 4/8-byte aligned, coalesced by vertex id):
//     rp[V+1], col[nnz], hface[nnz]   CSR of the half-edges v->col (ascending col), the
//                                     face holding half-edge v->col (closed oriented mesh)
//     lay[V] int32                    layer id held (global id, 0 = base only)
//     phi[V] double                   its value; the base is implicit: 1 - phi (Sec. 2)
//     cover[V] int32                  first step the vertex left the pure base (-1 never)
//   Each vertex holds at most one non-base layer at a step boundary: merges are resolved
//   within the step (Sec. 3.1), so the transient co-presence of several layers at a vertex
//   lives only in the per-frontier-row output buffer (KMAX entries per row).
//   Layers have global ids; problem p owns [lbase[p], lbase[p] + lcap[p]); local id =
//   global - lbase[p] (1 = seed layer, then creation order).
#pragma once
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vls.h"

namespace vls {

constexpr int KMAX = 4;            // non-base layers that may meet at one vertex in one step
constexpr int MAX_GROUP = 32;      // layers in one merge group
constexpr int MAX_TRACES = 64;     // isoline traces per round of the merge phase (all problems)
constexpr int TRACE_CAP = 1 << 16; // crossing edges per traced isoline
constexpr int MASS_SLOTS = 16;     // accumulators per problem of the mass check (power of two)
constexpr int MASS_SPREAD_MAXP = 64; // batches of at most this many problems spread them

enum LayerState : int32_t { L_UNUSED = 0, L_ALIVE = 1, L_DEAD = 2, L_MERGED = 3, L_ENDED = 4 };
enum NodeKind : int32_t { N_SEED = 0, N_SPLIT = 1, N_MERGE = 2, N_END = 3 };

constexpr int LV_MAX = 64; // longest row of the register / local-memory row paths

// Minimum resident blocks of 256 threads per SM that the frontier-update kernels are compiled
// for (it caps their registers: 2 -> 128, 3 -> 80, 4 -> 64 per thread).  The rows are chains of
// dependent gathers, so more resident warps hide more of their latency.
#ifndef VLS_UPDATE_MINB
#define VLS_UPDATE_MINB 3
#endif

struct Params {
  double mu, e, w, ah, dt, s, eps0, one_m_eps, theta;
  double lv[LV_MAX + 1];  // s / d: off-diagonal operator entry of a row with d kept neighbours
  double mun[KMAX + 2];   // mu / n for n phases meeting at a vertex
  double mv[LV_MAX + 1];  // d / s: lumped mass of a row with d neighbours (m_v L_vu = 1, symmetric)
  // FP32 form: the same constants rounded to float, and the recheck margin
  double margin;
  double offset;          // loop classification: normal offset in mean edge lengths (Sec. 3.5)
  double drift;           // FP32 / BF16 forms: a decision whose FP64 value lies within this of its
                          // threshold is counted uncertified (0 in the FP64 form)
  float f_e, f_w, f_ah, f_dt, f_s, f_eps0, f_one_m_eps, f_theta, f_margin, f_drift;
  float f_lv[LV_MAX + 1];
  float f_mun[KMAX + 2];
};

// Global device state of one batch.  Passed by value to kernels.
struct Dev {
  int32_t P;
  int32_t V;
  int32_t NF;
  int64_t nnz;
  int32_t Lcap;
  const double *X;
  const int32_t *F;
  int32_t *rp, *col, *hface;
  // problem tables
  const int32_t *voff, *foff, *lbase, *lcap, *seed;
  int32_t *lcount;   // layers created per problem (local ids 1..lcount)
  int32_t *pstatus;  // per-problem status
  int32_t *pdone;    // 1 when the initial pass of p ended
  int32_t *psteps;   // steps executed per problem
  int32_t *pnodes;   // Reeb nodes per problem
  int32_t *pfront;   // frontier rows per problem of the list being built
  int32_t *pmerge;   // 1 if p has a merge this step
  int64_t *pupd;     // row updates per problem
  int32_t *pev;      // [P][3] merges, splits, ends
  // state
  int32_t *lay;
  double *phi;       // FP64 form: layer values
  float *phif;       // FP32 form: layer values (non-null selects the FP32 form; phi unused)
  __nv_bfloat16 *phih; // BF16 form: layer values (non-null selects the BF16 form; phi, phif unused)
  unsigned long long *nrecheck; // [2] rows redone in FP64: initial pass, tunnel passes
  unsigned long long *punc;     // [P] uncertified decisions of the initial pass (see Params::drift)
  int32_t *runc;                // [P] the same, this step (step records)
  double *pmass;     // [P][mslots][2] this step's sum over frontier rows of m_v (L base)_v, and of its
                     // terms' magnitudes, spread over mslots addresses per problem
  int32_t rpw;       // frontier rows per warp of the one-thread-per-row kernels (8, 16 or 32)
  int32_t mslots;    // a power of two: MASS_SLOTS for batches of few problems (their rows share a few
                     // addresses), 1 for many (rows spread over many problems already)
  double *pmres;     // [P] largest relative residual |sum| / magnitude over the steps so far
  int32_t *cover;
  int32_t *stamp;    // candidate dedup stamp (step id)
  int32_t *fmark;    // step at which the vertex was last in the frontier
  int32_t *uf;       // union-find parent for band CCL
  int32_t *multi;    // frontier row of a vertex holding several layers this step, else -1
  // the new state of this step's frontier rows, vertex-indexed, written by the update (one layer or
  // the base; unchanged rows keep their state): the band phases read it, the band count scatters it
  // into (lay, phi) -- unless a merge step scattered the rows first (CTL_APPLIED)
  int32_t *nlay;
  void *nph;         // stored value type of the form (double, float or bfloat16)
  // layers (global ids)
  int32_t *lstate, *lfwd, *lbirth, *ldeath, *lcnt;
  int32_t *lprob;
  // frontier lists (double buffered) and per-row outputs
  int32_t *front[2];
  int32_t *nfront;   // [2]
  int32_t *fseg[2];  // [V] per step parity: the frontier's vertices grouped by problem (problem p's
                     // pfront[p] vertices at fseg[voff[p]..]) for kernels that work per problem
  int32_t *onl;      // [Vcap] layers in the new row
  int32_t *olay;     // [Vcap * KMAX]
  double *ophi;      // [Vcap * KMAX]
  int32_t *coll;     // collision rows (frontier indices with >= 2 layers)
  int32_t *ncoll;
  // merge groups of the step
  int32_t *ngroups;
  int32_t *gprob, *gnew, *gnode, *gnmem, *gmem; // gmem [MAX_TRACES][MAX_GROUP]
  int32_t *ntrace;
  int32_t *tgroup, *tlayer;                     // per trace slot
  int32_t *tcount;                              // crossing edges found per trace
  int32_t *tlen;                                // ordered loop length per trace
  unsigned long long *tkey;                     // [MAX_TRACES][TRACE_CAP] sort keys (a<<32|b)
  int32_t *tslot;                               // [MAX_TRACES][TRACE_CAP] CSR slot of a->b
  int32_t *tsucc, *tpar, *trank, *tnext, *tord; // [MAX_TRACES][TRACE_CAP]
  unsigned long long *tbest;                    // per trace: packed best component
  // Reeb nodes (global pool): kind, step, problem ; position
  int32_t *nkind, *nstep, *nprob;
  double *npos;
  int32_t *nnodes;  // global node counter
  int32_t ncap;
  int32_t *nlocal;  // local node index within its problem
  // handles (global pool)
  int32_t *nhand;
  int32_t hcap;
  int32_t *hprob, *hstep, *hlayer, *hnode, *hoff, *hn, *hvoff, *hvn;
  double *hlen;
  int32_t *nhedge;  // edge pool counter
  int32_t ecap;
  int32_t *hedge;   // [ecap][2] global vertex ids
  double *hpts;     // [ecap][3]
  int32_t *hverts;  // [ecap]
  // records
  int32_t record;
  int32_t rcap;
  long long *rec;   // [P][rcap][5]
  unsigned long long *rhash; // [P]
  int32_t *rband;   // [P]
  // loop classification (Sec. 3.5): unit vertex normals [V][3], per-vertex sums of the lengths of
  // the edges to larger ids [V], mean edge length per problem [P], handle-loop length change [hcap]
  double *vn, *elen, *pmedge, *hdl;
  // error word
  int32_t *err;
  // device control block (see CTL_*), per-problem live layers and layers holding a band root
  int32_t *ctl;
  int32_t *nalive, *nbl;
};

// Control block: the step loops run on the device (a CUDA graph WHILE node around the step
// body), so the step counters live in device memory and every step kernel reads them.
enum Ctl : int {
  CTL_T = 0,          // current initial-pass step
  CTL_ACTIVE = 1,     // problems still running
  CTL_MERGE = 2,      // a collision row appeared this step
  CTL_SPLIT = 3,      // a band has != 1 components this step
  CTL_DONE_APPLY = 4, // last-block counters
  CTL_DONE_COUNT = 5,
  CTL_LIMIT = 6,      // hard step bound of the initial pass
  CTL_TAU = 7,        // current tunnel-pass step
  CTL_TACTIVE = 8,    // passes still running
  CTL_TLIMIT = 9,     // hard step bound of the tunnel passes
  CTL_NMERGE = 10,    // merge phases executed (launch accounting)
  CTL_NSPLIT = 11,    // split phases executed
  CTL_DONE_FRONT = 12, // last-block counter of the initial-pass frontier kernel
  CTL_DONE_TFRONT = 13, // last-block counter of the tunnel-pass frontier kernel
  CTL_MSKIP = 14,     // merge groups of this step already resolved by earlier rounds of the phase
  CTL_APPLIED = 15,   // 1: this step's rows were scattered into the state before the band phases (a
                      // merge step); 0: the band phases read the rows' new states from nlay / nph
  CTL_SIZE = 16
};

// Conditional handles of the step graph; `use` = 0 when the kernels run from a host loop.
struct Handles {
  cudaGraphConditionalHandle loop, merge, split;
  cudaGraphConditionalHandle mround; // rounds of the merge phase (more groups than trace slots)
  int32_t use;
};

// Programmatic dependent launch between consecutive step kernels of a graph: wait until the grids
// this one depends on have completed and their memory is visible (returns at once when the launch
// has no programmatic dependency), then let the next grid's blocks be scheduled -- they wait in
// their own pdl_enter, so the launch of the next kernel overlaps the tail of this one.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// True in exactly one thread of the grid: thread 0 of the last block to finish.  Every thread of
// every block must call it (after its share of the work).  The last block may read only data whose
// writers made it visible themselves (a __threadfence after the write, in the writing thread):
// the other threads skip the fence, which would hold every warp of every block until its stores
// have drained.
__device__ __forceinline__ bool last_block_done_fenced(int32_t *counter) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1) == (int32_t)gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    *counter = 0;
    return true;
  }
  return false;
}

// True in every thread of the last block of the grid to finish, for kernels whose writers fenced
// their own writes (see last_block_done_fenced).
__device__ __forceinline__ bool last_block_fenced(int32_t *counter) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1) == (int32_t)gridDim.x - 1;
    if (last) *counter = 0;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// ----------------------------------------------------------- FP64 arithmetic
// Explicit round-to-nearest operations: no contraction into FMA, each operation rounded on
// its own in the order written (the CPU oracle is compiled the same way).
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double dsqrt(double a) { return __dsqrt_rn(a); }

__device__ __forceinline__ bool frozen_state(int32_t st) { return st == L_DEAD || st == L_ENDED; }

// Exact tests on stored values x in [0, 1] (never NaN) done on the bit pattern: for
// non-negative doubles the order of the bits is the order of the values, and 1 - x > 0 holds
// exactly when x < 1.  (GB300 has few FP64 units; these keep decisions off them.)
__device__ __forceinline__ bool val_pos(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool val_lt1(double x) { return __double_as_longlong(x) < 0x3FF0000000000000LL; }
__device__ __forceinline__ bool val_band(double x) { return val_pos(x) && val_lt1(x); }
__device__ __forceinline__ bool val_pos(float x) { return __float_as_int(x) > 0; }
__device__ __forceinline__ bool val_lt1(float x) { return __float_as_int(x) < 0x3F800000; }
__device__ __forceinline__ bool val_band(float x) { return val_pos(x) && val_lt1(x); }
__device__ __forceinline__ bool val_pos(__nv_bfloat16 x) { return (int16_t)__bfloat16_as_ushort(x) > 0; }
__device__ __forceinline__ bool val_lt1(__nv_bfloat16 x) { return (int16_t)__bfloat16_as_ushort(x) < 0x3F80; }
__device__ __forceinline__ bool val_band(__nv_bfloat16 x) { return val_pos(x) && val_lt1(x); }
// exact widening of a stored value
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return (double)x; }
__device__ __forceinline__ double to_f64(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

// ------------------------------------------------------------ row loops
// Grid-stride loops over the n rows of a frontier list that spread warps over the whole grid:
// loop warp w runs as warp w / gridDim.x of block w % gridDim.x, so a frontier of a few
// thousand rows occupies every SM instead of filling the first blocks (and so a few SMs)
// while the rest idle.  Lanes of a warp take consecutive rows (FOR_ROWS: 32 rows per warp, one
// lane each; FOR_ROWS_G: 32 / GL rows per warp, a group of GL lanes each that share the row's
// neighbours).  The loop bounds are uniform per warp; the body runs once per row, `continue`
// moves on to the next row.
constexpr int GL = 8; // lanes per row of the neighbour-parallel kernels (mesh degrees are 3..10)
#define VLS_WARP_LOOP(w, rows_per_warp, n)                                                          \
  for (int32_t w = (int32_t)(blockIdx.x + gridDim.x * (threadIdx.x >> 5)); w * (rows_per_warp) < (n); \
       w += (int32_t)(gridDim.x * (blockDim.x >> 5)))
#define FOR_ROWS(i, n) FOR_ROWS_R(i, n, 32)
// R rows per warp (R = 8, 16 or 32): lanes R..31 take no row
#define FOR_ROWS_R(i, n, R)                                                                         \
  VLS_WARP_LOOP(vls_w_, (R), n)                                                                     \
  for (int32_t i = vls_w_ * (R) + (int32_t)(threadIdx.x & 31);                                      \
       (int32_t)(threadIdx.x & 31) < (R) && i < (n); i = INT32_MAX)
#define FOR_ROWS_G(i, n)                                                                            \
  VLS_WARP_LOOP(vls_w_, 32 / GL, n)                                                                 \
  for (int32_t i = vls_w_ * (32 / GL) + (int32_t)((threadIdx.x & 31) / GL); i < (n); i = INT32_MAX)
// lane within the row's group, and the warp mask of the group
__device__ __forceinline__ int32_t group_lane() { return (int32_t)(threadIdx.x & (GL - 1)); }
__device__ __forceinline__ unsigned group_mask() { return ((1u << GL) - 1u) << (threadIdx.x & (32 - GL)); }

// ------------------------------------------------------------ stored values
// The layer value of a vertex is stored as double (FP64 form), float (FP32 form, d.phif
// non-null) or bfloat16 (BF16 form, d.phih non-null).  Readers that only test a value use the
// bit tests above on the stored type.
__device__ __forceinline__ double ph_ld(const Dev &d, int32_t v) {
  return d.phih ? to_f64(d.phih[v]) : d.phif ? (double)d.phif[v] : d.phi[v];
}
__device__ __forceinline__ bool ph_lt1(const Dev &d, int32_t v) {
  return d.phih ? val_lt1(d.phih[v]) : d.phif ? val_lt1(d.phif[v]) : val_lt1(d.phi[v]);
}
__device__ __forceinline__ bool ph_band(const Dev &d, int32_t v) {
  return d.phih ? val_band(d.phih[v]) : d.phif ? val_band(d.phif[v]) : val_band(d.phi[v]);
}
template <class TV> __device__ __forceinline__ const TV *ph_arr(const Dev &d);
template <> __device__ __forceinline__ const double *ph_arr<double>(const Dev &d) { return d.phi; }
template <> __device__ __forceinline__ const float *ph_arr<float>(const Dev &d) { return d.phif; }
template <> __device__ __forceinline__ const __nv_bfloat16 *ph_arr<__nv_bfloat16>(const Dev &d) { return d.phih; }

// FP32 storage of an FP64 value without moving it across any threshold that later steps test
// on stored values: 0 < x, x < 1 and x >= theta keep their truth value (x in [0, 1]).  Only
// one ulp separates a rounded value from x, so one step towards x's side suffices.
__device__ __forceinline__ float f32_keep_side(double x, double theta) {
  float f = __double2float_rn(x);
  const double fd = (double)f;
  int32_t bits = __float_as_int(f);
  if (x > 0.0 && !(fd > 0.0)) bits = 1;                   // smallest positive float
  else if (x < 1.0 && !(fd < 1.0)) bits = 0x3F7FFFFF;     // largest float below 1
  else if (x < theta && fd >= theta) bits -= 1;
  else if (x >= theta && fd < theta) bits += 1;
  return __int_as_float(bits);
}
// The same for bfloat16 storage (8 significant bits): the nearest bfloat16, then one step
// back towards x's side of 0, 1 or theta if the rounding crossed it.
__device__ __forceinline__ __nv_bfloat16 bf16_keep_side(double x, double theta) {
  const __nv_bfloat16 h = __double2bfloat16(x);
  const double hd = to_f64(h);
  uint16_t bits = __bfloat16_as_ushort(h);
  if (x > 0.0 && !(hd > 0.0)) bits = 1;                   // smallest positive bfloat16
  else if (x < 1.0 && !(hd < 1.0)) bits = 0x3F7F;         // largest bfloat16 below 1
  else if (x < theta && hd >= theta) bits -= 1;
  else if (x >= theta && hd < theta) bits += 1;
  return __ushort_as_bfloat16(bits);
}
// Rounding of an FP64 value to the stored type keeping its side of every threshold (the FP64
// form stores it as is).
template <class TV> __device__ __forceinline__ double round_keep(double x, double theta);
template <> __device__ __forceinline__ double round_keep<double>(double x, double) { return x; }
template <> __device__ __forceinline__ double round_keep<float>(double x, double theta) {
  return (double)f32_keep_side(x, theta);
}
template <> __device__ __forceinline__ double round_keep<__nv_bfloat16>(double x, double theta) {
  return to_f64(bf16_keep_side(x, theta));
}
// a value of a row output (exactly representable in the stored type) into the state
__device__ __forceinline__ void ph_st(const Dev &d, int32_t v, double x) {
  if (d.phih) d.phih[v] = __double2bfloat16(x);
  else if (d.phif) d.phif[v] = (float)x;
  else d.phi[v] = x;
}
// a row's new state (one layer l or the base, value exactly representable in the stored type)
__device__ __forceinline__ void row_new(const Dev &d, int32_t v, int32_t l, double x) {
  d.nlay[v] = l;
  if (d.phih) static_cast<__nv_bfloat16 *>(d.nph)[v] = __double2bfloat16(x);
  else if (d.phif) static_cast<float *>(d.nph)[v] = (float)x;
  else static_cast<double *>(d.nph)[v] = x;
}
__device__ __forceinline__ bool nph_band(const Dev &d, int32_t v) {
  return d.phih ? val_band(static_cast<const __nv_bfloat16 *>(d.nph)[v])
         : d.phif ? val_band(static_cast<const float *>(d.nph)[v])
                  : val_band(static_cast<const double *>(d.nph)[v]);
}
// the row's new state into (lay, phi)
__device__ __forceinline__ void row_scatter(const Dev &d, int32_t v) {
  d.lay[v] = d.nlay[v];
  if (d.phih) d.phih[v] = static_cast<const __nv_bfloat16 *>(d.nph)[v];
  else if (d.phif) d.phif[v] = static_cast<const float *>(d.nph)[v];
  else d.phi[v] = static_cast<const double *>(d.nph)[v];
}
// any FP64 value into the state (FP32 / BF16 forms: rounded keeping its side of every threshold)
__device__ __forceinline__ void ph_st_round(const Dev &d, const Params &P, int32_t v, double x) {
  if (d.phih) d.phih[v] = bf16_keep_side(x, P.theta);
  else if (d.phif) d.phif[v] = f32_keep_side(x, P.theta);
  else d.phi[v] = x;
}

// One explicit Euler step of Eq. (2) at one vertex (base present; nl non-base layers in
// ascending id order with own values x[] and Laplacians lap[]; base value xb, Laplacian
// lapb).  Only pairs (layer, base) have mu_ij, e_ij != 0 (Sec. 2); e is antisymmetric so the
// rates sum to zero; n = nl + 1 phases meet at the vertex.  Then clamp to [0,1], snap at
// eps0 / 1 - eps0 and divide by the column sum (Sec. 2, normalisation).  Returns false if
// the column sum vanished (values left unchanged).  unc (FP32 / BF16 forms): set when a decision of
// the step -- a clamped value against eps0 or 1 - eps0, a new value against theta -- lies within
// P.drift of its threshold, closer than the low-precision trajectory can be trusted to be.
__device__ __forceinline__ bool vertex_update(const Params &P, int nl, const double *x, const double *lap,
                                              double xb, double lapb, double *out, bool *unc = nullptr) {
  const double mun = P.mun[nl + 1]; // = mu / n, rounded once on the host (same IEEE quotient)
  double y[KMAX];
  double sr = 0.0;
#pragma unroll
  for (int i = 0; i < KMAX; ++i) {
    if (i < nl) {
      double t1 = dmul(P.w, dsub(x[i], xb));
      double t2 = dmul(P.ah, dsub(lap[i], lapb));
      double t3 = dmul(P.e, dsqrt(dmul(x[i], xb)));
      double r = dmul(mun, dadd(dadd(t1, t2), t3));
      sr = dadd(sr, r);
      y[i] = dadd(x[i], dmul(P.dt, r));
    }
  }
  double yb = dadd(xb, dmul(P.dt, -sr));
#pragma unroll
  for (int i = 0; i <= KMAX; ++i) {
    if (i <= nl) {
      double v = (i < nl) ? y[i] : yb;
      if (v < 0.0) v = 0.0;
      if (v > 1.0) v = 1.0;
      if (unc) *unc |= fabs(v - P.eps0) < P.drift || fabs(v - P.one_m_eps) < P.drift;
      if (v < P.eps0) v = 0.0;
      if (v > P.one_m_eps) v = 1.0;
      if (i < nl) y[i] = v;
      else yb = v;
    }
  }
  double S = yb;
#pragma unroll
  for (int i = 0; i < KMAX; ++i)
    if (i < nl) S = dadd(S, y[i]);
  if (S == 0.0) return false;
#pragma unroll
  for (int i = 0; i < KMAX; ++i)
    if (i < nl) {
      out[i] = ddiv(y[i], S);
      if (unc) *unc |= fabs(out[i] - P.theta) < P.drift;
    }
  return true;
}

// FP32 form of vertex_update for one layer and the base (n = 2), the common case.  Returns
// false when any decision of the step lies within the recheck margin: a clamped value near
// eps0 or 1 - eps0 (snap), a new value near theta (isoline, arrival), or a vanishing column
// sum; the caller then redoes the row in FP64.  unc: as in vertex_update, tested here only when the
// drift bound exceeds the margin (the BF16 form; otherwise a row near a threshold is redone anyway).
__device__ __forceinline__ bool vertex_update_f32(const Params &P, float x, float lap, float xb, float lapb,
                                                  float &out, bool &unc) {
  const float t1 = P.f_w * (x - xb);
  const float t2 = P.f_ah * (lap - lapb);
  const float t3 = P.f_e * sqrtf(x * xb);
  const float r = P.f_mun[2] * (t1 + t2 + t3);
  float y = x + P.f_dt * r;
  float yb = xb - P.f_dt * r;
  y = fminf(fmaxf(y, 0.f), 1.f);
  yb = fminf(fmaxf(yb, 0.f), 1.f);
  const float m = P.f_margin, dr = P.f_drift;
  bool near = fabsf(y - P.f_eps0) < m || fabsf(y - P.f_one_m_eps) < m || fabsf(yb - P.f_eps0) < m ||
              fabsf(yb - P.f_one_m_eps) < m;
  const bool wide = dr > m;
  unc = wide && (fabsf(y - P.f_eps0) < dr || fabsf(y - P.f_one_m_eps) < dr || fabsf(yb - P.f_eps0) < dr ||
                 fabsf(yb - P.f_one_m_eps) < dr);
  if (y < P.f_eps0) y = 0.f;
  if (y > P.f_one_m_eps) y = 1.f;
  if (yb < P.f_eps0) yb = 0.f;
  if (yb > P.f_one_m_eps) yb = 1.f;
  const float S = y + yb;
  if (S == 0.f) return false;
  out = y / S;
  near |= fabsf(out - P.f_theta) < m;
  unc |= wide && fabsf(out - P.f_theta) < dr;
  return !near;
}

// Count the lanes with `flag` into cnt[key] with one atomic per key present in the warp.  Every
// lane of the warp calls (key of a lane without flag: anything).
__device__ __forceinline__ void count_keyed(unsigned long long *cnt, int32_t key, bool flag) {
  const unsigned fl = __ballot_sync(0xffffffffu, flag);
  if (!fl) return;
  const unsigned peers = __match_any_sync(0xffffffffu, flag ? key : -1) & fl;
  if (flag && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cnt[key], (unsigned long long)__popc(peers));
}
__device__ __forceinline__ void count_keyed(int32_t *cnt, int32_t key, bool flag) {
  const unsigned fl = __ballot_sync(0xffffffffu, flag);
  if (!fl) return;
  const unsigned peers = __match_any_sync(0xffffffffu, flag ? key : -1) & fl;
  if (flag && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cnt[key], (int32_t)__popc(peers));
}

// ------------------------------------------------------------ union-find
// Lock-free union by index: the larger root is hooked under the smaller, so a component's
// root is its smallest member (the canonical label).
__device__ __forceinline__ int32_t uf_find(int32_t *par, int32_t x) {
  int32_t p = par[x];
  while (p != x) {
    int32_t gp = par[p];
    if (gp != p) par[x] = gp; // path halving (benign race: only shortens paths)
    x = p;
    p = par[x];
  }
  return x;
}
// Returns true when this call linked two components (each link joins two distinct trees: links
// only point from a larger root to a smaller id).
__device__ __forceinline__ bool uf_unite(int32_t *par, int32_t a, int32_t b) {
  int32_t ra = uf_find(par, a), rb = uf_find(par, b);
  while (ra != rb) {
    if (ra > rb) { int32_t t = ra; ra = rb; rb = t; }
    int32_t old = atomicCAS(&par[rb], rb, ra);
    if (old == rb) return true;
    rb = uf_find(par, old);
    ra = uf_find(par, ra);
  }
  return false;
}

// Append to a list shared by the whole grid with one atomic per warp (the lanes that reach this
// call together), and bump a per-key counter with one atomic per key present in the warp.
// Returns this lane's slot; *key_slot (if given) receives the lane's position among its key's
// entries.  Must be called only by lanes that append.
__device__ __forceinline__ int32_t warp_append(int32_t *counter, int32_t *key_counts, int32_t key,
                                               int32_t *key_slot = nullptr) {
  namespace cg = cooperative_groups;
  cg::coalesced_group g = cg::coalesced_threads();
  int32_t base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(counter, (int32_t)g.size());
  base = g.shfl(base, 0) + (int32_t)g.thread_rank();
  cg::coalesced_group kg = cg::labeled_partition(g, key);
  int32_t kb = 0;
  if (kg.thread_rank() == 0) kb = atomicAdd(&key_counts[key], (int32_t)kg.size());
  if (key_slot) *key_slot = kg.shfl(kb, 0) + (int32_t)kg.thread_rank();
  return base;
}

// Mass-check sums of a warp's rows, keyed by problem (initial pass) or pass (tunnel passes):
// FP64 atomics on `slots` addresses per key (a power of two), since a frontier list interleaves
// keys and same-address atomics serialise.  A warp with few keys sums each key's rows first: one
// pair of atomics per key per warp.  key < 0: the lane holds no row.  Every lane of the warp calls.
__device__ __forceinline__ void mass_sums(double *acc, int32_t slots, int32_t key, int32_t lane, double2 m) {
  const int32_t slot = (int32_t)((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) & (slots - 1));
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  unsigned leaders = __ballot_sync(0xffffffffu, lane == __ffs(peers) - 1);
  if (__popc(leaders) <= 4) {
    while (leaders) {
      const int32_t k = __shfl_sync(0xffffffffu, key, __ffs(leaders) - 1);
      leaders &= leaders - 1;
      double sx = key == k ? m.x : 0.0, sy = key == k ? m.y : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, off);
        sy += __shfl_xor_sync(0xffffffffu, sy, off);
      }
      if (lane == 0 && k >= 0 && sy != 0.0) {
        atomicAdd(&acc[((int64_t)k * slots + slot) * 2], sx);
        atomicAdd(&acc[((int64_t)k * slots + slot) * 2 + 1], sy);
      }
    }
  } else if (m.y != 0.0) {
    const int32_t ls = (slot + lane) & (slots - 1);
    atomicAdd(&acc[((int64_t)key * slots + ls) * 2], m.x);
    atomicAdd(&acc[((int64_t)key * slots + ls) * 2 + 1], m.y);
  }
}
// The relative residual |sum| / magnitude of one key's sums (0 when nothing was summed); clears them.
__device__ __forceinline__ double mass_fold(double *acc, int32_t slots, int32_t key) {
  double2 *pm = reinterpret_cast<double2 *>(acc) + (int64_t)key * slots;
  double sm = 0.0, mag = 0.0;
  for (int k = 0; k < slots; ++k) {
    const double2 a = __ldcg(pm + k);
    sm += a.x;
    mag += a.y;
    pm[k] = make_double2(0.0, 0.0);
  }
  return mag > 0.0 ? fabs(sm) / mag : 0.0;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// problem of a global vertex (voff ascending, P small): binary search
__device__ __forceinline__ int32_t prob_of_vertex(const int32_t *voff, int32_t P, int32_t v) {
  int32_t lo = 0, hi = P - 1;
  while (lo < hi) {
    int32_t m = (lo + hi + 1) >> 1;
    if (voff[m] <= v) lo = m;
    else hi = m - 1;
  }
  return lo;
}

// slot of half-edge u->w in the CSR (binary search over the sorted row), -1 if absent
__device__ __forceinline__ int32_t slot_of(const int32_t *rp, const int32_t *col, int32_t u, int32_t w) {
  int32_t lo = rp[u], hi = rp[u + 1] - 1;
  while (lo <= hi) {
    int32_t m = (lo + hi) >> 1;
    int32_t c = col[m];
    if (c == w) return m;
    if (c < w) lo = m + 1;
    else hi = m - 1;
  }
  return -1;
}

__device__ __forceinline__ void set_err(int32_t *err, int32_t code) { atomicCAS(err, 0, code); }

// Checked builds (-DVLS_CHECKED): every guarded index is range-checked; the first violation
// records (site, index) in err[2], err[3] and the access is skipped.  Unchecked builds
// compile the guard to `true`.
#ifdef VLS_CHECKED
__device__ __forceinline__ bool vchk(int32_t *err, long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  if (atomicCAS(err + 2, 0, site) == 0) err[3] = (int32_t)i;
  return false;
}
#define VCHK(err, i, n, site) ::vls::vchk((err), (long long)(i), (long long)(n), (site))
#else
#define VCHK(err, i, n, site) true
#endif

// ------------------------------------------------------------------ host side
struct Batch; // defined in api.cu

cudaError_t launch_operator(Batch &b, int32_t *status);
}  // namespace vls
