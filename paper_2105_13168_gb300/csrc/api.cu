// api.cu -- host engine and C ABI (include/vls.h).
//
// One call = one batch: the host lays the batch out in a grow-only device arena owned by
// the context, copies (or, for device meshes, moves on the device) the inputs into the union
// graph, and drives the phases on the context's stream: operator build (a0), initial pass
// (steps of kernels, the host polls a device "still running" counter every sync_interval
// steps), tunnel passes, result download.  Nothing on the path runs on the host except
// launch bookkeeping and the final repacking of downloaded results.
#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "vls_batch.cuh"

using namespace vls;

namespace {

struct ProbResult {
  int32_t status = 0, genus = 0, steps = 0, tunnel_steps = 0;
  int64_t nv = 0;
  vls_stats stats{};
  std::vector<int32_t> nodes;  // [n][2]
  std::vector<double> npos;    // [n][3]
  std::vector<int32_t> layers; // [L][3]
  struct Handle {
    std::vector<int32_t> edges, verts;
    std::vector<double> pts;
    int32_t info[3];
    double len;
  };
  std::vector<Handle> handles;
  struct Tunnel {
    int32_t info[3];
    std::vector<int32_t> verts;
    int32_t sst = -1;          // PL streamline (Sec. 3.2): status, -1 not traced
    std::vector<double> spts;  // [n][3] closed polyline
    double slen = 0.0;
  };
  std::vector<Tunnel> tunnels;
  std::vector<Tunnel> refined;             // refined handle loops (Sec. 3.3), one per handle
  std::vector<std::array<double, 3>> dlen; // offset length change: handle, tunnel, refined (Sec. 3.5)
  std::vector<int32_t> lay, cover;
  std::vector<double> phi;
  std::vector<int64_t> rec;
};

}  // namespace

struct vls_result {
  std::vector<ProbResult> p;
  std::vector<int64_t> klaunch;
  std::vector<double> kms;
};

// Pinned host memory for the set-up tables and small outputs of the pass chunks in flight: grow-only
// blocks owned by the context, handed out afresh by every call.
struct PinnedPool {
  std::vector<std::pair<char *, size_t>> blocks;
  size_t bi = 0, used = 0;
  void reset() { bi = 0; used = 0; }
  void *take(size_t n) {
    n = (n + 63) & ~size_t(63);
    while (bi < blocks.size() && used + n > blocks[bi].second) { ++bi; used = 0; }
    if (bi == blocks.size()) {
      const size_t sz = std::max(n, size_t(4) << 20);
      char *p = nullptr;
      if (cudaMallocHost(reinterpret_cast<void **>(&p), sz) != cudaSuccess) return nullptr;
      blocks.push_back({p, sz});
      used = 0;
    }
    void *r = blocks[bi].first + used;
    used += n;
    return r;
  }
  void release() {
    for (auto &b : blocks) cudaFreeHost(b.first);
    blocks.clear();
    reset();
  }
};

constexpr int PASS_STREAMS = 8; // pass chunks in flight at once, each on its own stream

struct vls_ctx {
  vls_options opt;
  cudaStream_t st = nullptr;
  cudaStream_t sp[PASS_STREAMS] = {}; // pass chunks, concurrent with the initial pass and each other
  cudaStream_t st3 = nullptr;         // downloads of finished chunks
  cudaMemPool_t pool = nullptr;       // device blocks of the pass chunks (stream-ordered)
  PinnedPool pinned;
  Arena arena;
  int sm = 148;
  std::vector<cudaEvent_t> evpool; // profiling events, reused across calls
};

cudaError_t Arena::reserve(size_t bytes) {
  if (bytes <= cap) return cudaSuccess;
  if (base) cudaFree(base);
  base = nullptr;
  cap = 0;
  size_t want = bytes + bytes / 8;
  cudaError_t e = cudaMalloc(&base, want);
  if (e != cudaSuccess) { base = nullptr; return e; }
  cap = want;
  return cudaSuccess;
}

extern "C" void vls_default_options(vls_options *o) {
  std::memset(o, 0, sizeof(*o));
  o->mu = 0.25;
  o->e = 1.0 / 30.0;
  o->a = 1.0 / 25.0;
  o->w = o->a / 5.0;
  o->dt_factor = 0.5;
  o->eps0 = 1e-3;
  o->theta_iso = 0.5;
  o->lbar = 0.0;
  o->recheck_margin = 1e-5;
  o->max_steps = 200000;
  o->max_pass_steps = 200000;
  o->tunnels = 1;
  o->keep_state = 0;
  o->record_steps = 0;
  o->sync_interval = 16;
  o->threads = 0;
  o->blocks_per_sm = 0;
  o->precision = VLS_FP64;
  o->profile = 0;
  o->host_loop = 0;
  o->hook_variant = 0;
  o->rows_per_warp = 0;
  o->refine = 1;
  o->offset = 0.5;
  o->K = 4;
  o->laplacian = 0;
  o->max_passes = 0;
  o->autotune = 1;
  o->drift_bound = 0.0;
  o->streamlines = 1;
}

extern "C" void vls_constants(const vls_options *o, double out[4]) {
  const double pi = 3.14159265358979323846;
  double eta = pi * o->a / std::sqrt(2.0 * o->w);
  double lbar = o->lbar > 0 ? o->lbar : eta / 4.0;
  double D = o->mu * o->a * o->a / 2.0;
  double dt = o->dt_factor * lbar * lbar / (4.0 * D);
  out[0] = eta;
  out[1] = lbar;
  out[2] = dt;
  out[3] = 4.0 / (lbar * lbar);
}

extern "C" const char *vls_status_string(vls_status s) {
  switch (s) {
  case VLS_OK: return "ok";
  case VLS_EINVAL: return "invalid argument or mesh index";
  case VLS_ENOTMANIFOLD: return "mesh is open or not manifold";
  case VLS_ENONORIENTABLE: return "mesh faces are not consistently oriented";
  case VLS_EDISCONNECTED: return "mesh is disconnected or has unused vertices";
  case VLS_EMAXSTEPS: return "step limit reached";
  case VLS_ESLOTS: return "too many layers met at one vertex";
  case VLS_ELAYERS: return "layer, event or loop capacity exceeded";
  case VLS_ELOOPFAIL: return "tunnel pass failed to reach the far side";
  case VLS_ETIMEOUT: return "device wait timed out";
  case VLS_ENOMEM: return "out of memory";
  case VLS_ECUDA: return "CUDA error";
  case VLS_ESTALL: return "front stopped before covering the surface";
  case VLS_ETOOLARGE: return "input above the fixed limits of the no-allocation entry point";
  }
  return "unknown status";
}

extern "C" vls_status vls_create(vls_ctx **ctx, const vls_options *o, void *stream) {
  if (!ctx) return VLS_EINVAL;
  vls_ctx *c = new (std::nothrow) vls_ctx();
  if (!c) return VLS_ENOMEM;
  if (o) c->opt = *o;
  else vls_default_options(&c->opt);
  if ((c->opt.precision != VLS_FP64 && c->opt.precision != VLS_FP32_RECHECK && c->opt.precision != VLS_BF16_RECHECK) ||
      (c->opt.precision != VLS_FP64 && !(c->opt.recheck_margin > 0.0 && c->opt.recheck_margin < 0.25)) ||
      (c->opt.rows_per_warp != 0 && c->opt.rows_per_warp != 8 && c->opt.rows_per_warp != 16 &&
       c->opt.rows_per_warp != 32) ||
      (c->opt.K != 0 && c->opt.K != KMAX) || c->opt.laplacian != 0 || !(c->opt.offset > 0.0) ||
      c->opt.max_passes < 0 || (c->opt.autotune != 0 && c->opt.autotune != 1) || c->opt.drift_bound < 0.0 ||
      (c->opt.streamlines != 0 && c->opt.streamlines != 1)) {
    delete c;
    return VLS_EINVAL;
  }
  c->st = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete c;
    return VLS_ECUDA;
  }
  bool ok = true;
  for (int i = 0; i < PASS_STREAMS; ++i) ok &= cudaStreamCreateWithFlags(&c->sp[i], cudaStreamNonBlocking) == cudaSuccess;
  ok &= cudaStreamCreateWithFlags(&c->st3, cudaStreamNonBlocking) == cudaSuccess;
  {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    ok &= cudaMemPoolCreate(&c->pool, &props) == cudaSuccess;
    if (ok) {
      // keep up to 4 GiB of freed blocks for the next chunks and calls (larger chunks are returned at
      // the next synchronisation, so that chunks of other sizes never pile up)
      uint64_t keep = uint64_t(4) << 30;
      ok &= cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess;
    }
  }
  if (!ok) {
    vls_destroy(c);
    return VLS_ECUDA;
  }
  *ctx = c;
  return VLS_OK;
}

extern "C" void vls_destroy(vls_ctx *ctx) {
  if (!ctx) return;
  for (int i = 0; i < PASS_STREAMS; ++i)
    if (ctx->sp[i]) {
      cudaStreamSynchronize(ctx->sp[i]);
      cudaStreamDestroy(ctx->sp[i]);
    }
  if (ctx->st3) {
    cudaStreamSynchronize(ctx->st3);
    cudaStreamDestroy(ctx->st3);
  }
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  ctx->pinned.release();
  if (ctx->arena.base) cudaFree(ctx->arena.base);
  for (cudaEvent_t e : ctx->evpool) cudaEventDestroy(e);
  delete ctx;
}

namespace {

// two-pass layout: first pass counts bytes, second hands out pointers
struct Layout {
  Arena *a;
  bool sizing;
  size_t bytes = 0;
  template <class T> T *take(size_t n) {
    if (sizing) {
      bytes = ((bytes + 255) & ~size_t(255)) + n * sizeof(T);
      return nullptr;
    }
    return a->take<T>(n);
  }
};

void layout_batch(Layout &L, Batch &b) {
  Dev &d = b.d;
  const size_t P = b.P, V = b.V, NF = b.NF, nnz = b.nnz, Lc = b.Lcap;
  d.X = L.take<double>(3 * V);
  d.F = L.take<int32_t>(3 * NF);
  d.rp = L.take<int32_t>(V + 1);
  d.col = L.take<int32_t>(nnz);
  d.hface = L.take<int32_t>(nnz);
  d.voff = L.take<int32_t>(P + 1);
  d.foff = L.take<int32_t>(P + 1);
  d.lbase = L.take<int32_t>(P);
  d.lcap = L.take<int32_t>(P);
  d.seed = L.take<int32_t>(P);
  d.lcount = L.take<int32_t>(P);
  d.pstatus = L.take<int32_t>(P);
  d.pdone = L.take<int32_t>(P);
  d.psteps = L.take<int32_t>(P);
  d.pnodes = L.take<int32_t>(P);
  d.pfront = L.take<int32_t>(2 * P);
  d.pmerge = L.take<int32_t>(P);
  d.pupd = L.take<int64_t>(P);
  d.pev = L.take<int32_t>(4 * P);
  d.lay = L.take<int32_t>(V);
  const vls_precision pr = b.opt.precision;
  d.phi = pr == VLS_FP64 ? L.take<double>(V) : nullptr;
  d.phif = pr == VLS_FP32_RECHECK ? L.take<float>(V) : nullptr;
  d.phih = pr == VLS_BF16_RECHECK ? L.take<__nv_bfloat16>(V) : nullptr;
  d.nrecheck = L.take<unsigned long long>(2);
  d.punc = L.take<unsigned long long>(P);
  d.runc = L.take<int32_t>(P);
  d.mslots = P <= (size_t)MASS_SPREAD_MAXP ? MASS_SLOTS : 1;
  d.pmass = L.take<double>(2 * (size_t)d.mslots * P);
  d.pmres = L.take<double>(P);
  d.cover = L.take<int32_t>(V);
  d.stamp = L.take<int32_t>(V);
  d.fmark = L.take<int32_t>(V);
  d.uf = L.take<int32_t>(V);
  d.multi = L.take<int32_t>(V);
  d.lstate = L.take<int32_t>(Lc);
  d.lfwd = L.take<int32_t>(Lc);
  d.lbirth = L.take<int32_t>(Lc);
  d.ldeath = L.take<int32_t>(Lc);
  d.lcnt = L.take<int32_t>(3 * Lc);
  d.lprob = L.take<int32_t>(Lc);
  d.front[0] = L.take<int32_t>(2 * V);
  d.front[1] = L.take<int32_t>(2 * V);
  d.fseg[0] = L.take<int32_t>(V);
  d.fseg[1] = L.take<int32_t>(V);
  d.nfront = L.take<int32_t>(2);
  d.onl = L.take<int32_t>(V);
  d.olay = L.take<int32_t>(KMAX * V);
  d.ophi = L.take<double>(KMAX * V);
  d.coll = L.take<int32_t>(V);
  d.ncoll = L.take<int32_t>(1);
  d.ngroups = L.take<int32_t>(1);
  d.gprob = L.take<int32_t>(MAX_TRACES);
  d.gnew = L.take<int32_t>(MAX_TRACES);
  d.gnode = L.take<int32_t>(MAX_TRACES);
  d.gnmem = L.take<int32_t>(MAX_TRACES);
  d.gmem = L.take<int32_t>(MAX_TRACES * MAX_GROUP);
  d.ntrace = L.take<int32_t>(1);
  d.tgroup = L.take<int32_t>(MAX_TRACES);
  d.tlayer = L.take<int32_t>(MAX_TRACES);
  d.tcount = L.take<int32_t>(MAX_TRACES);
  d.tlen = L.take<int32_t>(MAX_TRACES);
  d.tkey = L.take<unsigned long long>((size_t)MAX_TRACES * TRACE_CAP);
  d.tslot = L.take<int32_t>((size_t)MAX_TRACES * TRACE_CAP);
  d.tsucc = L.take<int32_t>((size_t)MAX_TRACES * TRACE_CAP);
  d.tpar = L.take<int32_t>((size_t)MAX_TRACES * TRACE_CAP);
  d.trank = L.take<int32_t>((size_t)MAX_TRACES * TRACE_CAP * 2);
  d.tnext = L.take<int32_t>((size_t)MAX_TRACES * TRACE_CAP * 2);
  d.tord = L.take<int32_t>((size_t)MAX_TRACES * TRACE_CAP);
  d.tbest = L.take<unsigned long long>(MAX_TRACES);
  d.ncap = (int32_t)(Lc + P);
  d.nkind = L.take<int32_t>(d.ncap);
  d.nstep = L.take<int32_t>(d.ncap);
  d.nprob = L.take<int32_t>(d.ncap);
  d.nlocal = L.take<int32_t>(d.ncap);
  d.npos = L.take<double>(3 * (size_t)d.ncap);
  d.nnodes = L.take<int32_t>(1);
  d.hcap = (int32_t)Lc;
  d.nhand = L.take<int32_t>(1);
  d.hprob = L.take<int32_t>(d.hcap);
  d.hstep = L.take<int32_t>(d.hcap);
  d.hlayer = L.take<int32_t>(d.hcap);
  d.hnode = L.take<int32_t>(d.hcap);
  d.hoff = L.take<int32_t>(d.hcap);
  d.hn = L.take<int32_t>(d.hcap);
  d.hvoff = L.take<int32_t>(d.hcap);
  d.hvn = L.take<int32_t>(d.hcap);
  d.hlen = L.take<double>(d.hcap);
  // handle-loop crossing edges of the whole batch: every handle loop of a high-genus problem
  // together (thousands of loops of ~1k edges on a 20M-face mesh)
  d.ecap = (int32_t)std::max<size_t>(1u << 20, V);
  d.nhedge = L.take<int32_t>(1);
  d.hedge = L.take<int32_t>(2 * (size_t)d.ecap);
  d.hpts = L.take<double>(3 * (size_t)d.ecap);
  d.hverts = L.take<int32_t>(d.ecap);
  d.rec = L.take<long long>(d.record ? (size_t)P * d.rcap * 5 : 1);
  d.rhash = L.take<unsigned long long>(P);
  d.rband = L.take<int32_t>(P);
  d.vn = L.take<double>(3 * V);
  d.elen = L.take<double>(V);
  d.pmedge = L.take<double>(P);
  d.hdl = L.take<double>(d.hcap);
  d.err = L.take<int32_t>(4);
  d.ctl = L.take<int32_t>(CTL_SIZE);
  d.nalive = L.take<int32_t>(P);
  d.nbl = L.take<int32_t>(P);
  d.nlay = L.take<int32_t>(V);
  d.nph = pr == VLS_FP64 ? static_cast<void *>(L.take<double>(V))
          : pr == VLS_FP32_RECHECK ? static_cast<void *>(L.take<float>(V))
                                   : static_cast<void *>(L.take<__nv_bfloat16>(V));
}

// nx > 0: a refinement chunk -- its own border-edge pool (nx edges) and the tunnel cycles it starts
// from (ncyc vertex ids)
void layout_tunnels(Layout &L, Batch &b, int32_t NP, int64_t PV, int64_t ncut, int64_t nx, int64_t ncyc, int64_t scap) {
  TDev &T = b.td;
  T.NP = NP;
  T.PV = (int32_t)PV;
  T.pbase = L.take<int32_t>(NP + 1);
  T.pprob = L.take<int32_t>(NP);
  T.pstep = L.take<int32_t>(NP);
  T.pcoff = L.take<int32_t>(NP);
  T.pcn = L.take<int32_t>(NP);
  T.cut = L.take<int32_t>(ncut);
  T.heoff = L.take<int32_t>(NP);
  T.hen = L.take<int32_t>(NP);
  T.flag = L.take<int8_t>(PV);
  const vls_precision pr = b.opt.precision;
  T.phi = pr == VLS_FP64 ? L.take<double>(PV) : nullptr;
  T.phif = pr == VLS_FP32_RECHECK ? L.take<float>(PV) : nullptr;
  T.phih = pr == VLS_BF16_RECHECK ? L.take<__nv_bfloat16>(PV) : nullptr;
  T.T = L.take<int32_t>(PV);
  T.stamp = L.take<int32_t>(PV);
  T.fv[0] = L.take<int32_t>(PV);
  T.fq[0] = L.take<int32_t>(PV);
  T.fv[1] = L.take<int32_t>(PV);
  T.fq[1] = L.take<int32_t>(PV);
  T.nf = L.take<int32_t>(2);
  T.onew = L.take<double>(PV);
  T.qdone = L.take<int32_t>(NP);
  T.qsteps = L.take<int32_t>(NP);
  T.qstatus = L.take<int32_t>(NP);
  T.qbstar = L.take<int32_t>(NP);
  T.qcnt = L.take<int32_t>(2 * NP);
  T.qslots = NP <= MASS_SPREAD_MAXP ? MASS_SLOTS : 1;
  T.qmass = L.take<double>(2 * (size_t)T.qslots * NP);
  T.qmres = L.take<double>(NP);
  T.qunc = L.take<unsigned long long>(NP);
  T.qupd = L.take<long long>(NP);
  T.active = L.take<int32_t>(1);
  T.tvoff = L.take<int32_t>(NP);
  T.tvn = L.take<int32_t>(NP);
  T.tvcap = (int32_t)std::min<int64_t>(PV, INT32_MAX / 2);
  T.tverts = L.take<int32_t>(T.tvcap);
  T.ntverts = L.take<int32_t>(1);
  T.path = L.take<int32_t>(PV);
  T.qdl = L.take<double>(NP);
  T.ctl = L.take<int32_t>(CTL_SIZE);
  T.tfa = nullptr;
  if (b.opt.streamlines) {
    // streamline points: each pass's region of its point budget (see sl_budget), and a compact pool
    // of the same total that is downloaded
    T.scap = scap;
    T.tfa = L.take<double>(PV);
    T.sroff = L.take<int32_t>(NP + 1);
    T.sreg = L.take<double>(3 * scap);
    T.sst = L.take<int32_t>(NP);
    T.sn = L.take<int32_t>(NP);
    T.soff = L.take<int32_t>(NP);
    T.slen = L.take<double>(NP);
    T.spts = L.take<double>(3 * T.scap);
    T.nspts = L.take<int32_t>(1);
  }
  if (nx > 0) {
    T.xedge = L.take<int32_t>(2 * nx);
    b.r_cyc = L.take<int32_t>(ncyc);
    b.r_coff = L.take<int32_t>(NP);
    b.r_clen = L.take<int32_t>(NP);
    b.r_xcap = L.take<int32_t>(NP);
  }
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

// VLS_DEBUG=1 reports the first failing runtime call of a batch on stderr
bool debug_on() {
  const char *e = std::getenv("VLS_DEBUG");
  return e && e[0] == '1';
}
#define CK(x)                                                                                     \
  do {                                                                                            \
    cudaError_t _e = (x);                                                                         \
    if (_e != cudaSuccess) {                                                                      \
      if (debug_on()) std::fprintf(stderr, "vls: %s failed at api.cu:%d: %s\n", #x, __LINE__,      \
                                   cudaGetErrorString(_e));                                       \
      err = _e;                                                                                   \
      goto fail;                                                                                  \
    }                                                                                             \
  } while (0)

int64_t *g_d2h_counter = nullptr; // bytes downloaded by the call in progress (single-threaded ctx)
template <class T> bool d2h(std::vector<T> &dst, const T *src, size_t n, cudaStream_t st) {
  dst.resize(n);
  if (n == 0) return true;
  if (g_d2h_counter) *g_d2h_counter += (int64_t)(n * sizeof(T));
  return cudaMemcpyAsync(dst.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, st) == cudaSuccess;
}

#define CKR(x)                                                                                    \
  do {                                                                                            \
    cudaError_t _e = (x);                                                                         \
    if (_e != cudaSuccess) {                                                                      \
      if (debug_on()) std::fprintf(stderr, "vls: %s failed at api.cu:%d: %s\n", #x, __LINE__,      \
                                   cudaGetErrorString(_e));                                       \
      return _e;                                                                                  \
    }                                                                                             \
  } while (0)

// Results of single-layer passes (tunnel or refinement), per handle of the batch.  A pass that did
// not run reports (status -1, stop step 0, first vertex 0).
struct PassOut {
  std::vector<int32_t> status, steps, bstar, voff, vn;
  std::vector<int64_t> upd, unc;
  std::vector<double> mres, dl;
  std::vector<int32_t> verts; // vertex cycles (local ids), pool
  std::vector<int32_t> sst;   // streamlines: status (-1 not traced), offset in spts (points), points
  std::vector<int64_t> soff;
  std::vector<int32_t> sn;
  std::vector<double> slen, spts;
  explicit PassOut(int32_t nh)
      : status(nh, -1), steps(nh, 0), bstar(nh, 0), voff(nh, 0), vn(nh, 0), upd(nh, 0), unc(nh, 0), mres(nh, 0.0),
        dl(nh, std::nan("")), sst(nh, -1), soff(nh, 0), sn(nh, 0), slen(nh, 0.0) {}
};
enum PassKind : int { PASS_TUNNEL = 0, PASS_REFINE = 1 };
// a pass's streamline point budget (the closure included) on a mesh of nv vertices: min(16384, nv / 4
// + 64); the loops seen take a few hundredths of nv
int64_t sl_budget(int64_t nv) { return std::min<int64_t>(16384, nv / 4 + 64); }

// A chunk of single-layer passes in flight on one stream: its own device block (from the context's
// stream-ordered pool) and control block, so that chunks on different streams run independently of
// each other and of the initial pass; host-side outputs in pinned memory, filled by asynchronous
// copies ordered after the passes.
struct PassBatch {
  int kind = 0;
  std::vector<int32_t> chunk;
  TDev T{};
  cudaStream_t st = nullptr;
  char *mem = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int32_t *pin_i = nullptr;     // [7 NP + 2]: status, steps, first vertex, cycle offset, length, border edges; ntv, tau
  long long *pin_l = nullptr;   // [2 NP]: rows updated, uncertified decisions
  double *pin_d = nullptr;      // [2 NP]: mass-check residual, offset length change
  int32_t *pin_s = nullptr;     // streamlines [3 NP + 1]: status, points, pool offset; points stored
  double *pin_sl = nullptr;     // streamlines [NP]: length
};

// Enqueue one chunk of passes on stream st (no host wait): tunnel passes (Sec. 3.2) take handle h's
// crossing edges as the border and dom[h] as the domain step; refinement passes (Sec. 3.3) take the
// border from tunnel loop h in tun.  Lays the pass state out in a fresh block, sets the passes up,
// runs them (tunnel.cu), classifies their loops (refine.cu) and queues the copies of the results.
cudaError_t enqueue_chunk(vls_ctx *ctx, Batch &b, int kind, const std::vector<int32_t> &chunk,
                          const std::vector<int32_t> &h_hprob, const std::vector<int32_t> &dom,
                          const std::vector<int32_t> &h_hoff, const std::vector<int32_t> &h_hn, const PassOut *tun,
                          cudaStream_t st, PassBatch &pb) {
  Dev &d = b.d;
  const int32_t NP = (int32_t)chunk.size();
  pb.kind = kind;
  pb.chunk = chunk;
  pb.st = st;
  // set-up tables, staged in pinned memory (a copy from pageable memory would wait for the stream)
  int32_t ncyc_total = 0;
  if (kind == PASS_REFINE)
    for (int32_t h : chunk) ncyc_total += tun->vn[h];
  int32_t *ht = static_cast<int32_t *>(ctx->pinned.take(sizeof(int32_t) * (size_t)(11 * NP + 2 + ncyc_total)));
  pb.pin_i = static_cast<int32_t *>(ctx->pinned.take(sizeof(int32_t) * (size_t)(7 * NP + 2)));
  pb.pin_l = static_cast<long long *>(ctx->pinned.take(sizeof(long long) * (size_t)(2 * NP)));
  pb.pin_d = static_cast<double *>(ctx->pinned.take(sizeof(double) * (size_t)(2 * NP)));
  if (!ht || !pb.pin_i || !pb.pin_l || !pb.pin_d) return cudaErrorMemoryAllocation;
  pb.pin_s = nullptr;
  pb.pin_sl = nullptr;
  if (b.opt.streamlines) {
    pb.pin_s = static_cast<int32_t *>(ctx->pinned.take(sizeof(int32_t) * (size_t)(3 * NP + 1)));
    pb.pin_sl = static_cast<double *>(ctx->pinned.take(sizeof(double) * (size_t)NP));
    if (!pb.pin_s || !pb.pin_sl) return cudaErrorMemoryAllocation;
  }
  int32_t *pbase = ht, *pprob = ht + NP + 1, *pstep = pprob + NP, *pcoff = pstep + NP, *pcn = pcoff + NP;
  int32_t *heoff = pcn + NP, *hen = heoff + NP, *rcoff = hen + NP, *rclen = rcoff + NP, *xcap = rclen + NP;
  int32_t *sroff = xcap + NP; // [NP + 1]
  int32_t *rcyc = sroff + NP + 1;
  int64_t PV = 0, ncut = 0, nx = 0, stot = 0;
  int32_t nc = 0;
  for (int32_t q = 0; q < NP; ++q) {
    const int32_t h = chunk[q], p = h_hprob[h];
    pbase[q] = (int32_t)PV;
    pprob[q] = p;
    pstep[q] = dom[h];
    if (kind == PASS_TUNNEL) {
      heoff[q] = h_hoff[h];
      hen[q] = h_hn[h];
      pcn[q] = 2 * h_hn[h];
      pcoff[q] = (int32_t)ncut;
      ncut += 2 * h_hn[h];
    } else {
      const int32_t len = tun->vn[h];
      rcoff[q] = nc;
      rclen[q] = len;
      for (int32_t i = 0; i < len; ++i) rcyc[nc++] = tun->verts[tun->voff[h] + i] + b.voff[p];
      // a cycle vertex has at most degree - 2 neighbours on one side (degree <= LV_MAX, checked)
      xcap[q] = (LV_MAX - 2) * std::max(len, 1);
      heoff[q] = (int32_t)nx;
      nx += xcap[q];
      pcoff[q] = (int32_t)ncut;
      ncut += 2 * (int64_t)xcap[q];
    }
    sroff[q] = (int32_t)stot;
    stot += sl_budget(b.voff[p + 1] - b.voff[p]);
    PV += b.voff[p + 1] - b.voff[p];
  }
  pbase[NP] = (int32_t)PV;
  sroff[NP] = (int32_t)stot;
  if (!b.opt.streamlines) stot = 0;
  if (PV >= INT32_MAX / 2 || ncut >= INT32_MAX / 2 || stot >= INT32_MAX / 4) {
    if (debug_on()) std::fprintf(stderr, "vls: pass chunk of %lld pass-vertices\n", (long long)PV);
    return cudaErrorMemoryAllocation;
  }
  Layout L{nullptr, true};
  layout_tunnels(L, b, NP, PV, ncut, nx, nc, stot);
  CKR(cudaEventCreateWithFlags(&pb.ev0, cudaEventDefault));
  CKR(cudaEventCreateWithFlags(&pb.ev1, cudaEventDefault));
  CKR(cudaEventRecord(pb.ev0, st));
  CKR(cudaMallocFromPoolAsync(reinterpret_cast<void **>(&pb.mem), L.bytes + 256, ctx->pool, st));
  Arena a;
  a.base = pb.mem;
  a.cap = L.bytes + 256;
  Layout L2{&a, false};
  layout_tunnels(L2, b, NP, PV, ncut, nx, nc, stot);
  pb.T = b.td;
  TDev &T = pb.T;
  T.err = d.err;
  if (kind == PASS_TUNNEL) T.xedge = d.hedge;
  auto up = [&](const int32_t *dst, const int32_t *src, size_t n) {
    b.h2d += (int64_t)(sizeof(int32_t) * n);
    return cudaMemcpyAsync(const_cast<int32_t *>(dst), src, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
  };
  CKR(up(T.pbase, pbase, NP + 1));
  CKR(up(T.pprob, pprob, NP));
  CKR(up(T.pstep, pstep, NP));
  CKR(up(T.pcoff, pcoff, NP));
  CKR(up(T.heoff, heoff, NP));
  if (T.tfa) CKR(up(T.sroff, sroff, NP + 1));
  if (kind == PASS_TUNNEL) {
    CKR(up(T.pcn, pcn, NP));
    CKR(up(T.hen, hen, NP));
  }
  CKR(cudaMemsetAsync(T.ctl, 0, sizeof(int32_t) * CTL_SIZE, st));
  k_fill_i32<<<1, 32, 0, st>>>(T.ctl + CTL_TLIMIT, 1, b.opt.max_pass_steps); VLS_LAUNCH(b);
  CKR(cudaMemsetAsync(T.flag, 0, (size_t)PV, st));
  if (T.phih) CKR(cudaMemsetAsync(T.phih, 0, sizeof(__nv_bfloat16) * PV, st));
  else if (T.phif) CKR(cudaMemsetAsync(T.phif, 0, sizeof(float) * PV, st));
  else CKR(cudaMemsetAsync(T.phi, 0, sizeof(double) * PV, st));
  CKR(cudaMemsetAsync(T.T, 0xff, sizeof(int32_t) * PV, st));
  CKR(cudaMemsetAsync(T.stamp, 0, sizeof(int32_t) * PV, st));
  CKR(cudaMemsetAsync(T.nf, 0, sizeof(int32_t) * 2, st));
  CKR(cudaMemsetAsync(T.qdone, 0, sizeof(int32_t) * NP, st));
  CKR(cudaMemsetAsync(T.qsteps, 0, sizeof(int32_t) * NP, st));
  CKR(cudaMemsetAsync(T.qstatus, 0xff, sizeof(int32_t) * NP, st));
  k_fill_i32<<<(NP + 255) / 256, 256, 0, st>>>(T.qbstar, NP, 0x7fffffff); VLS_LAUNCH(b);
  CKR(cudaMemsetAsync(T.qcnt, 0, sizeof(int32_t) * 2 * NP, st));
  CKR(cudaMemsetAsync(T.qmass, 0, sizeof(double) * 2 * T.qslots * NP, st));
  CKR(cudaMemsetAsync(T.qmres, 0, sizeof(double) * NP, st));
  CKR(cudaMemsetAsync(T.qunc, 0, sizeof(unsigned long long) * NP, st));
  CKR(cudaMemsetAsync(T.qupd, 0, sizeof(long long) * NP, st));
  CKR(cudaMemsetAsync(T.ntverts, 0, sizeof(int32_t), st));
  CKR(cudaMemsetAsync(T.tvn, 0, sizeof(int32_t) * NP, st));
  if (kind == PASS_REFINE) {
    CKR(up(b.r_cyc, rcyc, nc));
    CKR(up(b.r_coff, rcoff, NP));
    CKR(up(b.r_clen, rclen, NP));
    CKR(up(b.r_xcap, xcap, NP));
    CKR(launch_refine_prep(b, T, st, b.r_cyc, b.r_coff, b.r_clen, const_cast<int32_t *>(T.xedge), b.r_xcap,
                           const_cast<int32_t *>(T.hen), const_cast<int32_t *>(T.pcn)));
  }
  int32_t *pi = pb.pin_i;
  CKR(run_tunnels(b, T, st, pi + 7 * NP + 1, &pb.ge));
  CKR(launch_classify_passes(b, T, st, d.vn, d.pmedge));
  auto dn = [&](void *dst, const void *src, size_t bytes) {
    b.d2h += (int64_t)bytes;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st);
  };
  CKR(dn(pi, T.qstatus, sizeof(int32_t) * NP));
  CKR(dn(pi + NP, T.qsteps, sizeof(int32_t) * NP));
  CKR(dn(pi + 2 * NP, T.qbstar, sizeof(int32_t) * NP));
  CKR(dn(pi + 3 * NP, T.tvoff, sizeof(int32_t) * NP));
  CKR(dn(pi + 4 * NP, T.tvn, sizeof(int32_t) * NP));
  CKR(dn(pi + 5 * NP, T.hen, sizeof(int32_t) * NP));
  CKR(dn(pi + 7 * NP, T.ntverts, sizeof(int32_t)));
  CKR(dn(pb.pin_l, T.qupd, sizeof(long long) * NP));
  CKR(dn(pb.pin_l + NP, T.qunc, sizeof(long long) * NP));
  CKR(dn(pb.pin_d, T.qmres, sizeof(double) * NP));
  CKR(dn(pb.pin_d + NP, T.qdl, sizeof(double) * NP));
  if (T.tfa) {
    CKR(dn(pb.pin_s, T.sst, sizeof(int32_t) * NP));
    CKR(dn(pb.pin_s + NP, T.sn, sizeof(int32_t) * NP));
    CKR(dn(pb.pin_s + 2 * NP, T.soff, sizeof(int32_t) * NP));
    CKR(dn(pb.pin_s + 3 * NP, T.nspts, sizeof(int32_t)));
    CKR(dn(pb.pin_sl, T.slen, sizeof(double) * NP));
  }
  CKR(cudaEventRecord(pb.ev1, st));
  return cudaSuccess;
}

// Wait for a chunk, move its results into out (per handle), download its loop vertices on the
// download stream and release its device block.  *tau_sum += its steps (launch accounting); *ms +=
// its device time.
cudaError_t finish_chunk(vls_ctx *ctx, Batch &b, PassBatch &pb, PassOut &out, int32_t *tau_sum, double *ms) {
  CKR(cudaEventSynchronize(pb.ev1));
  const int32_t NP = (int32_t)pb.chunk.size();
  const int32_t *pi = pb.pin_i;
  const int32_t ntv = std::min(pi[7 * NP], pb.T.tvcap);
  *tau_sum += pi[7 * NP + 1] - 1;
  float t = 0.f;
  if (cudaEventElapsedTime(&t, pb.ev0, pb.ev1) == cudaSuccess) *ms += t;
  const size_t tv0 = out.verts.size();
  out.verts.resize(tv0 + (size_t)ntv);
  if (ntv) {
    CKR(cudaMemcpyAsync(out.verts.data() + tv0, pb.T.tverts, sizeof(int32_t) * ntv, cudaMemcpyDeviceToHost, ctx->st3));
    b.d2h += (int64_t)sizeof(int32_t) * ntv;
  }
  const int64_t ns = pb.pin_s ? std::min<int64_t>(pb.pin_s[3 * NP], pb.T.scap) : 0;
  const size_t sp0 = out.spts.size() / 3;
  if (ns > 0) {
    out.spts.resize(3 * (sp0 + (size_t)ns));
    CKR(cudaMemcpyAsync(out.spts.data() + 3 * sp0, pb.T.spts, sizeof(double) * 3 * ns, cudaMemcpyDeviceToHost, ctx->st3));
    b.d2h += (int64_t)sizeof(double) * 3 * ns;
  }
  CKR(cudaFreeAsync(pb.mem, ctx->st3));
  CKR(cudaStreamSynchronize(ctx->st3));
  pb.mem = nullptr;
  for (int32_t q = 0; q < NP; ++q) {
    const int32_t h = pb.chunk[q];
    out.status[h] = pi[q];
    out.steps[h] = pi[NP + q];
    out.bstar[h] = pi[2 * NP + q] == 0x7fffffff ? -1 : pi[2 * NP + q];
    out.voff[h] = (int32_t)tv0 + pi[3 * NP + q];
    out.vn[h] = pi[4 * NP + q];
    out.upd[h] = pb.pin_l[q];
    out.unc[h] = pb.pin_l[NP + q];
    out.mres[h] = pb.pin_d[q];
    out.dl[h] = pb.pin_d[NP + q];
    if (pb.pin_s) {
      const int32_t *ps = pb.pin_s;
      const bool ok = ps[q] == VLS_OK && (int64_t)ps[2 * NP + q] + ps[NP + q] <= ns;
      out.sst[h] = ps[q] == VLS_OK && !ok ? VLS_ELAYERS : ps[q];
      out.sn[h] = ok ? ps[NP + q] : 0;
      out.soff[h] = (int64_t)sp0 + (ok ? ps[2 * NP + q] : 0);
      out.slen[h] = ok ? pb.pin_sl[q] : 0.0;
    }
    if (pb.kind == PASS_REFINE && pi[5 * NP + q] == 0) { // no border: a degenerate tunnel cycle
      out.status[h] = VLS_ELOOPFAIL;
      out.steps[h] = 0;
      out.bstar[h] = -1;
      out.vn[h] = 0;
      out.dl[h] = std::nan("");
    }
  }
  if (pb.ge) cudaGraphExecDestroy(pb.ge);
  pb.ge = nullptr;
  cudaEventDestroy(pb.ev0);
  cudaEventDestroy(pb.ev1);
  pb.ev0 = pb.ev1 = nullptr;
  return cudaSuccess;
}
#undef CKR

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

// ---- autotuner
// Launch shapes chosen by measurement, kept per device, precision and batch size class (total
// vertices rounded up to a power of two) for the life of the process.  Until a candidate wins,
// every kernel uses lane-group hooking and as many blocks per SM as fit.
struct TuneEntry {
  int dev = -1, vclass = -1, prec = -1;
  Batch::Shape shape[KK_COUNT_KINDS];
  int hook_variant = 2;
  int rpw = 32;
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;

constexpr int TUNE_STEPS = 600;
// (threads per block, blocks per SM (64: as many as fit), band union-find variant, frontier
// rows per warp of the one-thread-per-row kernels)
const int kTuneCands[][4] = {{128, 64, 2, 32}, {256, 64, 2, 32}, {64, 64, 2, 32}, {128, 64, 1, 32}, {128, 4, 2, 32},
                             {128, 64, 2, 16}, {128, 64, 2, 8},  {256, 64, 2, 8}, {64, 64, 2, 8}};

// Each candidate launch shape / union-find variant runs the first TUNE_STEPS steps of this
// batch's initial pass the way real calls run (device-driven graph, every kernel with that
// shape), timed with CUDA events around the whole call; the fastest candidate is kept.  Per
// kernel timings from host-launched steps mislead here: a graph hides launch costs that host
// launches expose, and the early steps' small frontiers favour small grids.
void autotune(vls_ctx *ctx, int32_t n_mesh, const vls_mesh *meshes, const int32_t *seeds, const int32_t *spm,
              TuneEntry &te) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return;
  float best = 1e30f;
  for (const auto &c : kTuneCands) {
    vls_options o = ctx->opt;
    o.threads = c[0];
    o.blocks_per_sm = c[1];
    o.hook_variant = c[2];
    o.rows_per_warp = c[3];
    o.max_steps = TUNE_STEPS;
    o.tunnels = 0;
    o.profile = 0;
    o.host_loop = 0;
    o.keep_state = 0;
    o.record_steps = 0;
    vls_ctx *t = nullptr;
    if (vls_create(&t, &o, ctx->st) != VLS_OK) continue;
    vls_result *r = nullptr;
    vls_detect_batch(t, n_mesh, meshes, seeds, spm, &r); // first run sizes the arena
    if (r) vls_result_free(r);
    r = nullptr;
    cudaEventRecord(e0, ctx->st);
    const vls_status st = vls_detect_batch(t, n_mesh, meshes, seeds, spm, &r);
    cudaEventRecord(e1, ctx->st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    if (st == VLS_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best) {
      best = ms;
      for (int k = 0; k < KK_COUNT_KINDS; ++k) {
        te.shape[k].threads = c[0];
        te.shape[k].bps = c[1];
      }
      te.hook_variant = c[2];
      te.rpw = c[3];
    }
    if (r) vls_result_free(r);
    vls_destroy(t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

}  // namespace

extern "C" vls_status vls_detect_batch(vls_ctx *ctx, int32_t n_mesh, const vls_mesh *meshes, const int32_t *seeds,
                                       const int32_t *seeds_per_mesh, vls_result **out) {
  if (!ctx || !out || n_mesh <= 0 || !meshes || !seeds || !seeds_per_mesh) return VLS_EINVAL;
  *out = nullptr;
  // launch shapes: explicit options, else the autotuned table of this device / size class
  TuneEntry tuned;
  bool have_tuned = false;
  if (ctx->opt.threads == 0 && ctx->opt.blocks_per_sm == 0 && ctx->opt.autotune) {
    int dev = 0;
    cudaGetDevice(&dev);
    int64_t vt = 0;
    for (int32_t m = 0, si = 0; m < n_mesh; ++m) {
      if (seeds_per_mesh[m] < 0) return VLS_EINVAL;
      vt += (int64_t)std::max<int64_t>(meshes[m].nv, 0) * seeds_per_mesh[m];
      si += seeds_per_mesh[m];
    }
    int vclass = 0;
    while (vclass < 62 && (int64_t(1) << vclass) < vt) ++vclass;
    const int prec = (int)ctx->opt.precision;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      for (const TuneEntry &e : g_tune)
        if (e.dev == dev && e.vclass == vclass && e.prec == prec) {
          tuned = e;
          have_tuned = true;
        }
    }
    if (!have_tuned) {
      tuned.dev = dev;
      tuned.vclass = vclass;
      tuned.prec = prec;
      autotune(ctx, n_mesh, meshes, seeds, seeds_per_mesh, tuned);
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune.push_back(tuned);
      have_tuned = true;
    }
  }
  vls_result *res = new (std::nothrow) vls_result();
  if (!res) return VLS_ENOMEM;
  ctx->pinned.reset(); // the previous call's copies have completed
  // problems (mesh-major, seed-minor); those failing host checks never reach the device
  std::vector<int32_t> pm, ps, pres_status;
  int64_t si = 0;
  for (int32_t m = 0; m < n_mesh; ++m) {
    if (seeds_per_mesh[m] < 0) { delete res; return VLS_EINVAL; }
    for (int32_t k = 0; k < seeds_per_mesh[m]; ++k, ++si) {
      pm.push_back(m);
      ps.push_back(seeds[si]);
    }
  }
  const int32_t NPROB = (int32_t)pm.size();
  res->p.resize(NPROB);
  Batch b;
  b.prof.pool = &ctx->evpool;
  b.prof.on = ctx->opt.profile != 0;
  {
    const char *hl = std::getenv("VLS_HOST_LOOP");
    // kernel timing needs CUDA events around single launches: profiling runs the host loop
    b.host_loop = ctx->opt.profile != 0 || ctx->opt.host_loop != 0 || (hl && hl[0] == '1');
  }
  g_d2h_counter = &b.d2h;
  b.st = ctx->st;
  b.opt = ctx->opt;
  b.arena = &ctx->arena;
  b.sm_count = ctx->sm;
  // row kernels (one thread per frontier row): small blocks spread a few thousand rows over
  // every SM; lane-group kernels (GL lanes per row): 256-thread blocks
  if (have_tuned) {
    // the tuner times the initial pass only: the pass kernels keep the default shapes
    for (int k = 0; k < KK_COUNT_KINDS; ++k)
      if (k != KK_TUPDATE && k != KK_TAPPLY && k != KK_TFRONTIER) b.shape[k] = tuned.shape[k];
    b.hook_variant = tuned.hook_variant;
    b.d.rpw = tuned.rpw;
  } else {
    b.d.rpw = 32;
    for (int k = 0; k < KK_COUNT_KINDS; ++k) {
      b.shape[k].threads = ctx->opt.threads;
      b.shape[k].bps = ctx->opt.blocks_per_sm;
    }
  }
  if (ctx->opt.hook_variant == 1 || ctx->opt.hook_variant == 2) b.hook_variant = ctx->opt.hook_variant;
  if (ctx->opt.rows_per_warp != 0) b.d.rpw = ctx->opt.rows_per_warp;
  configure_initial(b);
  configure_events(b);
  configure_tunnel(b);
  {
    double c[4];
    vls_constants(&ctx->opt, c);
    Params &P = b.prm;
    P.mu = ctx->opt.mu;
    P.e = ctx->opt.e;
    P.w = ctx->opt.w;
    P.ah = ctx->opt.a * ctx->opt.a / 2.0;
    P.dt = c[2];
    P.s = c[3];
    P.eps0 = ctx->opt.eps0;
    P.one_m_eps = 1.0 - ctx->opt.eps0;
    P.theta = ctx->opt.theta_iso;
    P.lv[0] = 0.0;
    for (int k = 1; k <= LV_MAX; ++k) P.lv[k] = P.s / (double)k;
    P.mv[0] = 0.0;
    for (int k = 1; k <= LV_MAX; ++k) P.mv[k] = (double)k / P.s;
    P.mun[0] = 0.0;
    for (int k = 1; k <= KMAX + 1; ++k) P.mun[k] = P.mu / (double)k;
    P.margin = ctx->opt.recheck_margin;
    P.offset = ctx->opt.offset;
    P.drift = ctx->opt.precision == VLS_FP64 ? 0.0
              : ctx->opt.drift_bound > 0.0 ? ctx->opt.drift_bound
              : ctx->opt.precision == VLS_BF16_RECHECK ? 2e-2 : 1e-6;
    P.f_e = (float)P.e;
    P.f_w = (float)P.w;
    P.f_ah = (float)P.ah;
    P.f_dt = (float)P.dt;
    P.f_s = (float)P.s;
    P.f_eps0 = (float)P.eps0;
    P.f_one_m_eps = (float)P.one_m_eps;
    P.f_theta = (float)P.theta;
    P.f_margin = (float)P.margin;
    P.f_drift = (float)P.drift;
    for (int k = 0; k <= LV_MAX; ++k) P.f_lv[k] = (float)P.lv[k];
    for (int k = 0; k <= KMAX + 1; ++k) P.f_mun[k] = (float)P.mun[k];
  }
  std::vector<int32_t> dev_probs; // result index of each device problem
  int64_t V = 0, NF = 0, Lc = 0;
  for (int32_t i = 0; i < NPROB; ++i) {
    const vls_mesh &m = meshes[pm[i]];
    ProbResult &r = res->p[i];
    r.nv = m.nv;
    if (!m.X || !m.F || m.nv < 4 || m.nf < 4 || ps[i] < 0 || ps[i] >= m.nv) { r.status = VLS_EINVAL; continue; }
    b.voff.push_back((int32_t)V);
    b.foff.push_back((int32_t)NF);
    const int32_t lc = (int32_t)std::min<int64_t>(256 + m.nv / 64, 1 << 24);
    b.lbase.push_back((int32_t)Lc);
    b.lcap.push_back(lc);
    b.seed.push_back(ps[i]);
    b.mesh_of.push_back(pm[i]);
    dev_probs.push_back(i);
    V += m.nv;
    NF += m.nf;
    Lc += lc;
  }
  if (dev_probs.empty()) { *out = res; return VLS_OK; }
  if (V >= INT32_MAX / 2 || 3 * NF >= INT32_MAX) { delete res; return VLS_EINVAL; }
  b.voff.push_back((int32_t)V);
  b.foff.push_back((int32_t)NF);
  b.P = (int32_t)dev_probs.size();
  b.V = (int32_t)V;
  b.NF = (int32_t)NF;
  b.nnz = 3 * NF;
  b.Lcap = (int32_t)Lc;
  b.d.P = b.P;
  b.d.V = b.V;
  b.d.NF = b.NF;
  b.d.nnz = b.nnz;
  b.d.Lcap = b.Lcap;
  b.d.record = ctx->opt.record_steps ? 1 : 0;
  b.d.rcap = b.d.record ? std::min(ctx->opt.max_steps, 1 << 20) : 0;

  cudaError_t err = cudaSuccess;
  cudaStream_t st = b.st;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  std::vector<int32_t> stage, h_rpb, h_status, h_steps, h_nodes_cnt;
  int32_t h_nn = 0, h_nh = 0;
  int32_t tunnel_tau = 0, refine_tau = 0;
  std::vector<int32_t> h_hprob, h_hstep, h_hlayer, h_hnode, h_hoff, h_hn, h_hvoff, h_hvn;
  std::vector<double> h_hlen, h_hdl;
  {
    Layout L{&ctx->arena, true};
    layout_batch(L, b);
    CK(ctx->arena.reserve(L.bytes));
    ctx->arena.reset();
    Layout L2{&ctx->arena, false};
    layout_batch(L2, b);
  }
  for (int i = 0; i < 6; ++i) CK(cudaEventCreate(&ev[i]));
  if (const char *pz = std::getenv("VLS_POISON"))
    if (pz[0] == '1') CK(cudaMemsetAsync(ctx->arena.base, 0xab, ctx->arena.cap, st)); // debug: expose unset reads
  {
    Dev &d = b.d;
    // inputs into the union graph: a host mesh crosses to the device once, for its first problem;
    // the mesh's other seeds copy that problem's slots on the device
    {
      std::vector<int32_t> first_of(n_mesh, -1);
      for (int32_t q = 0; q < b.P; ++q) {
        const int32_t mi = b.mesh_of[q];
        const vls_mesh &m = meshes[mi];
        const int32_t q0 = first_of[mi];
        double *xq = const_cast<double *>(d.X) + 3 * (int64_t)b.voff[q];
        int32_t *fq = const_cast<int32_t *>(d.F) + 3 * (int64_t)b.foff[q];
        if (q0 >= 0 && !m.device) {
          CK(cudaMemcpyAsync(xq, d.X + 3 * (int64_t)b.voff[q0], sizeof(double) * 3 * m.nv, cudaMemcpyDeviceToDevice, st));
          CK(cudaMemcpyAsync(fq, d.F + 3 * (int64_t)b.foff[q0], sizeof(int32_t) * 3 * m.nf, cudaMemcpyDeviceToDevice, st));
          continue;
        }
        first_of[mi] = q;
        const cudaMemcpyKind kx = m.device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (!m.device) b.h2d += (int64_t)(sizeof(double) * 3 * m.nv + sizeof(int32_t) * 3 * m.nf);
        CK(cudaMemcpyAsync(xq, m.X, sizeof(double) * 3 * m.nv, kx, st));
        CK(cudaMemcpyAsync(fq, m.F, sizeof(int32_t) * 3 * m.nf, kx, st));
      }
    }
    CK(cudaMemcpyAsync(const_cast<int32_t *>(d.voff), b.voff.data(), sizeof(int32_t) * (b.P + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(const_cast<int32_t *>(d.foff), b.foff.data(), sizeof(int32_t) * (b.P + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(const_cast<int32_t *>(d.lbase), b.lbase.data(), sizeof(int32_t) * b.P, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(const_cast<int32_t *>(d.lcap), b.lcap.data(), sizeof(int32_t) * b.P, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(const_cast<int32_t *>(d.seed), b.seed.data(), sizeof(int32_t) * b.P, cudaMemcpyHostToDevice, st));
    b.h2d += (int64_t)sizeof(int32_t) * (2 * (b.P + 1) + 3 * b.P);
    CK(cudaEventRecord(ev[0], st));
    // ---- a0: operator
    int32_t *stage_d = d.pev; // 5 * P ints needed: pev holds 4 * P, spill into pupd (2 * P ints)
    stage_d = reinterpret_cast<int32_t *>(d.ophi); // V * KMAX doubles: ample scratch before the first step
    CK(build_operator(b, stage_d));
    CK(launch_vnormals(b, d.vn, d.elen, d.pmedge));
    stage.resize(5 * (size_t)b.P);
    CK(cudaMemcpyAsync(stage.data(), stage_d, sizeof(int32_t) * 5 * b.P, cudaMemcpyDeviceToHost, st));
    b.d2h += (int64_t)sizeof(int32_t) * (6 * b.P + 1);
    h_rpb.resize(b.P + 1);
    for (int32_t q = 0; q <= b.P; ++q)
      CK(cudaMemcpyAsync(&h_rpb[q], d.rp + b.voff[q], sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    h_status.assign(b.P, 0);
    for (int32_t q = 0; q < b.P; ++q) {
      const int32_t *s = &stage[5 * q];
      int32_t stt = 0;
      if (s[0]) stt = VLS_EINVAL;
      else if (s[1]) stt = VLS_ENONORIENTABLE;
      else if (s[2]) stt = VLS_ENOTMANIFOLD;
      else if (s[3] != INT_MAX) stt = s[3] & 15;
      else if (s[4] != 1) stt = VLS_EDISCONNECTED;
      h_status[q] = stt;
      const int64_t E = (int64_t)(h_rpb[q + 1] - h_rpb[q]) / 2;
      const vls_mesh &m = meshes[b.mesh_of[q]];
      res->p[dev_probs[q]].genus = (int32_t)((2 - (m.nv - E + m.nf)) / 2);
    }
    CK(cudaEventRecord(ev[1], st));
    // ---- state init
    CK(cudaMemcpyAsync(d.pstatus, h_status.data(), sizeof(int32_t) * b.P, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(d.lay, 0, sizeof(int32_t) * b.V, st));
    if (d.phih) CK(cudaMemsetAsync(d.phih, 0, sizeof(__nv_bfloat16) * b.V, st));
    else if (d.phif) CK(cudaMemsetAsync(d.phif, 0, sizeof(float) * b.V, st));
    else CK(cudaMemsetAsync(d.phi, 0, sizeof(double) * b.V, st));
    CK(cudaMemsetAsync(d.nrecheck, 0, sizeof(unsigned long long) * 2, st));
    CK(cudaMemsetAsync(d.punc, 0, sizeof(unsigned long long) * b.P, st));
    CK(cudaMemsetAsync(d.runc, 0, sizeof(int32_t) * b.P, st));
    CK(cudaMemsetAsync(d.pmass, 0, sizeof(double) * 2 * d.mslots * b.P, st));
    CK(cudaMemsetAsync(d.pmres, 0, sizeof(double) * b.P, st));
    CK(cudaMemsetAsync(d.cover, 0xff, sizeof(int32_t) * b.V, st));
    CK(cudaMemsetAsync(d.stamp, 0, sizeof(int32_t) * b.V, st));
    CK(cudaMemsetAsync(d.fmark, 0, sizeof(int32_t) * b.V, st));
    CK(cudaMemsetAsync(d.multi, 0xff, sizeof(int32_t) * b.V, st));
    CK(cudaMemsetAsync(d.nlay, 0, sizeof(int32_t) * b.V, st)); // layer ids stay in range before the first write
    CK(cudaMemsetAsync(d.lstate, 0, sizeof(int32_t) * b.Lcap, st));
    CK(cudaMemsetAsync(d.lfwd, 0, sizeof(int32_t) * b.Lcap, st));
    CK(cudaMemsetAsync(d.lcnt, 0, sizeof(int32_t) * b.Lcap, st));
    CK(cudaMemsetAsync(d.lcnt + b.Lcap, 0xff, sizeof(int32_t) * b.Lcap, st));
    CK(cudaMemsetAsync(d.pdone, 0, sizeof(int32_t) * b.P, st));
    CK(cudaMemsetAsync(d.lcount, 0, sizeof(int32_t) * b.P, st));
    CK(cudaMemsetAsync(d.psteps, 0, sizeof(int32_t) * b.P, st));
    CK(cudaMemsetAsync(d.pnodes, 0, sizeof(int32_t) * b.P, st));
    CK(cudaMemsetAsync(d.pfront, 0, sizeof(int32_t) * 2 * b.P, st));
    CK(cudaMemsetAsync(d.pmerge, 0, sizeof(int32_t) * b.P, st));
    CK(cudaMemsetAsync(d.pupd, 0, sizeof(int64_t) * b.P, st));
    CK(cudaMemsetAsync(d.pev, 0, sizeof(int32_t) * 4 * b.P, st));
    CK(cudaMemsetAsync(d.nfront, 0, sizeof(int32_t) * 2, st));
    CK(cudaMemsetAsync(d.ncoll, 0, sizeof(int32_t), st));
    CK(cudaMemsetAsync(d.nnodes, 0, sizeof(int32_t), st));
    CK(cudaMemsetAsync(d.nhand, 0, sizeof(int32_t), st));
    CK(cudaMemsetAsync(d.nhedge, 0, sizeof(int32_t), st));
    CK(cudaMemsetAsync(d.rhash, 0, sizeof(unsigned long long) * b.P, st));
    CK(cudaMemsetAsync(d.rband, 0, sizeof(int32_t) * b.P, st));
    CK(cudaMemsetAsync(d.err, 0, sizeof(int32_t) * 4, st));
    CK(cudaMemsetAsync(d.nalive, 0, sizeof(int32_t) * b.P, st));
    CK(cudaMemsetAsync(d.nbl, 0, sizeof(int32_t) * b.P, st));
    {
      int32_t ctl[CTL_SIZE] = {};
      ctl[CTL_LIMIT] = ctx->opt.max_steps;
      ctl[CTL_TLIMIT] = ctx->opt.max_pass_steps;
      CK(cudaMemcpyAsync(d.ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, st));
      b.h2d += (int64_t)sizeof(ctl);
    }
    if (d.record) CK(cudaMemsetAsync(d.rec, 0, sizeof(long long) * 5 * (size_t)b.P * d.rcap, st));
    CK(init_state(b));
    // ---- initial pass, and the single-layer passes (Sec. 3.2, 3.3) of the handles found so far
    // running beside it: the initial pass is a chain of small latency-bound steps that leaves most
    // of the GPU idle, so with step loops as graphs it runs in segments of SEG steps; after each
    // segment the new handles' tunnel passes start on the pass streams (their domain, the area
    // covered by the handle's step, no longer changes), and a problem whose initial pass has
    // ended gets the refinement passes of its finished tunnel loops (their domain is the whole
    // surface).  Passes are independent of one another and of the order they run in.
    PassOut tun(d.hcap), ref(d.hcap);
    std::vector<int32_t> pass_h, pass_dom(d.hcap, 0), per_prob(b.P, 0), pdone(b.P, 0);
    std::vector<int32_t> pend_t, pend_r, retry;
    std::vector<PassBatch> inflight;
    double ms_t = 0.0, ms_r = 0.0;
    int next_sp = 0;
    int64_t inflight_bytes = 0;
    // passes run in chunks whose dense per-pass state (one entry per vertex of the pass's problem:
    // at most 52 B in the FP64 form, 72 B with the streamlines' arrival times and point regions)
    // fits a bound set by the free device memory; chunks in flight together stay within twice that
    const int64_t pv_bytes = ctx->opt.streamlines ? 72 : 52;
    int64_t pv_cap = (int64_t(1) << 30) - (int64_t(1) << 20); // pass-vertex ids stay below INT32_MAX / 2
    {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) pv_cap = std::min<int64_t>(pv_cap, (int64_t)(fr / 4 / pv_bytes));
      // VLS_PASS_VERTS overrides the bound (smaller chunks; the results do not change)
      if (const char *ev = std::getenv("VLS_PASS_VERTS")) pv_cap = std::atoll(ev);
      pv_cap = std::max<int64_t>(pv_cap, 1);
    }
    const int64_t inflight_cap = 2 * pv_cap * pv_bytes;
    h_hprob.assign(d.hcap, 0);
    h_hstep.assign(d.hcap, 0);
    h_hoff.assign(d.hcap, 0);
    h_hn.assign(d.hcap, 0);
    int32_t seen = 0;
    // take the handles [seen, nh) in: their tables, and their tunnel passes (problems still OK)
    auto admit = [&](int32_t nh, const std::vector<int32_t> &pst) -> cudaError_t {
      nh = std::min(nh, d.hcap);
      if (nh <= seen) return cudaSuccess;
      const size_t n = (size_t)(nh - seen);
      cudaError_t e = cudaMemcpy(h_hprob.data() + seen, d.hprob + seen, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(h_hstep.data() + seen, d.hstep + seen, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(h_hoff.data() + seen, d.hoff + seen, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(h_hn.data() + seen, d.hn + seen, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
      b.d2h += (int64_t)(16 * n);
      if (e != cudaSuccess) return e;
      for (int32_t h = seen; h < nh; ++h) {
        const int32_t p = h_hprob[h];
        if (!ctx->opt.tunnels || pst[p] != VLS_OK) continue;
        if (ctx->opt.max_passes > 0 && per_prob[p]++ >= ctx->opt.max_passes) continue;
        pass_h.push_back(h);
        pass_dom[h] = h_hstep[h];
        pend_t.push_back(h);
      }
      seen = nh;
      return cudaSuccess;
    };
    auto chunk_bytes = [&](const std::vector<int32_t> &hs) {
      int64_t pv = 0;
      for (int32_t h : hs) pv += b.voff[h_hprob[h] + 1] - b.voff[h_hprob[h]];
      return pv_bytes * pv;
    };
    // start chunks of the pending handles (in order) while the in-flight bound allows (one chunk always
    // starts when none is in flight); refinements wait for their problem's initial pass to end;
    // after_ev: the initial-pass point the chunks must follow
    auto launch = [&](int kind, std::vector<int32_t> &pend, const std::vector<int32_t> &dom,
                      cudaEvent_t after_ev) -> cudaError_t {
      std::vector<int32_t> keep;
      size_t i = 0;
      while (i < pend.size()) {
        std::vector<int32_t> chunk;
        int64_t pv = 0;
        size_t j = i;
        for (; j < pend.size(); ++j) {
          const int32_t h = pend[j], p = h_hprob[h];
          if (kind == PASS_REFINE && !pdone[p]) { keep.push_back(h); continue; }
          const int64_t nvp = b.voff[p + 1] - b.voff[p];
          if (!chunk.empty() && pv + nvp > pv_cap) break;
          chunk.push_back(h);
          pv += nvp;
        }
        i = j;
        if (chunk.empty()) continue;
        const int64_t bytes = chunk_bytes(chunk);
        if (!inflight.empty() && inflight_bytes + bytes > inflight_cap) { // wait for room
          keep.insert(keep.end(), chunk.begin(), chunk.end());
          keep.insert(keep.end(), pend.begin() + (std::ptrdiff_t)i, pend.end());
          break;
        }
        PassBatch pb;
        const cudaStream_t sp = ctx->sp[next_sp++ % PASS_STREAMS];
        if (after_ev) {
          cudaError_t e = cudaStreamWaitEvent(sp, after_ev, 0);
          if (e != cudaSuccess) return e;
        }
        cudaError_t e = enqueue_chunk(ctx, b, kind, chunk, h_hprob, dom, h_hoff, h_hn, &tun, sp, pb);
        if (e != cudaSuccess) return e;
        inflight_bytes += bytes;
        inflight.push_back(std::move(pb));
      }
      pend.swap(keep);
      return cudaSuccess;
    };
    // finish the chunks that are done (all of them when `wait`); finished tunnel loops of problems
    // whose initial pass is done queue their refinement (others wait for it), failed ones a retry
    auto collect = [&](bool wait) -> cudaError_t {
      std::vector<PassBatch> rest;
      for (auto &pb : inflight) {
        if (!wait && cudaEventQuery(pb.ev1) == cudaErrorNotReady) {
          rest.push_back(std::move(pb));
          continue;
        }
        const int kind = pb.kind;
        std::vector<int32_t> ch = pb.chunk;
        cudaError_t e = finish_chunk(ctx, b, pb, kind == PASS_TUNNEL ? tun : ref,
                                     kind == PASS_TUNNEL ? &tunnel_tau : &refine_tau, kind == PASS_TUNNEL ? &ms_t : &ms_r);
        if (e != cudaSuccess) return e;
        inflight_bytes -= chunk_bytes(ch);
        if (kind == PASS_TUNNEL)
          for (int32_t h : ch) {
            if (tun.status[h] == VLS_OK) {
              if (ctx->opt.refine) pend_r.push_back(h);
            } else if (tun.status[h] == VLS_ELOOPFAIL && tun.bstar[h] < 0 && h_hn[h] > 0 && pass_dom[h] != INT32_MAX) {
              retry.push_back(h); // Sec. 3.2: the kept loop separates the covered area: whole surface
            }
          }
      }
      inflight.swap(rest);
      return cudaSuccess;
    };
    std::vector<int32_t> whole(d.hcap, INT32_MAX);
    std::vector<int32_t> pst(b.P, 0);
    // Overlapping the passes with the initial pass was measured slower on the tube chain (464 against
    // 340 ms per detection): many small pass loops running beside the initial pass contend with it
    // for kernel dispatch, while one batched pass loop afterwards costs a single step chain.  It stays
    // available for experiments (VLS_OVERLAP_PASSES=1); the results are the same either way.
    const char *ovl = std::getenv("VLS_OVERLAP_PASSES");
    const bool pipe = !b.host_loop && ctx->opt.tunnels && ovl && ovl[0] == '1';
    if (b.host_loop) {
      const int sync_every = ctx->opt.sync_interval > 0 ? ctx->opt.sync_interval : 16;
      for (int t = 1;; ++t) {
        CK(initial_step_host(b));
        if (t % sync_every == 0 || t >= ctx->opt.max_steps) {
          int32_t act = 0;
          CK(cudaMemcpyAsync(&act, d.ctl + CTL_ACTIVE, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
          b.d2h += (int64_t)sizeof(int32_t);
          CK(cudaStreamSynchronize(st));
          if (act == 0) break;
        }
      }
    } else {
      constexpr int32_t SEG = 256;
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      cudaEvent_t ev_seg = nullptr;
      int32_t *pin = static_cast<int32_t *>(ctx->pinned.take(sizeof(int32_t) * (size_t)(4 + 2 * b.P)));
      if (!pin) { err = cudaErrorMemoryAllocation; goto fail; }
      err = build_initial_graph(b, &g);
      if (err == cudaSuccess) err = cudaGraphInstantiate(&ge, g, 0);
      if (g) cudaGraphDestroy(g);
      if (err == cudaSuccess) err = cudaEventCreateWithFlags(&ev_seg, cudaEventDisableTiming);
      int32_t seg_end = pipe ? SEG : ctx->opt.max_steps;
      while (err == cudaSuccess) {
        pin[0] = std::min(seg_end, ctx->opt.max_steps);
        err = cudaMemcpyAsync(d.ctl + CTL_LIMIT, pin, sizeof(int32_t), cudaMemcpyHostToDevice, st);
        if (err == cudaSuccess) err = cudaGraphLaunch(ge, st);
        if (err != cudaSuccess || !pipe) break;
        // the segment's outcome: step, problems running, handles found, per-problem status and end
        err = cudaMemcpyAsync(pin + 1, d.ctl + CTL_T, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaMemcpyAsync(pin + 2, d.ctl + CTL_ACTIVE, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaMemcpyAsync(pin + 3, d.nhand, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaMemcpyAsync(pin + 4, d.pstatus, sizeof(int32_t) * b.P, cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaMemcpyAsync(pin + 4 + b.P, d.pdone, sizeof(int32_t) * b.P, cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaEventRecord(ev_seg, st);
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
        if (err != cudaSuccess) break;
        b.d2h += (int64_t)sizeof(int32_t) * (3 + 2 * b.P);
        for (int32_t p = 0; p < b.P; ++p) {
          pst[p] = pin[4 + p];
          pdone[p] = pin[4 + b.P + p] && pst[p] == VLS_OK;
        }
        const bool last = pin[2] == 0 || pin[1] > ctx->opt.max_steps;
        if (!last) {
          err = admit(pin[3], pst);
          if (err == cudaSuccess) err = collect(false);
          if (err == cudaSuccess) err = launch(PASS_TUNNEL, pend_t, pass_dom, ev_seg);
          if (err == cudaSuccess) err = launch(PASS_REFINE, pend_r, whole, ev_seg);
        }
        if (last || err != cudaSuccess) break;
        seg_end += SEG;
      }
      if (ge) cudaGraphExecDestroy(ge);
      if (ev_seg) cudaEventDestroy(ev_seg);
      if (err != cudaSuccess) goto fail;
    }
    CK(final_checks(b));
    CK(cudaEventRecord(ev[2], st));
    // ---- the rest of the passes, once the initial pass has ended
    CK(cudaMemcpyAsync(&h_nh, d.nhand, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&h_nn, d.nnodes, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    h_status.resize(b.P);
    CK(cudaMemcpyAsync(h_status.data(), d.pstatus, sizeof(int32_t) * b.P, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    b.d2h += (int64_t)sizeof(int32_t) * (2 + b.P);
    h_nh = std::min(h_nh, d.hcap);
    h_nn = std::min(h_nn, d.ncap);
    for (int32_t p = 0; p < b.P; ++p) pdone[p] = h_status[p] == VLS_OK;
    CK(admit(h_nh, h_status));
    CK(cudaEventRecord(ev[5], st));
    while (!pend_t.empty() || !pend_r.empty() || !retry.empty() || !inflight.empty()) {
      for (int32_t h : retry) {
        pass_dom[h] = INT32_MAX;
        pend_t.push_back(h);
      }
      retry.clear();
      CK(launch(PASS_TUNNEL, pend_t, pass_dom, ev[5]));
      CK(launch(PASS_REFINE, pend_r, whole, ev[5]));
      CK(collect(true));
    }
    for (int32_t sp = 0; sp < PASS_STREAMS; ++sp) CK(cudaStreamSynchronize(ctx->sp[sp]));
    // passes of a problem whose initial pass failed (started before it failed) do not count
    for (int32_t h : pass_h)
      if (h_status[h_hprob[h]] != VLS_OK) {
        tun.status[h] = ref.status[h] = -1;
        tun.steps[h] = ref.steps[h] = 0;
        tun.bstar[h] = ref.bstar[h] = 0;
        tun.vn[h] = ref.vn[h] = 0;
        tun.dl[h] = ref.dl[h] = std::nan("");
      }
    // tables of every handle, classification of the handle (isoline) loops (Sec. 3.5)
    h_hprob.resize(h_nh);
    h_hstep.resize(h_nh);
    h_hoff.resize(h_nh);
    h_hn.resize(h_nh);
    if (!d2h(h_hlayer, d.hlayer, h_nh, st) || !d2h(h_hnode, d.hnode, h_nh, st) || !d2h(h_hvoff, d.hvoff, h_nh, st) ||
        !d2h(h_hvn, d.hvn, h_nh, st) || !d2h(h_hlen, d.hlen, h_nh, st)) {
      err = cudaErrorUnknown;
      goto fail;
    }
    CK(launch_classify_handles(b, d.vn, d.pmedge, d.hdl, h_nh));
    if (!d2h(h_hdl, d.hdl, h_nh, st)) {
      err = cudaErrorUnknown;
      goto fail;
    }
    CK(cudaStreamSynchronize(st));
    for (int32_t h : pass_h) {
      if (h_status[h_hprob[h]] != VLS_OK) continue;
      ProbResult &r = res->p[dev_probs[h_hprob[h]]];
      r.stats.pass_updates += tun.upd[h];
      r.stats.pass_uncertified += tun.unc[h];
      r.stats.pass_mass_resid = std::max(r.stats.pass_mass_resid, tun.mres[h]);
      r.tunnel_steps = std::max(r.tunnel_steps, tun.steps[h]);
      if (ref.status[h] != -1) {
        r.stats.refine_updates += ref.upd[h];
        r.stats.refine_uncertified += ref.unc[h];
        r.stats.refine_mass_resid = std::max(r.stats.refine_mass_resid, ref.mres[h]);
        r.stats.refine_steps = std::max(r.stats.refine_steps, ref.steps[h]);
      }
    }
    CK(cudaEventRecord(ev[3], st));
    // ---- download
    std::vector<int32_t> nkind, nstep, nprob, nlocal, lstate, lbirth, ldeath, lcount, psteps, pev, hedge, hverts;
    std::vector<double> npos, hpts;
    std::vector<int64_t> pupd;
    std::vector<unsigned long long> punc;
    std::vector<double> pmres;
    int32_t ne = 0;
    CK(cudaMemcpyAsync(&ne, d.nhedge, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    b.d2h += (int64_t)sizeof(int32_t);
    ne = std::min(ne, d.ecap);
    if (!d2h(nkind, d.nkind, h_nn, st) || !d2h(nstep, d.nstep, h_nn, st) || !d2h(nprob, d.nprob, h_nn, st) ||
        !d2h(nlocal, d.nlocal, h_nn, st) || !d2h(npos, d.npos, 3 * (size_t)h_nn, st) ||
        !d2h(lcount, d.lcount, b.P, st) || !d2h(psteps, d.psteps, b.P, st) || !d2h(pev, d.pev, 3 * (size_t)b.P, st) ||
        !d2h(pupd, reinterpret_cast<const int64_t *>(d.pupd), b.P, st) || !d2h(pmres, d.pmres, b.P, st) ||
        !d2h(punc, d.punc, b.P, st) || !d2h(hedge, d.hedge, 2 * (size_t)ne, st) ||
        !d2h(hverts, d.hverts, ne, st) || !d2h(hpts, d.hpts, 3 * (size_t)ne, st) ||
        !d2h(lstate, d.lstate, b.Lcap, st) || !d2h(lbirth, d.lbirth, b.Lcap, st) || !d2h(ldeath, d.ldeath, b.Lcap, st)) {
      err = cudaErrorUnknown;
      goto fail;
    }
    std::vector<int32_t> lay_all, cover_all;
    std::vector<double> phi_all;
    std::vector<long long> rec_all;
    if (ctx->opt.keep_state) {
      if (!d2h(lay_all, d.lay, b.V, st) || !d2h(cover_all, d.cover, b.V, st)) {
        err = cudaErrorUnknown;
        goto fail;
      }
      if (d.phih) {
        std::vector<uint16_t> phih_all;
        if (!d2h(phih_all, reinterpret_cast<const uint16_t *>(d.phih), b.V, st)) {
          err = cudaErrorUnknown;
          goto fail;
        }
        CK(cudaStreamSynchronize(st));
        phi_all.resize(phih_all.size());
        for (size_t k = 0; k < phih_all.size(); ++k) { // a bfloat16 is the high half of a float
          const uint32_t bits = (uint32_t)phih_all[k] << 16;
          float f;
          memcpy(&f, &bits, sizeof f);
          phi_all[k] = f;
        }
      } else if (d.phif) {
        std::vector<float> phif_all;
        if (!d2h(phif_all, d.phif, b.V, st)) {
          err = cudaErrorUnknown;
          goto fail;
        }
        CK(cudaStreamSynchronize(st));
        phi_all.assign(phif_all.begin(), phif_all.end());
      } else if (!d2h(phi_all, d.phi, b.V, st)) {
        err = cudaErrorUnknown;
        goto fail;
      }
    }
    if (d.record) {
      if (!d2h(rec_all, d.rec, (size_t)b.P * d.rcap * 5, st)) { err = cudaErrorUnknown; goto fail; }
    }
    int32_t h_ctl[CTL_SIZE] = {};
    CK(cudaMemcpyAsync(h_ctl, d.ctl, sizeof(h_ctl), cudaMemcpyDeviceToHost, st));
    b.d2h += (int64_t)sizeof(h_ctl);
    unsigned long long h_rechk[2] = {0ull, 0ull};
    CK(cudaMemcpyAsync(h_rechk, d.nrecheck, sizeof(h_rechk), cudaMemcpyDeviceToHost, st));
    b.d2h += (int64_t)sizeof(h_rechk) + (int64_t)sizeof(double) * b.P;
    CK(cudaEventRecord(ev[4], st));
    CK(cudaStreamSynchronize(st));
    if (!b.host_loop) {
      // kernels run inside the graphs: 5 per initial step, 4 per merge phase, 1 per split
      // phase, 3 per tunnel step
      const int64_t steps = h_ctl[CTL_T] - 1;
      b.launches += 5 * steps;
      b.launches += 4 * (int64_t)h_ctl[CTL_NMERGE] + (int64_t)h_ctl[CTL_NSPLIT];
      if (tunnel_tau > 0) b.launches += 3 * (int64_t)tunnel_tau;
      if (refine_tau > 0) b.launches += 3 * (int64_t)refine_tau;
    }
#ifdef VLS_CHECKED
    {
      int32_t e4[4] = {0, 0, 0, 0};
      cudaMemcpy(e4, d.err, sizeof(e4), cudaMemcpyDeviceToHost);
      if (e4[2] != 0) {
        fprintf(stderr, "vls checked build: index check failed at site %d (index %d)\n", e4[2], e4[3]);
        for (auto &r : res->p) r.status = VLS_ECUDA;
      }
    }
#endif
    // ---- repack per problem
    // pass times: device time of the pass chunks (they overlap the initial pass and one another)
    const float ms_op = elapsed(ev[0], ev[1]), ms_init = elapsed(ev[1], ev[2]), ms_tun = (float)ms_t,
                ms_ref = (float)ms_r, ms_dl = elapsed(ev[3], ev[4]);
    std::vector<double> pmedge;
    if (!d2h(pmedge, d.pmedge, b.P, st) || cudaStreamSynchronize(st) != cudaSuccess) {
      err = cudaErrorUnknown;
      goto fail;
    }
    double ms_k[KK_COUNT_KINDS] = {};
    int64_t n_k[KK_COUNT_KINDS] = {};
    for (const auto &mk : b.prof.marks) {
      ms_k[mk.first] += elapsed((*b.prof.pool)[mk.second], (*b.prof.pool)[mk.second + 1]);
      n_k[mk.first]++;
    }
    res->klaunch.assign(n_k, n_k + KK_COUNT_KINDS);
    res->kms.assign(ms_k, ms_k + KK_COUNT_KINDS);
    for (int32_t q = 0; q < b.P; ++q) {
      ProbResult &r = res->p[dev_probs[q]];
      r.status = h_status[q];
      r.steps = psteps[q];
      r.stats.steps = psteps[q];
      r.stats.tunnel_steps = r.tunnel_steps;
      r.stats.row_updates = pupd[q];
      r.stats.merges = pev[3 * q];
      r.stats.splits = pev[3 * q + 1];
      r.stats.ends = pev[3 * q + 2];
      r.stats.layers = lcount[q];
      r.stats.ms_operator = ms_op;
      r.stats.ms_initial = ms_init;
      r.stats.ms_tunnel = ms_tun;
      r.stats.ms_refine = ms_ref;
      r.stats.mean_edge = pmedge[q];
      r.stats.ms_download = ms_dl;
      r.stats.kernel_launches = b.launches;
      r.stats.ms_update = ms_k[KK_UPDATE];
      r.stats.ms_pass_update = ms_k[KK_TUPDATE];
      r.stats.n_update = n_k[KK_UPDATE];
      r.stats.n_pass_update = n_k[KK_TUPDATE];
      r.stats.h2d_bytes = b.h2d;
      r.stats.d2h_bytes = b.d2h;
      r.stats.rechecks = (int64_t)h_rechk[0];
      r.stats.pass_rechecks = (int64_t)h_rechk[1];
      r.stats.mass_resid = pmres[q];
      r.stats.uncertified = (int64_t)punc[q];
      const int32_t nl = lcount[q];
      r.layers.resize(3 * (size_t)nl);
      for (int32_t l = 1; l <= nl; ++l) {
        const int32_t g = b.lbase[q] + l;
        r.layers[3 * (l - 1)] = lbirth[g];
        r.layers[3 * (l - 1) + 1] = ldeath[g];
        r.layers[3 * (l - 1) + 2] = lstate[g];
      }
      if (ctx->opt.keep_state) {
        const int32_t v0 = b.voff[q], n = b.voff[q + 1] - v0;
        r.lay.resize(n);
        r.phi.assign(phi_all.begin() + v0, phi_all.begin() + v0 + n);
        r.cover.assign(cover_all.begin() + v0, cover_all.begin() + v0 + n);
        for (int32_t i = 0; i < n; ++i) r.lay[i] = lay_all[v0 + i] ? lay_all[v0 + i] - b.lbase[q] : 0;
      }
      if (d.record) {
        const int32_t n = std::min(psteps[q], d.rcap);
        r.rec.resize(5 * (size_t)n);
        for (int32_t i = 0; i < 5 * n; ++i) r.rec[i] = rec_all[(size_t)q * d.rcap * 5 + i];
      }
    }
    // nodes in local order
    for (int32_t q = 0; q < b.P; ++q) {
      int32_t cnt = 0;
      for (int32_t g = 0; g < h_nn; ++g) cnt += nprob[g] == q;
      ProbResult &r = res->p[dev_probs[q]];
      r.nodes.assign(2 * (size_t)cnt, 0);
      r.npos.assign(3 * (size_t)cnt, 0.0);
    }
    for (int32_t g = 0; g < h_nn; ++g) {
      ProbResult &r = res->p[dev_probs[nprob[g]]];
      const int32_t loc = nlocal[g];
      if (loc < 0 || 2 * (size_t)loc >= r.nodes.size()) continue;
      r.nodes[2 * loc] = nkind[g];
      r.nodes[2 * loc + 1] = nstep[g];
      for (int c = 0; c < 3; ++c) r.npos[3 * loc + c] = npos[3 * (size_t)g + c];
    }
    // handles and tunnels, emission order per problem
    for (int32_t h = 0; h < h_nh; ++h) {
      const int32_t q = h_hprob[h];
      ProbResult &r = res->p[dev_probs[q]];
      const int32_t v0 = b.voff[q];
      ProbResult::Handle H;
      const int32_t o = h_hoff[h], n = h_hn[h];
      H.edges.resize(2 * (size_t)n);
      H.pts.resize(3 * (size_t)n);
      for (int32_t i = 0; i < n; ++i) {
        H.edges[2 * i] = hedge[2 * (size_t)(o + i)] - v0;
        H.edges[2 * i + 1] = hedge[2 * (size_t)(o + i) + 1] - v0;
        for (int c = 0; c < 3; ++c) H.pts[3 * i + c] = hpts[3 * (size_t)(o + i) + c];
      }
      H.verts.resize(h_hvn[h]);
      for (int32_t i = 0; i < h_hvn[h]; ++i) H.verts[i] = hverts[h_hvoff[h] + i] - v0;
      H.info[0] = h_hstep[h];
      H.info[1] = h_hlayer[h];
      H.info[2] = h_hnode[h];
      H.len = h_hlen[h];
      r.handles.push_back(std::move(H));
      for (int kind = 0; kind < 2; ++kind) {
        const PassOut &o = kind == 0 ? tun : ref;
        ProbResult::Tunnel T;
        T.info[0] = o.status[h];
        T.info[1] = o.steps[h];
        T.info[2] = o.bstar[h];
        if (o.status[h] == VLS_OK) T.verts.assign(o.verts.begin() + o.voff[h], o.verts.begin() + o.voff[h] + o.vn[h]);
        if (o.status[h] == VLS_OK && o.sst[h] >= 0) {
          T.sst = o.sst[h];
          T.slen = o.slen[h];
          T.spts.assign(o.spts.begin() + 3 * o.soff[h], o.spts.begin() + 3 * (o.soff[h] + o.sn[h]));
        }
        (kind == 0 ? r.tunnels : r.refined).push_back(std::move(T));
      }
      r.dlen.push_back({h_hdl[h], tun.dl[h], ref.dl[h]});
    }
    for (int32_t q = 0; q < b.P; ++q) {
      ProbResult &r = res->p[dev_probs[q]];
      if (r.status == VLS_OK)
        for (auto &T : r.tunnels)
          if (T.info[0] > 0) { r.status = T.info[0]; break; } // -1: the pass did not run
      if (r.status == VLS_OK)
        for (auto &T : r.refined)
          if (T.info[0] > 0) { r.status = T.info[0]; break; }
    }
  }
  for (int i = 0; i < 6; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  g_d2h_counter = nullptr;
  *out = res;
  return VLS_OK;
fail:
  g_d2h_counter = nullptr;
  for (int i = 0; i < 6; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  cudaGetLastError();
  for (auto &r : res->p)
    if (r.status == VLS_OK) r.status = (err == cudaErrorMemoryAllocation) ? VLS_ENOMEM : VLS_ECUDA;
  *out = res;
  return err == cudaErrorMemoryAllocation ? VLS_ENOMEM : VLS_ECUDA;
}

extern "C" vls_status vls_detect(vls_ctx *ctx, const vls_mesh *m, int32_t seed_vertex, vls_result **out) {
  if (!m) return VLS_EINVAL;
  const int32_t one = 1;
  return vls_detect_batch(ctx, 1, m, &seed_vertex, &one, out);
}

extern "C" int32_t vls_result_count(const vls_result *r) { return r ? (int32_t)r->p.size() : 0; }

#define GETP(r, p)                                                  \
  if (!(r) || (p) < 0 || (p) >= (int32_t)(r)->p.size()) return VLS_EINVAL; \
  const ProbResult &P_ = (r)->p[p];

extern "C" vls_status vls_result_status(const vls_result *r, int32_t p) {
  GETP(r, p);
  return (vls_status)P_.status;
}
extern "C" int32_t vls_result_genus(const vls_result *r, int32_t p) {
  if (!r || p < 0 || p >= (int32_t)r->p.size()) return -1;
  return r->p[p].genus;
}
extern "C" vls_status vls_result_stats(const vls_result *r, int32_t p, vls_stats *s) {
  GETP(r, p);
  if (!s) return VLS_EINVAL;
  *s = P_.stats;
  return VLS_OK;
}
extern "C" int32_t vls_result_num_loops(const vls_result *r, int32_t p, int32_t kind) {
  if (!r || p < 0 || p >= (int32_t)r->p.size()) return -1;
  return kind == 0   ? (int32_t)r->p[p].handles.size()
         : kind == 1 ? (int32_t)r->p[p].tunnels.size()
         : kind == 2 ? (int32_t)r->p[p].refined.size()
                     : -1;
}
extern "C" vls_status vls_result_loop(const vls_result *r, int32_t p, int32_t kind, int32_t i, const int32_t **verts,
                                      int64_t *n, const double **pts, int64_t *npts) {
  GETP(r, p);
  if (kind == 0) {
    if (i < 0 || i >= (int32_t)P_.handles.size()) return VLS_EINVAL;
    const auto &H = P_.handles[i];
    if (verts) *verts = H.verts.data();
    if (n) *n = (int64_t)H.verts.size();
    if (pts) *pts = H.pts.data();
    if (npts) *npts = (int64_t)H.pts.size() / 3;
    return VLS_OK;
  }
  if (kind != 1 && kind != 2) return VLS_EINVAL;
  const auto &L = kind == 1 ? P_.tunnels : P_.refined;
  if (i < 0 || i >= (int32_t)L.size()) return VLS_EINVAL;
  const auto &T = L[i];
  if (verts) *verts = T.verts.data();
  if (n) *n = (int64_t)T.verts.size();
  if (pts) *pts = nullptr;
  if (npts) *npts = 0;
  return VLS_OK;
}
extern "C" vls_status vls_result_handle(const vls_result *r, int32_t p, int32_t i, const int32_t **edges, int64_t *n,
                                        int32_t info[3], double *length) {
  GETP(r, p);
  if (i < 0 || i >= (int32_t)P_.handles.size()) return VLS_EINVAL;
  const auto &H = P_.handles[i];
  if (edges) *edges = H.edges.data();
  if (n) *n = (int64_t)H.edges.size() / 2;
  if (info) std::memcpy(info, H.info, sizeof(H.info));
  if (length) *length = H.len;
  return VLS_OK;
}
extern "C" vls_status vls_result_tunnel(const vls_result *r, int32_t p, int32_t i, int32_t info[3]) {
  GETP(r, p);
  if (i < 0 || i >= (int32_t)P_.tunnels.size() || !info) return VLS_EINVAL;
  std::memcpy(info, P_.tunnels[i].info, sizeof(int32_t) * 3);
  return VLS_OK;
}
extern "C" vls_status vls_result_refined(const vls_result *r, int32_t p, int32_t i, int32_t info[3]) {
  GETP(r, p);
  if (i < 0 || i >= (int32_t)P_.refined.size() || !info) return VLS_EINVAL;
  std::memcpy(info, P_.refined[i].info, sizeof(int32_t) * 3);
  return VLS_OK;
}
extern "C" vls_status vls_result_streamline(const vls_result *r, int32_t p, int32_t i, int32_t kind, int32_t *status,
                                            const double **pts, int64_t *n, double *length) {
  GETP(r, p);
  if (kind != 0 && kind != 1) return VLS_EINVAL;
  const auto &v = kind == 0 ? P_.tunnels : P_.refined;
  if (i < 0 || i >= (int32_t)v.size() || !status || !pts || !n || !length) return VLS_EINVAL;
  *status = v[i].sst;
  *pts = v[i].spts.data();
  *n = (int64_t)(v[i].spts.size() / 3);
  *length = v[i].slen;
  return VLS_OK;
}
extern "C" vls_status vls_result_offset_change(const vls_result *r, int32_t p, int32_t i, double out[3]) {
  GETP(r, p);
  if (i < 0 || i >= (int32_t)P_.dlen.size() || !out) return VLS_EINVAL;
  for (int k = 0; k < 3; ++k) out[k] = P_.dlen[i][k];
  return VLS_OK;
}
extern "C" vls_status vls_result_reeb(const vls_result *r, int32_t p, const int32_t **nodes, const double **pos,
                                      int32_t *n_nodes, const int32_t **layers, int32_t *n_layers) {
  GETP(r, p);
  if (nodes) *nodes = P_.nodes.data();
  if (pos) *pos = P_.npos.data();
  if (n_nodes) *n_nodes = (int32_t)(P_.nodes.size() / 2);
  if (layers) *layers = P_.layers.data();
  if (n_layers) *n_layers = (int32_t)(P_.layers.size() / 3);
  return VLS_OK;
}
extern "C" vls_status vls_result_state(const vls_result *r, int32_t p, const int32_t **layer, const double **phi,
                                       const int32_t **cover, int64_t *nv) {
  GETP(r, p);
  if (P_.lay.empty()) return VLS_EINVAL;
  if (layer) *layer = P_.lay.data();
  if (phi) *phi = P_.phi.data();
  if (cover) *cover = P_.cover.data();
  if (nv) *nv = (int64_t)P_.lay.size();
  return VLS_OK;
}
extern "C" vls_status vls_result_records(const vls_result *r, int32_t p, const int64_t **rec, int32_t *steps) {
  GETP(r, p);
  if (rec) *rec = P_.rec.data();
  if (steps) *steps = (int32_t)(P_.rec.size() / 5);
  return VLS_OK;
}
extern "C" vls_status vls_result_kernel_times(const vls_result *r, const char *const **names, const int64_t **launches,
                                              const double **ms, int32_t *n) {
  if (!r) return VLS_EINVAL;
  if (names) *names = kKernelNames;
  if (launches) *launches = r->klaunch.empty() ? nullptr : r->klaunch.data();
  if (ms) *ms = r->kms.empty() ? nullptr : r->kms.data();
  if (n) *n = r->klaunch.empty() ? 0 : (int32_t)KK_COUNT_KINDS;
  return VLS_OK;
}

extern "C" void vls_result_free(vls_result *r) { delete r; }
