// vls_batch.cuh -- host-side batch object shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "vls_internal.cuh"

namespace vls {

// Grow-only device arena owned by a context: one cudaMalloc reused by every call.
struct Arena {
  char *base = nullptr;
  size_t cap = 0, used = 0;
  cudaError_t reserve(size_t bytes);
  void reset() { used = 0; }
  template <class T> T *take(size_t n) {
    size_t off = (used + 255) & ~size_t(255);
    size_t bytes = n * sizeof(T);
    if (off + bytes > cap) return nullptr;
    used = off + bytes;
    return reinterpret_cast<T *>(base + off);
  }
};

// Tunnel-pass device state (Sec. 3.2 / Sec. 4: one dense single-layer field per pass).
struct TDev {
  int32_t NP;          // passes in this chunk
  int32_t PV;          // pass-vertex entries
  int32_t *err;        // the batch's error word
  const int32_t *pbase;  // [NP+1] pass-vertex offsets (pass q, local vertex v -> pbase[q] + v)
  const int32_t *pprob;  // [NP] problem of the pass
  const int32_t *pstep;  // [NP] step of its handle (domain: cover <= step)
  const int32_t *pcoff, *pcn;  // [NP] cut half-edge slots (sorted) offset / count
  const int32_t *cut;          // global CSR slots of the loop's half-edges, both directions
  const int32_t *heoff, *hen;  // [NP] the pass's border edges (inside, outside) in the pool xedge
  const int32_t *xedge;        // [..][2] border-edge pool (global vertex ids): the handle loops' crossing
                               // edges (tunnel passes) or the tunnel loops' right-side edges (refinement)
  double *qdl;                 // [NP] length change of the pass's loop under the normal offset (Sec. 3.5)
  int8_t *flag;        // [pass-vertex] bit0 source, bit1 target
  double *phi;         // [pass-vertex] FP64 form
  float *phif;         // [pass-vertex] FP32 form (non-null selects it; phi unused)
  __nv_bfloat16 *phih; // [pass-vertex] BF16 form (non-null selects it; phi, phif unused)
  int32_t *T;          // [pass-vertex] arrival step (-1 unreached)
  int32_t *stamp;      // [pass-vertex]
  int32_t *fv[2], *fq[2];  // frontier (vertex, pass)
  int32_t *nf;         // [2]
  double *onew;        // [V] per frontier row
  int32_t *qdone, *qsteps, *qstatus, *qbstar;  // [NP]
  int32_t *qcnt;       // [NP] rows in the frontier being built
  double *qmass;       // [NP][qslots][2] mass-check sums of the step (see mass_sums)
  int32_t qslots;
  double *qmres;       // [NP] largest mass-check residual of the pass
  unsigned long long *qunc; // [NP] uncertified decisions of the pass (see Params::drift)
  long long *qupd;     // [NP]
  int32_t *active;
  int32_t *ctl;        // [CTL_SIZE] the passes' own control block (step, passes running, step bound):
                       // chunks of passes in flight on different streams run independently
  // output: tunnel vertex cycles
  int32_t *tvoff, *tvn;  // [NP]
  int32_t *tverts;       // pool
  int32_t *ntverts;
  int32_t tvcap;
  int32_t *path;         // scratch [pass-vertex] for traces
  // PL streamlines (Sec. 3.2), when on (tfa non-null)
  double *tfa;           // [pass-vertex] arrival time with the step's fraction (read where T >= 0)
  const int32_t *sroff;  // [NP+1] the passes' regions in sreg (a pass's point budget each)
  double *sreg;          // [scap][3] the regions the traces write
  int32_t *sst, *sn, *soff; // [NP] status (-1 not traced), points, offset in the compact pool
  double *slen;          // [NP] length of the closed polyline
  double *spts;          // [scap][3] compact pool (what is downloaded)
  int32_t *nspts;        // points in the compact pool
  int64_t scap;
};

// Kernel kinds timed in profile mode.
enum KernelKind : int {
  KK_UPDATE = 0, KK_TUPDATE, KK_APPLY, KK_HOOK, KK_COUNT, KK_FRONTIER, KK_MERGE_GROUPS,
  KK_TRACE, KK_MERGE_FINISH, KK_RELABEL, KK_SPLIT, KK_TAPPLY, KK_TFRONTIER, KK_COUNT_KINDS
};
static const char *const kKernelNames[KK_COUNT_KINDS] = {
    "k_update", "k_tupdate", "k_apply", "k_band_hook", "k_band_count", "k_frontier",
    "k_merge_groups", "k_trace", "k_merge_finish", "k_relabel", "k_split", "k_tapply", "k_tfrontier"};

// Optional CUDA-event timing of selected launches (pairs drawn from a context-owned pool).
struct Prof {
  std::vector<cudaEvent_t> *pool = nullptr; // owned by the context, grows on demand
  size_t used = 0;
  std::vector<std::pair<int, size_t>> marks; // (kind, index of the start event)
  bool on = false;
  cudaEvent_t get() {
    if (used == pool->size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      pool->push_back(e);
    }
    return (*pool)[used++];
  }
  // record a start event for a launch of `kind`; returns the slot to close with end()
  long begin(cudaStream_t st, int kind) {
    if (!on) return -1;
    cudaEvent_t a = get(), b = get();
    if (!a || !b) return -1;
    cudaEventRecord(a, st);
    marks.push_back({kind, used - 2});
    return (long)(used - 1);
  }
  void end(cudaStream_t st, long slot) {
    if (slot >= 0) cudaEventRecord((*pool)[slot], st);
  }
};

struct Batch {
  Prof prof;
  bool host_loop = false; // debug / profiling: launch each step from the host
  int64_t h2d = 0, d2h = 0;
  cudaStream_t st = nullptr;
  vls_options opt;
  Params prm;
  Dev d;
  TDev td;
  int32_t P = 0, V = 0, NF = 0, Lcap = 0;
  int64_t nnz = 0;
  int sm_count = 148;
  // per-kernel launch shape: grid (SM count x blocks per SM) and threads per block
  struct Cfg {
    int grid = 0, threads = 0;
  } cfg[KK_COUNT_KINDS];
  // requested launch shape per kernel kind: threads per block, blocks per SM (0 = as many as
  // fit); set from the options or by the autotuner before configure_*()
  struct Shape {
    int threads = 0, bps = 0;
  } shape[KK_COUNT_KINDS];
  int hook_variant = 2; // band union-find: 1 one thread per band row, 2 a lane group per row
  long long launches = 0;
  Arena *arena = nullptr;
  // refinement chunks (Sec. 3.3): the tunnel cycles they start from, per pass offset / length, and
  // the capacity of each pass's border-edge list
  int32_t *r_cyc = nullptr, *r_coff = nullptr, *r_clen = nullptr, *r_xcap = nullptr;
  // host copies of problem tables
  std::vector<int32_t> voff, foff, lbase, lcap, seed, mesh_of;
  std::vector<int64_t> nv_local, nf_local;
};

#define VLS_LAUNCH(b) ((b).launches++)

// ---------------------------------------------------------------- graph helpers
template <class T> struct ident { using type = T; };

// Add a kernel node f<<<grid, block>>>(args...) to graph g after deps.
template <class... K>
inline cudaError_t add_kernel(cudaGraphNode_t *node, cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps,
                              void (*f)(K...), dim3 grid, dim3 block, typename ident<K>::type... args) {
  void *params[] = {(void *)&args..., nullptr};
  cudaKernelNodeParams p = {};
  p.func = (void *)f;
  p.gridDim = grid;
  p.blockDim = block;
  p.sharedMemBytes = 0;
  p.kernelParams = params;
  return cudaGraphAddKernelNode(node, g, deps, ndeps, &p);
}

// Add a conditional node (IF / WHILE) to g after deps; its handle is created on g with the
// given default (assigned at every launch of the graph).  *body receives the body graph.
// A programmatic edge from kernel node `from` to kernel node `to` (the kernels call pdl_enter
// first): `to` may be scheduled while `from` finishes.  Where the driver refuses the edge, an
// ordinary one.
inline cudaError_t add_programmatic_edge(cudaGraph_t g, cudaGraphNode_t from, cudaGraphNode_t to) {
  cudaGraphEdgeData ed = {};
  ed.from_port = cudaGraphKernelNodePortProgrammatic;
  ed.type = cudaGraphDependencyTypeProgrammatic;
  cudaError_t e = cudaGraphAddDependencies(g, &from, &to, &ed, 1);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    e = cudaGraphAddDependencies(g, &from, &to, nullptr, 1);
  }
  return e;
}

inline cudaError_t add_conditional(cudaGraphNode_t *node, cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps,
                                   cudaGraphConditionalNodeType type, unsigned dflt,
                                   cudaGraphConditionalHandle *h, cudaGraph_t *body) {
  cudaError_t e = cudaGraphConditionalHandleCreate(h, g, dflt, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = *h;
  np.conditional.type = type;
  np.conditional.size = 1;
  e = cudaGraphAddNode(node, g, deps, nullptr, ndeps, &np);
  if (e != cudaSuccess) return e;
  *body = np.conditional.phGraph_out[0];
  return cudaSuccess;
}

// launch shapes (one resident wave per kernel), per translation unit
void configure_initial(Batch &b);
void configure_events(Batch &b);
void configure_tunnel(Batch &b);
template <class K> inline Batch::Cfg wave_cfg(const Batch &b, K kernel, int threads) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, 0) != cudaSuccess || nb < 1) nb = 1;
  Batch::Cfg c;
  c.grid = b.sm_count * nb;
  c.threads = threads;
  return c;
}
// Launch shape of row kernel `kind`: b.shape[kind] (threads, blocks per SM) clamped to what fits
// on an SM; dflt_threads when no shape was requested.
template <class K> inline Batch::Cfg row_cfg(const Batch &b, K kernel, int kind, int dflt_threads) {
  const int threads = b.shape[kind].threads > 0 ? b.shape[kind].threads : dflt_threads;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, 0) != cudaSuccess || nb < 1) nb = 1;
  const int bps = b.shape[kind].bps > 0 && b.shape[kind].bps < nb ? b.shape[kind].bps : nb;
  Batch::Cfg c;
  c.grid = b.sm_count * bps;
  c.threads = threads;
  return c;
}
// operator.cu
cudaError_t build_operator(Batch &b, int32_t *d_status_stage);
// initial.cu: the initial pass as one graph (WHILE over steps) or, for debugging, a host loop
cudaError_t init_state(Batch &b);
cudaError_t build_initial_graph(Batch &b, cudaGraph_t *graph);
cudaError_t initial_step_host(Batch &b);
cudaError_t final_checks(Batch &b);
// events.cu: bodies of the IF nodes (and their host-loop launches)
cudaError_t add_merge_nodes(Batch &b, cudaGraph_t body, const cudaGraphNode_t *dep);
cudaError_t add_split_nodes(Batch &b, cudaGraph_t body);
cudaError_t merge_phase_host(Batch &b);
cudaError_t split_phase_host(Batch &b);
// tunnel.cu
cudaError_t run_tunnels(Batch &b, const TDev &T, cudaStream_t st, int32_t *tau_dst, cudaGraphExec_t *ge_out);
// refine.cu: vertex normals and mean edge lengths, loop classification, refinement set-up
cudaError_t launch_vnormals(Batch &b, double *vn, double *elen, double *pmedge);
cudaError_t launch_classify_handles(Batch &b, const double *vn, const double *pmedge, double *hdl, int32_t nh);
cudaError_t launch_classify_passes(Batch &b, const TDev &T, cudaStream_t st, const double *vn, const double *pmedge);
cudaError_t launch_refine_prep(Batch &b, const TDev &T, cudaStream_t st, int32_t *cyc_pool, const int32_t *coff,
                               const int32_t *clen, int32_t *xedge, const int32_t *xcap, int32_t *hen, int32_t *pcn);

}  // namespace vls
