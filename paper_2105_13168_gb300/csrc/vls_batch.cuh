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
  const int32_t *heoff, *hen;  // [NP] the handle's crossing edges in the global pool
  int8_t *flag;        // [pass-vertex] bit0 source, bit1 target
  double *phi;         // [pass-vertex]
  int32_t *T;          // [pass-vertex] arrival step (-1 unreached)
  int32_t *stamp;      // [pass-vertex]
  int32_t *fv[2], *fq[2];  // frontier (vertex, pass)
  int32_t *nf;         // [2]
  double *onew;        // [V] per frontier row
  int32_t *qdone, *qsteps, *qstatus, *qbstar;  // [NP]
  int32_t *qcnt;       // [NP] rows in the frontier being built
  long long *qupd;     // [NP]
  int32_t *active;
  // output: tunnel vertex cycles
  int32_t *tvoff, *tvn;  // [NP]
  int32_t *tverts;       // pool
  int32_t *ntverts;
  int32_t tvcap;
  int32_t *path;         // scratch [pass-vertex] for traces
};

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
  int64_t h2d = 0, d2h = 0;
  cudaStream_t st = nullptr;
  vls_options opt;
  Params prm;
  Dev d;
  TDev td;
  int32_t P = 0, V = 0, NF = 0, Lcap = 0;
  int64_t nnz = 0;
  int sm_count = 148;
  int grid = 0, threads = 256;
  long long launches = 0;
  Arena *arena = nullptr;
  // host copies of problem tables
  std::vector<int32_t> voff, foff, lbase, lcap, seed, mesh_of;
  std::vector<int64_t> nv_local, nf_local;
};

#define VLS_LAUNCH(b) ((b).launches++)

// operator.cu
cudaError_t build_operator(Batch &b, int32_t *d_status_stage);
// initial.cu
cudaError_t init_state(Batch &b);
cudaError_t initial_step(Batch &b, int t);
cudaError_t final_checks(Batch &b);
// events.cu
cudaError_t merge_phase(Batch &b, int t, int cur);
cudaError_t split_phase(Batch &b, int t, int cur);
// tunnel.cu
cudaError_t run_tunnels(Batch &b, int32_t *h_steps_out);

}  // namespace vls
