/*
 * vls.h -- C ABI of the GB300 variational loop-shrinking library.
 *
 * Implements the hot path of Weinrauch, Seidel, Mlakar, Steinberger, Zayer,
 * "A Variational Loop Shrinking Analogy for Handle and Tunnel Detection and Reeb
 * Graph Construction on Surfaces": a closed triangle mesh and a seed vertex go in;
 * handle loops, tunnel loops and the diffusion Reeb graph come out (problem
 * statement, Sec. 1; initial pass Sec. 3.1; tunnel pass Sec. 3.2; single-layer
 * passes Sec. 4; Reeb graph Sec. 5).  Every step runs in CUDA kernels on the
 * current device.
 *
 * Conventions
 *   - Every function returns vls_status (0 = VLS_OK) unless stated otherwise; no C++
 *     exception crosses this boundary.
 *   - Input arrays are borrowed: read during the call only, never retained.
 *   - Results live in library-owned host memory until vls_result_free(); every pointer
 *     a result accessor hands out stays valid until then.
 *   - A context is not thread-safe: use one per host thread.
 *   - Layer ids in results are per problem: 1 is the seed layer, then ids follow
 *     creation order.  Vertex ids are those of the input mesh.
 */
#ifndef VLS_H
#define VLS_H
#include <stdint.h>

#if defined(__GNUC__)
#define VLS_API __attribute__((visibility("default")))
#else
#define VLS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VLS_OK = 0,
  VLS_EINVAL = 1,          /* bad argument, index out of range, degenerate face, bad seed */
  VLS_ENOTMANIFOLD = 2,    /* open or non-manifold edge / vertex */
  VLS_ENONORIENTABLE = 3,  /* inconsistently oriented faces */
  VLS_EDISCONNECTED = 4,   /* more than one connected component, or unused vertex */
  VLS_EMAXSTEPS = 5,       /* step limit reached (state up to the limit is still returned) */
  VLS_ESLOTS = 6,          /* more than 4 layers met at one vertex */
  VLS_ELAYERS = 7,         /* layer table or event buffer capacity exceeded */
  VLS_ELOOPFAIL = 8,       /* a tunnel pass never reached the far side / trace got stuck */
  VLS_ETIMEOUT = 9,        /* reserved: bounded device-side wait gave up */
  VLS_ENOMEM = 10,         /* device or host allocation failed */
  VLS_ECUDA = 11,          /* CUDA runtime error (kernel launch / copy) */
  VLS_ESTALL = 12,         /* no front left but parts of the surface were never covered */
  VLS_ETOOLARGE = 13       /* input above the fixed limits of vls_tunnel_pass_noalloc */
} vls_status;

/*
 * Precision of the layer values (the paper does not state one):
 *   VLS_FP64          values stored and updated in FP64, every operation rounded on its own in
 *                     a fixed order (results are bit-reproducible).
 *   VLS_FP32_RECHECK  values stored as float; the Eq. (2) step of a frontier row runs in FP32.
 *                     A row whose step takes a decision within recheck_margin of its threshold
 *                     (snap at eps0 or 1 - eps0, the level theta_iso) or where several layers
 *                     meet is recomputed in FP64 from the same stored inputs, and its values are
 *                     rounded to float without crossing any threshold.  FP64 is used for nothing
 *                     else on the step path but the mass check (vls_stats.mass_resid).
 *   VLS_BF16_RECHECK  values stored as bfloat16 (8 significant bits); the step arithmetic is that of
 *                     VLS_FP32_RECHECK on the widened values, with the same FP64 recheck, and every
 *                     stored value is rounded to bfloat16 without crossing any threshold.  Halves the
 *                     value bytes again; the coarser storage moves the trajectory away from the FP64
 *                     one by far more than FP32 storage does (see vls_result_state).
 */
typedef enum { VLS_FP64 = 0, VLS_FP32_RECHECK = 1, VLS_BF16_RECHECK = 2 } vls_precision;

/*
 * Options.  Defaults (vls_default_options) are the paper's constants (Sec. 2,
 * "Implementation details": mu = 1/4, e = 1/30, a = 1/25, w = a/5) and the following
 * readings of what the paper leaves open: dt = dt_factor * lbar^2 / (4 mu a^2 / 2) with
 * dt_factor 0.5; lbar = eta / 4 with eta = pi a / sqrt(2 w) (band width of the
 * travelling wave of Eq. (2)); snap threshold eps0 = 1e-3; isoline / arrival level
 * theta_iso = 0.5; recheck margin 1e-5 (ten times the worst-case rounding of the FP32 step).
 */
typedef struct {
  double mu, e, a, w;       /* Eq. (2) coefficients */
  double dt_factor;         /* Euler step as a fraction of the diffusion stability limit */
  double eps0;              /* snap: values below eps0 -> 0, above 1 - eps0 -> 1 */
  double theta_iso;         /* isoline level of handle loops, arrival level of tunnel passes */
  double lbar;              /* operator length scale; <= 0 selects eta / 4 */
  double recheck_margin;    /* FP32 / BF16 forms: rows deciding within this of a threshold are redone in FP64; (0, 0.25) */
  int32_t max_steps;        /* initial-pass step limit (per problem) */
  int32_t max_pass_steps;   /* tunnel-pass step limit (per pass) */
  int32_t tunnels;          /* 1: run the tunnel passes (Sec. 3.2) */
  int32_t keep_state;       /* 1: results carry the final per-vertex state (layer, value, cover) */
  int32_t record_steps;     /* 1: results carry per-step frontier size, band size, band hash */
  int32_t sync_interval;    /* steps between host polls of the device "still running" flag */
  int32_t threads;          /* threads per block of the frontier kernels; with blocks_per_sm */
  int32_t blocks_per_sm;    /* grid = blocks_per_sm x SM count (clamped to what fits).  Both 0:
                               autotuned -- the first batch of a device, precision and size class
                               (total vertices rounded up to a power of two) runs the first 600
                               steps of its initial pass under each candidate shape and band
                               union-find variant and keeps the fastest for the life of the
                               process; the tunnel and refinement pass kernels keep the default
                               shapes */
  vls_precision precision;
  int32_t profile;          /* 1: time every frontier-update launch with CUDA events (vls_stats) */
  int32_t host_loop;        /* 1: launch each step's kernels from the host instead of running the
                               step loops as device-driven CUDA graphs (same results) */
  int32_t hook_variant;     /* band union-find: 1 one thread per band row, 2 a group of 8 lanes per
                               band row (one neighbour each), 0 autotuned or 2 (same results) */
  int32_t rows_per_warp;    /* frontier rows a warp of the initial pass's one-thread-per-row
                               kernels takes per pass: 32, 16 or 8 (fewer rows per warp spread a
                               small frontier over more warps and schedulers); 0 autotuned with the
                               launch shape, or 32 when the shape is given (same results).  The
                               tunnel and refinement pass kernels take 32 */
  int32_t refine;           /* 1: after each tunnel pass, the handle-refinement pass of its handle
                               (Sec. 3.3; needs tunnels = 1) */
  double offset;            /* loop classification (Sec. 3.5): normal offset as a fraction of the
                               mesh's mean edge length; > 0 */
  int32_t K;                /* layers that may meet at one vertex within a step: 0 or 4 (fixed by
                               the per-row output buffer; other values are VLS_EINVAL) */
  int32_t laplacian;        /* operator: 0 = uniform scaled Laplacian L_vu = s / d_v, L_vv = -s (the
                               only one built; other values are VLS_EINVAL) */
  int32_t max_passes;       /* tunnel (and refinement) passes per problem, in handle order; 0: all */
  int32_t autotune;         /* 1: tune the launch shapes when threads = blocks_per_sm = 0 (see
                               blocks_per_sm); 0: default shapes without tuning runs */
  double drift_bound;       /* FP32 / BF16 forms: a threshold decision (snap at eps0 or 1 - eps0,
                               theta_iso) whose FP64 value from the stored inputs lies within this of
                               its threshold is counted "uncertified": the low-precision trajectory
                               may have drifted from the FP64 one by this much, so the decision could
                               go the other way there.  0 selects 1e-6 (FP32) or 2e-2 (BF16), above
                               the largest drift measured on the workloads */
  int32_t streamlines;      /* 1: trace the PL streamline of every tunnel and refinement pass
                               (vls_result_streamline); 0: only the vertex cycles */
} vls_options;

/* A closed, oriented triangle mesh: X[nv][3] positions, F[nf][3] vertex ids (CCW). */
typedef struct {
  const double *X;
  int64_t nv;
  const int32_t *F;
  int64_t nf;
  int32_t device; /* 0: X and F are host pointers; 1: device pointers on the current device */
} vls_mesh;

typedef struct vls_ctx vls_ctx;
typedef struct vls_result vls_result;

typedef struct {
  int32_t steps;           /* initial-pass steps executed */
  int32_t tunnel_steps;    /* max tunnel-pass steps over this problem's passes */
  int64_t row_updates;     /* frontier rows updated in the initial pass */
  int64_t pass_updates;    /* rows updated in the tunnel passes */
  int32_t merges, splits, ends, layers;
  double ms_operator, ms_initial, ms_tunnel, ms_download; /* batch-wide phase times */
  int64_t kernel_launches; /* kernels launched for the whole batch */
  /* profile = 1: summed device time and launch count of the initial-pass update kernel and
   * of the tunnel-pass update kernel (batch-wide), from CUDA events around each launch */
  double ms_update, ms_pass_update;
  int64_t n_update, n_pass_update;
  int64_t h2d_bytes, d2h_bytes; /* batch-wide host<->device bytes of this call */
  /* precision = VLS_FP32_RECHECK or VLS_BF16_RECHECK: rows of the initial pass / tunnel passes whose FP32 step had
   * a decision within recheck_margin of its threshold (or several layers) and was redone in
   * FP64 (batch-wide); 0 in the FP64 form */
  int64_t rechecks, pass_rechecks;
  /* Mass check of the diffusion step, in FP64: at every initial-pass step the base's Laplacian
   * weighted by the lumped masses (m_v = d_v / s, so that m_v L_vu = 1 is symmetric) must sum to
   * zero over the rows that can change; this is the largest |sum| / sum of the terms'
   * magnitudes seen over the problem's steps.  Rounding alone gives about 1e-16 in the FP64
   * form and 1e-7 in the FP32 form; a wrong operator entry or a lost neighbour gives far more. */
  double mass_resid;
  /* The same check in the tunnel passes: the kept-edge operator of a pass is symmetric in the same
   * way, and the flux into the pass's sources (held at 1, never rows) is taken out; the largest
   * residual over the steps of the problem's passes. */
  double pass_mass_resid;
  /* refinement passes (Sec. 3.3): rows updated, max steps over the problem's passes, phase time
   * (batch-wide), largest mass-check residual */
  int64_t refine_updates;
  int32_t refine_steps;
  double ms_refine;
  double refine_mass_resid;
  double mean_edge;        /* the mesh's mean edge length (the classification offset's unit) */
  /* FP32 / BF16 forms: uncertified decisions (vls_options.drift_bound) of the initial pass, of the
   * tunnel passes and of the refinement passes; 0 in the FP64 form.  A result can differ from the
   * FP64 one only after such a decision. */
  int64_t uncertified, pass_uncertified, refine_uncertified;
} vls_stats;

/* Fill *o with the defaults above. */
VLS_API void vls_default_options(vls_options *o);

/* Derived constants of o: out[0] eta, out[1] lbar, out[2] dt, out[3] s = 4 / lbar^2. */
VLS_API void vls_constants(const vls_options *o, double out[4]);

/*
 * Create a context on the current CUDA device.  `cuda_stream` is a cudaStream_t (may be
 * NULL for the default stream); every kernel and copy is issued on it.  The context keeps
 * one grow-only device arena, sized to the largest batch it has run and released by
 * vls_destroy(); a call allocates device memory only when its batch needs more.
 */
VLS_API vls_status vls_create(vls_ctx **ctx, const vls_options *o, void *cuda_stream);
VLS_API void vls_destroy(vls_ctx *ctx);

/*
 * Loop detection for one mesh and one seed vertex (Sec. 3.1-3.2, Sec. 5): validates the
 * mesh, builds the operator, runs the initial pass and one tunnel pass per handle.
 * *out receives a result with one problem (even on error; its status says why).
 */
VLS_API vls_status vls_detect(vls_ctx *ctx, const vls_mesh *m, int32_t seed_vertex, vls_result **out);

/*
 * Batched detection: n_mesh meshes, mesh i with seeds_per_mesh[i] seed vertices taken in
 * order from `seeds`.  Problems are numbered mesh-major, seed-minor.  All problems advance
 * in the same kernels (one launch per step for the whole batch).  Each problem reports its
 * own status; one failing problem does not fail the others.  Returns VLS_OK unless the
 * batch as a whole could not run.
 */
VLS_API vls_status vls_detect_batch(vls_ctx *ctx, int32_t n_mesh, const vls_mesh *meshes, const int32_t *seeds,
                            const int32_t *seeds_per_mesh, vls_result **out);

VLS_API int32_t vls_result_count(const vls_result *r);                 /* problems in the result */
VLS_API vls_status vls_result_status(const vls_result *r, int32_t p);
VLS_API int32_t vls_result_genus(const vls_result *r, int32_t p);      /* (2 - chi) / 2 */
VLS_API vls_status vls_result_stats(const vls_result *r, int32_t p, vls_stats *s);

/* kind 0: handle loops (Sec. 3.1), kind 1: tunnel loops (Sec. 3.2), kind 2: refined handle loops
 * (Sec. 3.3); kinds 1 and 2 have one entry per handle (status -1 where the pass did not run) */
VLS_API int32_t vls_result_num_loops(const vls_result *r, int32_t p, int32_t kind);
/*
 * Loop i of the given kind.  Handles: *verts = the collapsed inside-vertex cycle of the
 * theta-isoline, *pts = its FP64 isoline points (one per crossing edge, *npts of them).
 * Tunnels and refined handles: *verts = the vertex cycle, *pts = NULL.
 */
VLS_API vls_status vls_result_loop(const vls_result *r, int32_t p, int32_t kind, int32_t i, const int32_t **verts,
                           int64_t *n, const double **pts, int64_t *npts);
/* Handle i: crossing edges [n][2] (inside, outside) in loop order; info[0] step, [1] layer,
 * [2] Reeb node of its merge; *length = polyline length of the isoline points. */
VLS_API vls_status vls_result_handle(const vls_result *r, int32_t p, int32_t i, const int32_t **edges, int64_t *n,
                             int32_t info[3], double *length);
/* Tunnel i (one per handle): info[0] status, [1] step its pass stopped, [2] first vertex reached */
VLS_API vls_status vls_result_tunnel(const vls_result *r, int32_t p, int32_t i, int32_t info[3]);
/* Refined handle i (Sec. 3.3; one per handle): info as vls_result_tunnel.  Its pass starts on the
 * tunnel loop (made simple by erasing its closed sub-loops) and spreads to the loop's left; the
 * loop's right neighbours are the far side. */
VLS_API vls_status vls_result_refined(const vls_result *r, int32_t p, int32_t i, int32_t info[3]);
/* Loop classification (Sec. 3.5) of handle i's loops: out[0] handle loop, out[1] tunnel loop,
 * out[2] refined handle loop: length of the loop offset along the unit vertex normals by
 * offset x mean edge length, minus its length (NaN where the loop does not exist).  Tunnel loops
 * tend to shrink (< 0), handle loops to grow (> 0). */
VLS_API vls_status vls_result_offset_change(const vls_result *r, int32_t p, int32_t i, double out[3]);
/* PL streamline (Sec. 3.2: the loop traced back from the first point reached, against the
 * gradient of the arrival time) of handle i's tunnel pass (kind 0) or refinement pass (kind 1).
 * Arrival time: the step at which theta_iso was crossed, with the fraction of that step from a
 * linear interpolation of the value in time; it is interpolated linearly over the faces of the
 * pass's cut, restricted domain.  The path runs from the first far-side vertex reached down the
 * steepest descent, face by face (through a vertex into the steepest face whose corner holds the
 * descent direction, else along the steepest descending edge; along an edge where the descent
 * leaves no face), to a source, and is closed along the border as the vertex cycle is.
 * *status: VLS_OK, VLS_ELOOPFAIL (no descent left), VLS_ELAYERS (more points than the budget
 * min(16384, nv / 4 + 64) for a mesh of nv vertices), -1 (not traced: the pass did not run or
 * failed, or streamlines = 0).  *pts = [n][3] positions of the closed polyline's points (the start vertex,
 * edge crossings, vertices passed), library-owned; *length = its length, closing segment
 * included.  VLS_EINVAL for a bad index or kind. */
VLS_API vls_status vls_result_streamline(const vls_result *r, int32_t p, int32_t i, int32_t kind, int32_t *status,
                                         const double **pts, int64_t *n, double *length);

/* Reeb graph (Sec. 5): nodes [n][2] = (kind 0 SEED / 1 SPLIT / 2 MERGE / 3 END, step),
 * positions [n][3] (mean of the narrow band); arcs = layers [L][3] = (birth node, death
 * node, final state: 2 dead after split, 3 merged, 4 ended). */
VLS_API vls_status vls_result_reeb(const vls_result *r, int32_t p, const int32_t **nodes, const double **pos,
                           int32_t *n_nodes, const int32_t **layers, int32_t *n_layers);

/* Final per-vertex state (keep_state = 1): layer id (0 none), value, cover step (-1 never). */
VLS_API vls_status vls_result_state(const vls_result *r, int32_t p, const int32_t **layer, const double **phi,
                            const int32_t **cover, int64_t *nv);
/* profile = 1: per-kernel device time of the batch from CUDA events around every launch
 * (host-driven launches).  names[i] (static strings), launches[i], ms[i] for i < *n. */
VLS_API vls_status vls_result_kernel_times(const vls_result *r, const char *const **names, const int64_t **launches,
                                           const double **ms, int32_t *n);
/* Per-step records (record_steps = 1): [steps][5] = frontier rows, band vertices, band hash
 * low 32 bits, high 32 bits, uncertified decisions of the step (FP32 / BF16 forms). */
VLS_API vls_status vls_result_records(const vls_result *r, int32_t p, const int64_t **rec, int32_t *steps);

VLS_API void vls_result_free(vls_result *r);

/*
 * One tunnel pass without any device allocation.  The paper has no counterpart: this is a
 * convenience for callers that cannot allocate device memory (code that must run inside a
 * pre-sized memory pool or an allocation-free region, where every device byte is budgeted
 * up front).  It computes exactly the tunnel loop vls_detect reports for a handle, from:
 *   F [nf][3]       device, the closed oriented mesh (vertex ids < nv) given to vls_detect
 *   cover [nv]      device, the cover step of every vertex (vls_result_state)
 *   handle_step     the step at which the handle was found (vls_result_handle info[0])
 *   edges [n][2]    device, the handle's crossing edges in loop order (vls_result_handle)
 * and writes, on the device, out_verts[0..n) (capacity nv) and out_info[4] = status, step the
 * pass stopped, first vertex reached, n.  Options o may be NULL (defaults); the pass always runs
 * in FP64 (o->precision is not used), so it matches the FP64 form of vls_detect.
 * Limits: nv <= 262144, nf <= 786432, n_edges <= 65536; larger inputs return VLS_ETOOLARGE.  A
 * vertex with more than 64 neighbours gives out_info[0] = VLS_EINVAL, as in vls_detect.
 * All scratch (about 22 MB) lives in one static device array of the library.  The array is
 * reserved on a device when the CUDA module holding it is loaded there: under CUDA's default
 * lazy module loading that is the first call of this function on that device (with
 * CUDA_MODULE_LOADING=EAGER, the creation of the device's context); from then on the device
 * holds it until the process exits.  That first call also looks up the array's device
 * address, so it can fail with VLS_ECUDA when the device has no room left for the array:
 * make it before entering any region where allocation is not allowed, and before any stream
 * capture.  Later calls allocate nothing and return after queueing one kernel on cuda_stream
 * (NULL: default stream).  Calls share the array: calls that overlap on the GPU (different
 * streams, different host threads) race and must be serialised by the caller.
 */
VLS_API vls_status vls_tunnel_pass_noalloc(const int32_t *F, int64_t nf, int64_t nv, const int32_t *cover,
                                           int32_t handle_step, const int32_t *edges, int64_t n_edges,
                                           const vls_options *o, void *cuda_stream, int32_t *out_verts,
                                           int32_t *out_info);
VLS_API const char *vls_status_string(vls_status s);

#ifdef __cplusplus
}
#endif
#endif /* VLS_H */
