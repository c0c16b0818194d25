/*
 * vls_oracle.h -- plain, slow, single-threaded FP64 CPU oracle of the
 * variational loop-shrinking hot path (initial pass + tunnel passes).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load or run this code.  It shares no code,
 * header, table or constant generator with the CUDA library, and it never calls
 * into it.
 *
 * Every public function returns results in oracle-owned memory that stays valid
 * until orc_free().
 */
#ifndef VLS_ORACLE_H
#define VLS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double mu, e, a, w;     /* Eq. (2) coefficients (Sec. 2, "Implementation details") */
  double dt_factor;       /* c in dt = c * lbar^2 / (4 D), D = mu a^2 / 2 */
  double eps0;            /* snap threshold */
  double theta_iso;       /* isoline / arrival threshold */
  double lbar;            /* operator length scale; <= 0 selects eta / 4 */
  int32_t max_steps;      /* initial-pass step limit */
  int32_t max_pass_steps; /* tunnel-pass step limit */
  int32_t seed_ring;      /* 1: seed region is the closed 1-ring of the seed vertex; 0: the vertex alone */
  int32_t naive;          /* 1: update/scan every vertex each step (cross-check of the frontier restriction) */
  int32_t tunnels;        /* 1: run the tunnel passes */
  int32_t record_steps;   /* 1: keep per-step frontier size / band size / band hash */
  int32_t refine;         /* 1: run the handle-refinement pass after each tunnel pass (Sec. 3.3) */
  double offset;          /* loop classification: normal offset in mean edge lengths (Sec. 3.5) */
  int32_t max_passes;     /* tunnel (and refinement) passes run: the first max_passes handles; 0: all */
  int32_t streamlines;    /* 1: trace the PL streamline of every successful pass (Sec. 3.2) */
} orc_options;

typedef struct orc_run orc_run;

void orc_default_options(orc_options *o);
/* derived constants: out[0]=eta, out[1]=lbar, out[2]=dt, out[3]=s (= 4/lbar^2) */
void orc_constants(const orc_options *o, double out[4]);

orc_run *orc_detect(const double *X, int64_t nv, const int32_t *F, int64_t nf, int32_t seed_vertex,
                    const orc_options *o);
void orc_free(orc_run *r);

int32_t orc_status(const orc_run *r);
int32_t orc_genus(const orc_run *r);   /* (2 - chi) / 2 */
int32_t orc_steps(const orc_run *r);   /* initial-pass steps executed */
/* counters: [0] frontier row updates, [1] anomalies, [2] tunnel-pass row updates,
 *           [3] merge events, [4] split events, [5] end events, [6] layers created */
const int64_t *orc_counters(const orc_run *r);

/* final state of the initial pass: layer id held (0 none), its value, cover step (-1 never) */
const int32_t *orc_state_layer(const orc_run *r);
const double *orc_state_phi(const orc_run *r);
const int32_t *orc_cover(const orc_run *r);

/* per-step records (record_steps): n = steps, each [frontier, band, hash_lo, hash_hi] */
const int64_t *orc_step_records(const orc_run *r, int32_t *n);

/* Reeb graph: nodes (kind 0 SEED, 1 SPLIT, 2 MERGE, 3 END; step), positions, arcs = layers */
int32_t orc_num_nodes(const orc_run *r);
const int32_t *orc_nodes(const orc_run *r);     /* [n][2]: kind, step */
const double *orc_node_pos(const orc_run *r);   /* [n][3] */
int32_t orc_num_layers(const orc_run *r);
const int32_t *orc_layers(const orc_run *r);    /* [L][3]: birth node, death node, final state */

/* handle loops in emission order */
int32_t orc_num_handles(const orc_run *r);
/* info: [0] step, [1] layer, [2] merge node, [3] n crossing edges, [4] n inside vertices */
const int32_t *orc_handle_info(const orc_run *r, int32_t h);
const int32_t *orc_handle_edges(const orc_run *r, int32_t h);   /* [n][2] inside, outside */
const int32_t *orc_handle_verts(const orc_run *r, int32_t h);   /* collapsed inside-vertex cycle */
const double *orc_handle_points(const orc_run *r, int32_t h);   /* [n][3] isoline points */
double orc_handle_length(const orc_run *r, int32_t h);

/* tunnel loops, one per handle: info [0] status, [1] stop step, [2] b*, [3] n verts */
const int32_t *orc_tunnel_info(const orc_run *r, int32_t h);
const int32_t *orc_tunnel_verts(const orc_run *r, int32_t h);
/* arrival steps of pass h (-1 unreached), kept only when record_steps is set */
const int32_t *orc_tunnel_arrival(const orc_run *r, int32_t h);
/* arrival times of pass h with the fraction of the step at which theta was crossed (linear in time
 * within the step; sources 0, unreached -1), kept only when record_steps is set */
const double *orc_tunnel_arrival_time(const orc_run *r, int32_t h);

/* refined handle loops (Sec. 3.3), one per handle: info [0] status (-1: not run), [1] stop step,
 * [2] first vertex reached, [3] n verts; verts = the vertex cycle */
const int32_t *orc_refined_info(const orc_run *r, int32_t h);
const int32_t *orc_refined_verts(const orc_run *r, int32_t h);
/* loop classification (Sec. 3.5): length change of the handle loop, the tunnel loop and the refined
 * handle loop of handle h when offset along the unit vertex normals by offset x mean edge length
 * (NaN where the loop does not exist); > 0 reads as a handle, < 0 as a tunnel */
const double *orc_loop_offset_change(const orc_run *r, int32_t h);
double orc_mean_edge(const orc_run *r);
/* PL streamlines (Sec. 3.2) of the tunnel pass (kind 0) and the refinement pass (kind 1) of handle h:
 * returns the status (-1: not run); n points [n][3] of the closed polyline, its length */
int32_t orc_streamline(const orc_run *r, int32_t h, int32_t kind, int64_t *n, double *len, const double **pts);
/* the streamline trace alone, on a given arrival field tf (sources 0, unreached -1) with the given
 * edges cut: writes up to cap points, returns the status, *n_out points, the source reached */
int32_t orc_trace_streamline(const double *X, int64_t nv, const int32_t *F, int64_t nf, const double *tf,
                             const int32_t *cut_edges, int64_t ncut, int32_t start, double *pts, int64_t cap,
                             int64_t *n_out, int32_t *end_vertex);

#ifdef __cplusplus
}
#endif
#endif
