/* Served ensemble: a runtime that admits independent cases of the time stepper
 * (include/ns.h) while others are running on the same GPU.
 *
 * The paper runs many cases of its method -- ensembles over soil parameters and input
 * waves (Sec. 2.3, 3) -- and reports throughput per case (Table 1).  This runtime keeps
 * a first-come-first-served queue of submitted cases and admits the head of the queue
 * as soon as a slot and memory are free: its spring state is kept in HBM when the
 * device budget allows, otherwise streamed from pinned host memory when the pinned
 * budget allows (Alg. 3), otherwise the case waits.
 *
 * Two ways to run the admitted cases:
 *  - batch = 0: every case in its own context (own streams and CUDA graphs) driven by its
 *    own host thread, so the kernels of all admitted cases overlap on the device; a
 *    case's result does not depend on what else runs (with NS_SCATTER_COLOUR it is
 *    bit-identical to running it alone);
 *  - batch = 1 (continuous batching): admitted cases with resident state and the same
 *    solver settings (precision form, dt, tolerances, inner solve, Rayleigh band, graphs)
 *    advance together as the members of one batched context -- the disjoint union of
 *    their meshes, each member with its own springs per point, materials, input and CG
 *    (ns_set_members, ns_set_member_springs) -- so that one launch of every kernel
 *    serves all of them.  When a case arrives or finishes, the batch is re-formed: a new
 *    context for the new membership takes the continuing members' state from the old one
 *    device to device and carries on from their own steps.  The atomic scatter is used
 *    (a member's result agrees with the case run alone to rounding).  Cases that only fit
 *    with streamed state run in their own context as with batch = 0.  Re-forming holds
 *    the old and the new context at once, so with batch = 1 cases are admitted only while
 *    the admitted cases' device bytes stay within half the device budget.
 *
 * Ownership: ns_server_submit copies every input array; results are copied into
 * caller-owned buffers by ns_server_result.  The server owns its threads, contexts and
 * device/pinned memory until ns_server_destroy, which waits for running cases.
 * All calls are thread-safe.  Errors: NS_ERR_* of include/ns.h.
 */
#ifndef NS_SERVER_H
#define NS_SERVER_H

#include <stdint.h>

#include "ns.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ns_server ns_server;

typedef struct {
  int32_t device;           /* CUDA device ordinal */
  int64_t device_budget;    /* bytes of device memory the admitted cases may hold together */
  int64_t pinned_budget;    /* bytes of pinned host memory for streamed spring state */
  int32_t max_active;       /* cases advanced concurrently (>= 1) */
  int32_t quantum_steps;    /* steps a case (or a batch) advances between checks of the stop flag,
                               arrivals and departures */
  int32_t batch;            /* 1: continuous batching of compatible cases (above); 0: a context per case */
} ns_server_config;

/* One case: the arrays of ns_upload_mesh, ns_set_materials, ns_set_boundary and
 * ns_set_ground_motion, the solver configuration of its context and the number of steps.
 * The surface record of all n_steps steps is kept (n_surf nodes). */
typedef struct {
  int64_t n_nodes;
  const double *xyz;
  int64_t n_elems;
  const int32_t *conn;
  const int32_t *mat;
  int32_t n_mat;
  const ns_material *mats;
  int64_t n_faces;
  const int32_t *faces;
  const int32_t *face_elem;
  const int32_t *face_kind;
  int64_t n_surf;
  const int32_t *surf;
  int64_t n_samples;
  const double *acc;
  ns_config cfg;            /* cfg.device, surface_ring_steps and device_state_budget are set
                               by the server */
  int64_t n_steps;
} ns_case;

#define NS_CASE_QUEUED 0
#define NS_CASE_RUNNING 1
#define NS_CASE_DONE 2
#define NS_CASE_FAILED 3

typedef struct {
  int32_t state;            /* NS_CASE_* */
  int32_t error;            /* NS_OK or the failing call's NS_ERR_* */
  int32_t streamed;         /* 1: admitted with its spring state in pinned host memory */
  int32_t batches;          /* batched contexts the case ran in (0: its own context) */
  double t_submit, t_admit, t_done;  /* seconds since the server's creation */
  int64_t device_bytes;     /* device memory reserved for the case at admission */
  int64_t state_bytes;      /* its spring state */
  int64_t elem_steps;       /* n_elems * n_steps */
  double ms_device;         /* CUDA-event time of its ns_advance calls (batched: its share of the
                               batches' time, in proportion to its elements) */
  int64_t kernel_launches;  /* the library's kernels its context launched (batched: its share) */
  double t_reform;          /* batched: seconds its batches spent being re-formed around it */
} ns_case_stats;

/* Device bytes a case needs with all its state resident (*device_bytes), the part of it
 * that is spring state (*state_bytes), and the device bytes when all spring state is
 * streamed through ring_depth chunk buffers (*streamed_device_bytes).  Host-only. */
int ns_case_bytes(const ns_case *c, int64_t *device_bytes, int64_t *state_bytes, int64_t *streamed_device_bytes);

int ns_server_create(ns_server **out, const ns_server_config *cfg);

/* Queue a case; *id identifies it.  NS_ERR_INVALID_ARG for inconsistent sizes,
 * NS_ERR_OOM_DEVICE if it could never be admitted within the budgets. */
int ns_server_submit(ns_server *s, const ns_case *c, int64_t *id);

/* State and timing of a case. */
int ns_server_status(ns_server *s, int64_t id, ns_case_stats *st);

/* Block until the case is done or failed, at most timeout_s seconds (NS_ERR_TIMEOUT). */
int ns_server_wait(ns_server *s, int64_t id, double timeout_s);

/* Surface record of a finished case: u, v, a [n_steps][n_surf][3] (NULL skips a field);
 * the case's own error if it failed. */
int ns_server_result(ns_server *s, int64_t id, double *u, double *v, double *a);

/* Forget a finished case (its result is freed). */
int ns_server_release(ns_server *s, int64_t id);

/* Stop admitting, wait for the running cases, free everything. */
void ns_server_destroy(ns_server *s);

#ifdef __cplusplus
}
#endif

#endif
