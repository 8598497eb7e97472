/* ns.h -- C ABI of the GB300 nonlinear seismic ground-response time stepper.
 *
 * One implicit Newmark-beta step (beta = 1/4, gamma = 1/2) of a 3D quadratic
 * tetrahedral finite-element ground model, as stated in Sec. 2.1 (Eq. 1):
 *   (4/dt^2 M + 2/dt C^n + K^n) du^n = f^n - q^{n-1} + C^n v^{n-1} + M (a^{n-1} + 4/dt v^{n-1}),
 *   q^n = q^{n-1} + K^n du^n,  u^n = u^{n-1} + du^n,
 *   v^n = -v^{n-1} + 2/dt du^n,  a^n = -a^{n-1} - 4/dt v^{n-1} + 4/dt^2 du^n,
 * solved by an element-by-element (EBE) preconditioned CG (Sec. 2.2, Alg. 4),
 * with K_e = sum_j w_j B^T D_j B (Eq. 2) and D from a multi-spring model of
 * modified Ramberg-Osgood springs with the Masing rule (Sec. 2.1), whose
 * 40-byte-per-spring state is kept in HBM or streamed from pinned host memory
 * in chunks that overlap with compute (Alg. 3).  The stiffness is lagged: the
 * solve of step n uses D left by step n-1 (Alg. 4).
 *
 * Conventions (all calls):
 *  - Every call returns an int status: NS_OK (0) or a negative NS_ERR_* code;
 *    ns_last_error(ctx) returns a static, human-readable message for the
 *    last failure on that context.
 *  - Inputs are caller-owned host buffers, read (copied) during the call and
 *    never retained.  Outputs go into caller-owned host buffers.
 *  - The context owns all device memory, pinned host memory, streams and
 *    events it creates, until ns_destroy.
 *  - A context is not thread-safe; different contexts are independent.
 *  - Units are SI.  Node vectors are node-major [n][3] (x, y, z).
 *  - Element node order: vertices 0-3 (positive orientation), then edge nodes
 *    on (0,1) (1,2) (0,2) (0,3) (1,3) (2,3).  Elements must be straight-sided
 *    (edge nodes at edge midpoints); geometry is taken from the vertices.
 *  - Voigt order of strain/stress: xx yy zz yz xz xy, shear strains in
 *    engineering form.  A 6x6 tangent D is returned full (36 doubles, row major).
 */
#ifndef NS_H
#define NS_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NS_OK 0
#define NS_ERR_INVALID_ARG (-1)   /* bad size, pointer, value or call order */
#define NS_ERR_OOM_DEVICE (-2)    /* device allocation failed */
#define NS_ERR_OOM_PINNED (-3)    /* pinned host allocation failed */
#define NS_ERR_CUDA (-4)          /* a CUDA runtime call failed */
#define NS_ERR_BAD_MESH (-5)      /* non-positive volume, curved edge, bad index */
#define NS_ERR_NOT_CONVERGED (-6) /* CG reached cg_max_iter; the step is not applied */
#define NS_ERR_TIMEOUT (-7)       /* a bounded host wait on the device expired */
#define NS_ERR_STATE (-8)         /* mesh/materials/boundary/input missing */

#define NS_PREC_FP64 0   /* FP64 PCG with FP64 3x3 block-Jacobi (plain method) */
#define NS_PREC_FP64_IR 1 /* FP64 outer CG, FP32 inner CG as preconditioner (paper's precision policy) */
#define NS_PREC_FP64_IR16 2 /* as NS_PREC_FP64_IR, the inner operator reading the tangent D in FP16
                               (D / G0 of the element's material; FP32 arithmetic) */

#define NS_SCATTER_ATOMIC 0 /* element results added with FP64/FP32 atomics (fast) */
#define NS_SCATTER_COLOUR 1 /* greedy element colouring, plain stores (deterministic) */

typedef struct ns_ctx ns_ctx;

/* Solver and runtime configuration.  ns_config_default fills documented
 * defaults; fields may then be changed before ns_create. */
typedef struct {
  int32_t n_springs;           /* springs per integration point, >= 5 (Sec. 2.1 uses 150) */
  double dt;                   /* time step (s), > 0 */
  double cg_tol;               /* relative residual ||r||/||b|| at convergence (Sec. 2.3: 1e-8) */
  int32_t cg_max_iter;         /* CG iteration limit per step */
  int32_t x0_prev;             /* 1: CG starts from the previous increment, 0: from zero */
  int32_t precision;           /* NS_PREC_* */
  int32_t scatter;             /* NS_SCATTER_* */
  int64_t chunk_elems;         /* elements per streamed state chunk (Alg. 3 partition) */
  int32_t ring_depth;          /* device chunk buffers, >= 2 (3 lets H2D, compute and D2H overlap) */
  int64_t device_state_budget; /* bytes of spring state kept in HBM; elements beyond it are
                                  host-resident and streamed; < 0: all resident */
  double rayleigh_f1, rayleigh_f2; /* Rayleigh damping calibration frequencies (Hz) */
  int64_t surface_ring_steps;  /* steps of surface response kept on the device */
  int32_t device;              /* CUDA device ordinal */
  int32_t timing;              /* 1: time kernels with CUDA events (ns_get_stats) */
  int32_t inner_max_iter;      /* NS_PREC_FP64_IR*: at most this many inner FP32 CG iterations per
                                  preconditioner call (default 45) */
  double inner_tol;            /* NS_PREC_FP64_IR*: inner relative residual target (default 1e-4) */
  double wait_timeout_s;       /* bound on each host wait for the device */
  int32_t graphs;              /* 1: each outer iteration of the flexible solver (inner FP32 solve
                                  included) and each batch of plain CG iterations is captured once
                                  as a CUDA graph and replayed; per-kernel times of the operators
                                  inside are then not recorded (ns_stats ms_ebe32 stays 0) */
  int32_t stage_elements;      /* FP32 inner operator (atomic scatter, one member): 1 stages each
                                  256-element tile of element data in shared memory with bulk copies;
                                  2 has each warp copy its 32 elements' tangent rows to shared memory
                                  asynchronously while it gathers the nodal values; 0 per-thread
                                  loads; -1 (default): 2 for the FP32 tangent, 0 for the FP16 one */
  int32_t l2_prefetch;         /* 1: each block of the element operators first prefetches its slice
                                  of the element rows into L2 with a bulk prefetch */
  int32_t pair_operator;       /* 1: the FP64-accuracy operator applications (right-hand side, outer
                                  CG, q update) run in double-float arithmetic on the FP32 pipes
                                  (relative accuracy ~1e-13, FP64 node vectors); 0: FP64 */
  int32_t stream_mode;         /* spring state beyond device_state_budget: NS_STREAM_RING (chunks
                                  copied through device buffers, Alg. 3) or NS_STREAM_ZERO_COPY
                                  (the spring kernel reads and writes the pinned host arrays in
                                  place over the host link) */
  int32_t spring_tile_points;  /* spring kernel launch shape: integration points per block (a
                                  multiple of 4 whose float pairs fit 200 KB of shared memory);
                                  0 (default): a size heuristic until ns_autotune picks */
  int32_t spring_tile_blocks;  /* its register budget: 4 (default: 64 registers a thread, four
                                  resident blocks per SM; measured faster at every spring count
                                  tried) or 1 (the compiler's budget; 0 reads as 1) */
  int32_t spring_tensor_cores; /* 1: the tangent D = K_b m m^T + sum_k G_k T_k is assembled on
                                  the tensor cores (bf16 digit products, exact FP32 sums,
                                  FP64-level result) with 16-point blocks when S <= 256; 0 (default, measured faster on GB300):
                                  double-float sums on the FP32 pipes */
  int32_t fault_pinned_alloc;  /* fault injection for tests (0 = off): the k-th pinned host
                                  allocation of this context (counted from ns_create, k >= 1)
                                  fails as if the host were out of pinned memory */
  int32_t fault_state_copy;    /* fault injection for tests (0 = off): the k-th state-stream copy
                                  of this context (a chunk's H2D or D2H, Alg. 3; k >= 1) fails
                                  before it is issued, as a failed cudaMemcpyAsync would */
  int32_t multigrid;           /* NS_PREC_FP64_IR*: 1 = two-level preconditioner (Sec. 2.2, after
                                  [SC14]): each outer iteration first solves the linear-element
                                  coarse model (the vertices, P^T A P) roughly in FP32, interpolates
                                  that solution onto the quadratic nodes and starts the inner FP32
                                  PCG from it; one member only; 0 (default): inner PCG from zero */
  int32_t coarse_max_iter;     /* multigrid: coarse PCG iterations per outer iteration (at most) */
  double coarse_tol;           /* multigrid: coarse relative residual target */
  int32_t shared_members;      /* M > 1: a batch of M members on ONE mesh (Sec. 2.2, Alg. 4: the
                                  problem sets share the mesh).  ns_upload_mesh and ns_set_boundary
                                  then take the shared mesh once; its connectivity and geometry are
                                  stored once and read by every member, while tangent, spring state,
                                  materials and node vectors are per member, member after member
                                  (member k: elements [k E, (k+1) E), nodes [k N, (k+1) N), surface
                                  rows [k Ns, (k+1) Ns), material table entry mat[e] + k (1 +
                                  max mat)).  The members are set by ns_set_boundary (no
                                  ns_set_members); each solves its own CG.  Atomic scatter, no
                                  multigrid.  0 or 1: one model */
  int32_t local_gather;        /* 1: the FP32 inner operator (one model, atomic scatter) gathers each
                                  block's distinct nodes into shared memory once and adds its forces
                                  there before one global atomic per node (node lists built at
                                  ns_upload_mesh; skipped when a block's list exceeds 1,536 nodes);
                                  0: per-element gathers and atomics */
} ns_config;

#define NS_STREAM_RING 0
#define NS_STREAM_ZERO_COPY 1

/* Material of one element group (Sec. 2.1; parameters of the readings):
 * density, S/P wave speeds, spring reference strain (secant modulus G0/2),
 * maximum hysteretic damping of the Masing loops, Rayleigh damping ratio. */
typedef struct {
  double rho, vs, vp, gamma_ref, h_max, rayleigh_h;
} ns_material;

typedef struct {
  int64_t steps;              /* steps taken */
  int64_t cg_iters_total;     /* CG iterations summed over steps (outer for NS_PREC_FP64_IR) */
  int32_t cg_iters_last;      /* CG iterations of the last step */
  int32_t inner_iters_last;   /* inner FP32 iterations of the last step (NS_PREC_FP64_IR) */
  double relres_last;         /* final relative residual of the last step */
  int64_t kernel_launches;    /* this library's kernels launched since creation */
  int64_t h2d_bytes, d2h_bytes; /* state bytes streamed since creation */
  int64_t resident_elems, streamed_elems;
  /* CUDA-event times (ms, summed since the last ns_reset_stats), valid when timing = 1 */
  double ms_rhs, ms_jacobi, ms_solve, ms_newmark, ms_springs, ms_step;
  int64_t n_ebe64, n_ebe32, n_spring;  /* launches of the FP64 operator, FP32 operator, spring kernel */
  double ms_ebe64, ms_ebe32, ms_spring; /* their summed durations */
  double ms_stream_wall;      /* multi-spring phase with a streamed part: its start to the last D2H */
  double ms_advance;          /* CUDA-event time of ns_advance calls, all streams joined (always valid) */
  int64_t h2d_bytes_early;    /* of h2d_bytes: chunks loaded at the start of a step, before its
                                 multi-spring phase (they overlap the solve) */
  int64_t inner_iters_total;  /* inner FP32 iterations summed since the last ns_reset_stats: the
                                 FP32 operator launches that did work (the others return at once) */
  /* spring-update counts since the last ns_reset_stats (read when ns_advance returns) */
  int64_t spring_moved;       /* springs whose strain changed (the others keep their state) */
  int64_t spring_reversals;   /* of those, springs that reversed direction (Masing branch start) */
  int64_t spring_fp64_roots;  /* springs whose skeleton root left the double-float fast path for the
                                 FP64 one (seed not converged, step too large, argument out of range) */
  int64_t coarse_iters_total; /* multigrid: coarse PCG iterations since the last ns_reset_stats */
} ns_stats;

/* Fill cfg with defaults: 10 springs, dt 0.01, tol 1e-8, 10000 iterations,
 * x0_prev 1, NS_PREC_FP64, NS_SCATTER_ATOMIC, chunk 100000 elements (Sec. 2.3),
 * ring 3, all state resident, Rayleigh 0.1/2.5 Hz, 64 surface steps,
 * device 0, timing 0, inner 45 iterations / 1e-4, waits 120 s, graphs on,
 * FP32 inner operator staged per warp (stage_elements -1), L2 prefetch on, FP64
 * operator (no pair arithmetic),
 * NS_STREAM_RING, spring launch shape from the size heuristic (tile 0) with the
 * 64-register budget (4 blocks), tangent assembly off the tensor cores. */
void ns_config_default(ns_config *cfg);

/* Create a context on cfg->device.  *ctx is set on success. */
int ns_create(ns_ctx **ctx, const ns_config *cfg);

/* Upload the mesh: xyz [n_nodes][3], conn [n_elems][10] (order above), mat
 * [n_elems] material indices.  Checks indices, positive volumes and straight
 * edges (NS_ERR_BAD_MESH).  Builds the per-element geometry on the device and,
 * for NS_SCATTER_COLOUR, the greedy element colouring.  Once per context. */
int ns_upload_mesh(ns_ctx *ctx, int64_t n_nodes, const double *xyz, int64_t n_elems, const int32_t *conn,
                   const int32_t *mat);

/* Material table, n >= 1 entries (indices used by mat[] must be < n).
 * After the mesh: allocates the spring state (virgin springs) and sets the
 * initial tangent D to the elastic one. */
int ns_set_materials(ns_ctx *ctx, int32_t n, const ns_material *mats);

/* Absorbing faces (Sec. 2.1: semi-infinite bottom and sides, Lysmer dashpots):
 * faces [n_faces][6] = three vertices then edge nodes (0,1) (1,2) (0,2);
 * face_elem [n_faces] owning element (material); face_kind [n_faces] 0 =
 * bottom (the input motion enters here), 1 = side.  surf_nodes [n_surf] are
 * the nodes whose response ns_read_surface returns.  n_faces may be 0. */
int ns_set_boundary(ns_ctx *ctx, int64_t n_faces, const int32_t *faces, const int32_t *face_elem,
                    const int32_t *face_kind, int64_t n_surf, const int32_t *surf_nodes);

/* Outcrop (2E) input acceleration acc [n_samples][3] at t = k*dt, k = 0..;
 * dt must equal the context's dt.  The input velocity is its trapezoidal
 * integral from zero; beyond the last sample the acceleration is zero.
 * May be called again to replace the record (steps already taken stay). */
int ns_set_ground_motion(ns_ctx *ctx, int64_t n_samples, double dt, const double *acc);

/* Batched ensemble (many cases of the method advanced together; Sec. 2.3 runs many
 * cases, and Table 1's throughput is per case).  Declares that the uploaded mesh is the
 * disjoint union of M independent members: member m owns elements
 * [elem_off[m], elem_off[m+1]) and nodes [node_off[m], node_off[m+1]) (elem_off[0] =
 * node_off[0] = 0, elem_off[M] = n_elems, node_off[M] = n_nodes, every range non-empty);
 * no element may use a node of another member (NS_ERR_BAD_MESH) and the boundary faces
 * must be ordered by member.  Members take their materials through their elements'
 * material ids (one table for all), their input from ns_set_member_ground_motion, and
 * each solves its own CG (own scalars, converged against its own ||b||); every kernel
 * launch of a step covers all members.  Call after ns_upload_mesh and ns_set_boundary and
 * before ns_set_ground_motion, once; needs NS_SCATTER_ATOMIC.  Arrays are copied. */
int ns_set_members(ns_ctx *ctx, int32_t M, const int64_t *elem_off, const int64_t *node_off);

/* Input acceleration of one member (same layout, dt and number of samples as the
 * record given to ns_set_ground_motion, which every member starts with). */
int ns_set_member_ground_motion(ns_ctx *ctx, int32_t member, int64_t n_samples, double dt, const double *acc);

/* Springs per point of each member (S [M], each >= 5), for a batch whose members are
 * different cases of the method (served requests differ in S).  Call after ns_set_members
 * and before the first step, once; all spring state resident (device_state_budget < 0).
 * Each member gets its own spring set (the multi-spring geometry of its S, Sec. 2.1) and
 * its spring update is launched over its own points.  The spring state of such a context
 * is not readable or writable through ns_read_state / ns_write_state, and it has no
 * checkpoint or autotuner; tangents and node vectors are as usual. */
int ns_set_member_springs(ns_ctx *ctx, int32_t M, const int32_t *S);

/* Outer CG iterations of each member at the last step into iters[M] (M = the context's
 * member count, 1 without ns_set_members). */
int ns_get_member_iters(ns_ctx *ctx, int32_t M, int32_t *iters);

/* Advance nsteps time steps.  Returns after the device work of all steps is
 * complete.  On NS_ERR_NOT_CONVERGED the failing step is not applied and
 * ns_get_stats().steps tells how many steps were taken. */
int ns_advance(ns_ctx *ctx, int64_t nsteps);

/* Surface response of steps [step0, step0 + nsteps) (1-based step numbers of
 * states t = step*dt) into u, v, a, each [nsteps][n_surf][3]; NULL skips a
 * field.  Only the last surface_ring_steps steps are available. */
int ns_read_surface(ns_ctx *ctx, int64_t step0, int64_t nsteps, double *u, double *v, double *a);

/* Spring state and tangent of elements [elem0, elem0 + n): theta
 * [n][4][n_springs] records of 40 bytes {double tau, gR, tR, gmax; int32 dir,
 * mode} (may be NULL), D [n][4][36] (may be NULL). */
int ns_read_state(ns_ctx *ctx, int64_t elem0, int64_t n, void *theta, double *D);

/* Overwrite the state of elements [elem0, elem0 + n) (same layouts; NULL skips). */
int ns_write_state(ns_ctx *ctx, int64_t elem0, int64_t n, const void *theta, const double *D);

#define NS_FIELD_U 0
#define NS_FIELD_V 1
#define NS_FIELD_A 2
#define NS_FIELD_Q 3
#define NS_FIELD_DU 4
/* Read / overwrite one node vector [n_nodes][3]. */
int ns_read_nodal(ns_ctx *ctx, int32_t field, double *out);
int ns_write_nodal(ns_ctx *ctx, int32_t field, const double *in);

#define NS_OP_K 0  /* K(D) */
#define NS_OP_M 1  /* consistent mass */
#define NS_OP_CB 2 /* boundary dashpots */
#define NS_OP_A 3  /* 4/dt^2 M + 2/dt (Rayleigh(K) + C_b) + K, the matrix of Eq. 1 */
#define NS_OP_CR 4 /* Rayleigh part alpha M + beta K */
/* y = Op x with the current tangent D, x and y [n_nodes][3] host buffers
 * (FP64 element-by-element operator on the device). */
int ns_apply_operator(ns_ctx *ctx, int32_t op, const double *x, double *y);

/* Multi-spring update of npts free-standing integration points on the device:
 * mat [npts], eps and deps [npts][6] (total strain and increment), theta
 * [npts][n_springs] 40-byte records updated in place, D [npts][36] out. */
int ns_spring_points(ns_ctx *ctx, int64_t npts, const int32_t *mat, const double *eps, const double *deps,
                     void *theta, double *D);

/* Coarse operator of the two-level preconditioner (cfg.multigrid): y_c = Op_c x_c with the
 * linear-element model on the mesh vertices (Sec. 2.2; the coarse level of [SC14]), op one of
 * NS_OP_K, NS_OP_M, NS_OP_CB, NS_OP_A, with the current tangent (its four-point mean per
 * element); x_c and y_c [n_coarse][3] host buffers (FP32 arithmetic on the device, the
 * inner solve's precision).  n_coarse must be the context's coarse node count. */
int ns_apply_coarse_operator(ns_ctx *ctx, int32_t op, int64_t n_coarse, const double *xc, double *yc);

/* Allocation-free ns_spring_points (no counterpart in the paper).  For callers that
 * must not allocate device memory at the point of the call -- e.g. a host application
 * that commits a fixed device-memory budget at start-up and forbids later allocation, or
 * threads that must not take the CUDA allocator's locks -- the device staging buffers
 * live in one file-scope device array of 8 MiB that the library reserves on every GPU
 * that loads it (kept until the process exits).  Same arguments, layouts and results
 * as ns_spring_points; no cudaMalloc/cudaFree or other allocating call is made.
 *  - npts may be at most ns_spring_points_noalloc_capacity(n_springs) (more points:
 *    NS_ERR_INVALID_ARG with a message giving the limit).
 *  - The first call on a device resolves the array's device address (once per device,
 *    with that device current); make that first call before any stream capture.
 *  - All calls share the array; each call writes every byte it reads, so nothing of a
 *    previous call is reused, but calls that overlap on the GPU (several host threads or
 *    contexts on one device) race on it and must be serialised by the caller.
 *  - The call works on the context's device and makes the caller's current device
 *    current again before it returns. */
int ns_spring_points_noalloc(ns_ctx *ctx, int64_t npts, const int32_t *mat, const double *eps, const double *deps,
                             void *theta, double *D);

/* Largest npts ns_spring_points_noalloc accepts at S springs per point. */
int64_t ns_spring_points_noalloc_capacity(int32_t S);

int ns_get_stats(ns_ctx *ctx, ns_stats *st);
int ns_reset_stats(ns_ctx *ctx);

/* Result of ns_autotune: the candidates it timed and what it chose. */
typedef struct {
  int32_t n_tile;                 /* spring-kernel launch shapes tried */
  int32_t tile_points[16];        /* integration points per block of each */
  int32_t tile_blocks[16];        /* its register budget: resident blocks per SM it was compiled
                                     for (1: the compiler's choice, 4: 64 registers a thread) */
  float tile_ms[16];              /* spring kernel time of each on the sample (ms) */
  int32_t chosen_tile_points;
  int32_t chosen_tile_blocks;
  int32_t n_chunk;                /* streamed-state chunk sizes tried (0: no streamed state) */
  int64_t chunk_elems[6];
  float chunk_gbps[6];            /* H2D + D2H bytes per second of each over the ring */
  int64_t chosen_chunk_elems;
} ns_tuning;

/* Autotuner (a tool of this library; the paper tunes nothing at run time): times the
 * spring kernel's launch shape (integration points per block, and one of two register
 * budgets it is compiled with) in one launch over a sample of up to 131,072 resident
 * elements (eight slices spread over the model) -- a copy of their spring state moved one
 * more increment along the last step's (strain eps + deps, increment deps), so that every
 * spring takes a root solve of a step's size -- and the streamed state's chunk size (a copy round trip through the ring buffers, which leaves
 * the host state as it was), and keeps the fastest of each for the following steps.
 * The simulation's state and results are unchanged (the block shape does not change the
 * order of any sum).  Call between ns_advance calls, after at least one step (the strains
 * of a step make the spring timings representative).  Allocates a temporary copy of the
 * sampled state. */
int ns_autotune(ns_ctx *ctx, ns_tuning *out);

/* Autotuner on the simulation's own steps: advances nsteps steps (at least one per
 * candidate launch shape: 4, 8, 16, 24, 32, 64 and 128 points per block, each with the two
 * register budgets, as many as fit the spring count -- 14 at 150 springs), each step's spring kernel with the
 * next candidate shape, timed with CUDA events; keeps the fastest for the following steps.
 * The steps are the simulation's ordinary steps -- the launch shape changes the order of no
 * sum, so the results are those of ns_advance(ctx, nsteps) -- and the timings are of the
 * actual workload (a sample moved by an extrapolated increment, as ns_autotune times,
 * measured smaller tiles faster than they run in the step).  out: the shapes and each
 * one's best spring-kernel time (ms); chunk fields zero.  Errors: NS_ERR_INVALID_ARG if
 * nsteps is below the candidate count, ns_advance's codes (the shape in use before the
 * call is kept). */
int ns_autotune_steps(ns_ctx *ctx, int32_t nsteps, ns_tuning *out);

/* Checkpoint of the whole time-stepping state (step counter, u, v, a, q, du,
 * D, spring state).  ns_checkpoint_size gives the byte count; the buffers are
 * caller-owned host memory of at least that size. */
int ns_checkpoint_size(ns_ctx *ctx, int64_t *bytes);
int ns_checkpoint(ns_ctx *ctx, void *buf, int64_t bytes);
int ns_restore(ns_ctx *ctx, const void *buf, int64_t bytes);

void ns_destroy(ns_ctx *ctx);
const char *ns_last_error(ns_ctx *ctx);

/* ---- host-only helpers (no device work) ---------------------------------- */

/* Spring directions q [S][6] and weight w of the multi-spring geometry:
 * hemispherical Fibonacci plane normals, slip directions rotated by 2 pi
 * frac(k sqrt2), shear projections made exactly isotropic so that
 * w sum_k q_k q_k^T = diag(2,2,2,1,1,1) - (2/3) m m^T with w = 5/(2S). */
int ns_spring_directions(int32_t S, double *q, double *w);

/* Greedy first-fit element colouring in element order (elements sharing a
 * node get different colours).  colour [n_elems]; *n_colours out. */
int ns_colour_elements(int64_t n_elems, int64_t n_nodes, const int32_t *conn, int32_t *colour,
                       int32_t *n_colours);

/* Coarse level of the two-level preconditioner (Sec. 2.2): cid [n_nodes] receives the coarse
 * index of each vertex node (vertices numbered in ascending node order) or -1 for an edge
 * node; par [n_nodes][2] the two coarse nodes that interpolate each node (a vertex twice, an
 * edge node its edge's end vertices, smaller first); *n_coarse the coarse node count.
 * NS_ERR_BAD_MESH if a node is a vertex in one element and an edge node in another, or an
 * edge node sits on two different edges. */
int ns_coarse_map(int64_t n_elems, int64_t n_nodes, const int32_t *conn, int32_t *cid, int32_t *par,
                  int64_t *n_coarse);

/* Bytes of spring state for n_elems elements with S springs per point
 * (4 points per element, 40 bytes per spring). */
int64_t ns_state_bytes(int64_t n_elems, int32_t S);

#ifdef __cplusplus
}
#endif
#endif
