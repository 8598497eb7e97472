// Internal declarations of the GB300 time stepper (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ns.h"
#include "df64.cuh"

namespace ns {

constexpr int kQ = 4;          // integration points per element
constexpr int kDPack = 21;     // unique entries of a symmetric 6x6
constexpr int kMaxMat = 1024;  // material table entries (members of a batch each bring their own)
constexpr int kBlock = 256;
constexpr int kSpringCountSlots = 64;  // spread of the spring kernel's counter atomics
constexpr int kLocalMaxNodes = 1536;   // largest node list of a locally gathered operator block

// Per-material constants derived on the host from ns_material and the config.
struct MatConst {
  double rho, vs, vp, G0, Kb, gref, alpha_ro, beta_ro, ray_a, ray_b;
  // spring-law constants: 1/G0, 1/(G0 gamma_ref), alpha (1 + beta), alpha (1 + beta) beta,
  // series coefficients beta (beta - 1)/2 and beta (beta - 1)(beta - 2)/6, FP32 copies
  double iG0, itref, ab1, ab1b, c2, c3, hab1b;
  float itref_f, iG0_f, alpha_f, beta_f, G0_f;
  float pad_f;
  RoPairs rp;       // the same constants as float pairs for the double-float root step
  // tangent assembly on tensor cores: 2^eG > G0 (eG = floor(log2 G0) + 1), gfix = 2^(49 - eG)
  // turns a tangent into a 49-bit integer, dsc = 2^eG scales the digit sums back (with the
  // column scales of the spring tables)
  float gfix;
  int32_t eg;
  double dsc;
};

// Coefficients of one element-by-element operator application, per material:
//   y_e = mM[m] * M_e xm + mK[m] * M_e xk + kK[m] * K_e xk
struct OpCoef {
  double mM[kMaxMat];
  double mK[kMaxMat];
  double kK[kMaxMat];
};

// Device mesh in structure-of-arrays form (element arrays have stride epad).
struct DevMesh {
  int64_t N = 0, E = 0, epad = 0, F = 0, fpad = 0, Ns = 0;
  int32_t *conn = nullptr;   // [10][epg]
  double *geom = nullptr;    // [10][epg]: grad L1 (3), grad L2 (3), grad L3 (3), volume
  float *geom32 = nullptr;   // [10][epg]
  int32_t *mat = nullptr;    // [epad]
  int32_t *fnode = nullptr;  // [6][fpg]
  double *fgeom = nullptr;   // [4][fpg]: area, unit normal
  int32_t *fmat = nullptr;   // [F]
  int32_t *fkind = nullptr;  // [Fb]
  int32_t *surf = nullptr;   // [Ns]
  // colour mode: element and face ids sorted by colour
  int32_t *ecol_ids = nullptr, *fcol_ids = nullptr;
  std::vector<int64_t> ecol_off, fcol_off;
  int32_t *kerr = nullptr;  // device flag: a bounded wait inside a kernel gave up
  dd *geom2 = nullptr;      // [10][epg] geometry as float pairs (double-float operator)
  int prefetch = 0;         // element kernels prefetch their blocks' element rows into L2
  // Members sharing one mesh (shared_members > 1): E, N, F and Ns count every member's
  // elements, nodes, faces and surface nodes (member after member), while the connectivity,
  // geometry, face nodes, face geometry and face kinds hold one copy of the shared mesh
  // (Eb elements, Nb nodes, Fb faces; rows of stride epg and fpg).  Element data (material,
  // tangent, state) and node vectors stay per member.  Without sharing Eb = E, Nb = N,
  // Fb = F, epg = epad, fpg = fpad.
  int32_t Msh = 1;
  int64_t Eb = 0, Nb = 0, Fb = 0, epg = 0, fpg = 0;
  // Local gathering of the FP32 inner operator (one model, atomic scatter): block b of
  // kBlock consecutive elements gathers its distinct nodes lnode[loff[b] .. loff[b+1])
  // (ascending) once into shared memory; lconn [10][epg] holds each element's nodes as
  // indices into its block's list.  lmax: the largest list (0: not built).
  uint16_t *lconn = nullptr;
  int32_t *lnode = nullptr;
  int64_t *loff = nullptr;
  int32_t lmax = 0;
  // members' element launch cuts all start at a multiple of 32 elements (the per-warp
  // staged FP32 operator can take them)
  bool eseg32 = false;
  // element offset argument of the kernels: 0 without sharing
  int64_t eb_arg() const { return Msh > 1 ? Eb : 0; }
  int64_t fb_arg() const { return Msh > 1 ? Fb : 0; }
};

// Spring state arrays (structure of arrays over springs ordered [elem][point][spring]).
struct SpringSoA {
  double *tau = nullptr, *gR = nullptr, *tR = nullptr, *gmax = nullptr;
  int32_t *dir = nullptr, *mode = nullptr;
};

struct CgScalars {
  double bb, rr, rz, rz_old, pAp, alpha, beta;
  double rr0;
  int32_t iters, done, status, pad;
  unsigned int counter;
  unsigned int counter2;
};
// int32 stride between the `done` flags of consecutive members' scalars
constexpr int kScStride = (int)(sizeof(CgScalars) / sizeof(int32_t));
static_assert(sizeof(CgScalars) % sizeof(int32_t) == 0, "CgScalars must be a whole number of int32");

// Batched members (independent sub-models of one disjoint-union mesh): a launch over
// elements, faces or nodes is cut into blocks that never straddle two members.  Block b
// covers indices [a0, a1) of member m; its partial sums land in slot b, and the
// partial sums of member m are the slots [off[m], off[m+1]) of that launch.
struct Seg {
  int64_t a0, a1;
  int32_t m, pad;
};
struct SegList {
  const Seg *seg = nullptr;  // nullptr: one member, the historical flat launch
  int n = 0;                 // blocks
  const int32_t *off = nullptr;  // [M + 1] block offsets per member (device)
};
// Which partial sums make up member m's value: slots [off1[m], off1[m+1]) and, when off2
// is set, base2 + [off2[m], off2[m+1]).  off1 == nullptr: one member, all n slots.
struct PartMap {
  const int32_t *off1 = nullptr;
  const int32_t *off2 = nullptr;
  int32_t base2 = 0;
};

// Coarse level of the two-level preconditioner (linear tetrahedra on the vertices).
struct MgLevel {
  int64_t Nc = 0;
  int32_t *conn1 = nullptr;   // [4][epad] coarse index of each element vertex
  int32_t *cfnode = nullptr;  // [3][fpad] coarse index of each boundary-face vertex
  int64_t *rptr = nullptr;    // [Nc + 1] restriction lists
  int32_t *rlist = nullptr;   // fine nodes gathered into each coarse node: n (weight 1) or ~n (edge, 1/2)
  int2 *par = nullptr;        // [N] the two coarse nodes that interpolate each fine node
  float *Dbar = nullptr;      // [21][epad] mean of the element's four point tangents
  float *Jd32 = nullptr, *Jinv32 = nullptr;  // [Nc][6] coarse diagonal blocks and their inverses
  float *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *Ap = nullptr;  // coarse PCG [Nc][4]
};

// ------------------------------------------------------------------ launchers (k_*.cu)
// All return cudaGetLastError() of their launch.
cudaError_t launch_geometry(const DevMesh &m, const double *xyz, int32_t *bad, cudaStream_t s);
cudaError_t launch_face_geometry(const DevMesh &m, const double *xyz, cudaStream_t s);

// y (+)= Op x over elements [e0, e1) or over the colour list ids[e0, e1) when ids != nullptr.
// xm may be nullptr (then mM is ignored).  If dot != nullptr, block partial sums of x_e . y_e go
// to dot[blockIdx.x] (the element-local energy of the application).
// With sg.seg set (members, atomic scatter) the launch covers sg's blocks instead of
// [e0, e1), and the skip flag of each block is that of its member (skip + m * kScStride).
// D2 (optional): the tangent as float pairs [84][epad]; with it (and m.geom2) the operator
// runs in double-float arithmetic on the FP32 pipes (relative accuracy ~1e-13).
cudaError_t launch_ebe64(const DevMesh &m, const double *D, const OpCoef *op, const double *xm, const double *xk,
                         double *y, const int32_t *ids, int64_t e0, int64_t e1, bool atomic, double *dot,
                         const int32_t *skip, cudaStream_t s, SegList sg = {}, const void *D2 = nullptr,
                         double *yk = nullptr);
// (with dot and yk set: the stiffness part K x, without its coefficient, also goes to yk)
// dst[i] = src[i] as a float pair (n values)
cudaError_t launch_to_pairs(const double *src, void *dst, int64_t n, cudaStream_t s);
// stage (whole-mesh atomic launches of one member): 1 stages each tile of elements in shared
// memory with bulk copies (cp.async.bulk); 2 has each warp copy its elements' tangent rows
// asynchronously (cp.async) while it gathers x; 0 per-thread loads.
cudaError_t launch_ebe32(const DevMesh &m, const float *D, const OpCoef *op, const float *xk, float *y,
                         const int32_t *ids, int64_t e0, int64_t e1, bool atomic, double *dot, const int32_t *skip,
                         cudaStream_t s, SegList sg = {}, int stage = 0);
// As launch_ebe32 with D stored as FP16 pairs [42][epad] (entries 2j, 2j+1 of the [84] point-major
// order) holding D / G0 of the element's material; op->kK carries the factor G0.
cudaError_t launch_ebe16(const DevMesh &m, const void *D16, const OpCoef *op, const float *xk, float *y,
                         const int32_t *ids, int64_t e0, int64_t e1, bool atomic, double *dot, const int32_t *skip,
                         cudaStream_t s, SegList sg = {}, int stage = 0);
// Boundary faces: y (+)= cC * C_f (x + [kind 0] vin) (vin may be nullptr); with members the
// input of face f is vin + fmem[f] * vin_stride.
cudaError_t launch_faces64(const DevMesh &m, const MatConst *mc, double cC, const double *x, const double *vin,
                           double *y, const int32_t *ids, int64_t f0, int64_t f1, bool atomic, double *dot,
                           const int32_t *skip, cudaStream_t s, SegList sg = {}, const int32_t *fmem = nullptr,
                           int64_t vin_stride = 0);
cudaError_t launch_faces32(const DevMesh &m, const MatConst *mc, float cC, const float *x, float *y,
                           const int32_t *ids, int64_t f0, int64_t f1, bool atomic, double *dot, const int32_t *skip,
                           cudaStream_t s, SegList sg = {});
// 3x3 diagonal blocks of A (packed xx yy zz yz xz xy) accumulated into Jd [N][6]
cudaError_t launch_jacobi_elems(const DevMesh &m, const double *D, const OpCoef *op, double *Jd, const int32_t *ids,
                                int64_t e0, int64_t e1, bool atomic, cudaStream_t s);
cudaError_t launch_jacobi_faces(const DevMesh &m, const MatConst *mc, double cC, double *Jd, const int32_t *ids,
                                int64_t f0, int64_t f1, bool atomic, cudaStream_t s);
// FP32 variants (the preconditioner of the flexible solver only needs single precision)
cudaError_t launch_jacobi_elems32(const DevMesh &m, const float *D, const OpCoef *op, float *Jd, const int32_t *ids,
                                  int64_t e0, int64_t e1, bool atomic, cudaStream_t s);
// from the FP16 tangent pairs (op->kK carries G0, as for launch_ebe16)
cudaError_t launch_jacobi_elems16(const DevMesh &m, const void *D16, const OpCoef *op, float *Jd, const int32_t *ids,
                                  int64_t e0, int64_t e1, bool atomic, cudaStream_t s);
cudaError_t launch_jacobi_faces32(const DevMesh &m, const MatConst *mc, double cC, float *Jd, const int32_t *ids,
                                  int64_t f0, int64_t f1, bool atomic, cudaStream_t s);
cudaError_t launch_invert_blocks32(const float *Jd, float *Jinv32, int64_t N, int32_t *bad, cudaStream_t s);
// strains eps, deps at the 4 points of elements [e0, e1), computed in double-float
// arithmetic: out float2 [E][4][12] (eps 6, deps 6 per point)
cudaError_t launch_strain_pairs(const DevMesh &m, const double *u, const double *du, void *out, int64_t e0, int64_t e1,
                                cudaStream_t s);

// ------------------------------------------------------------------ k_mg.cu (two-level preconditioner)
cudaError_t launch_mg_dbar(const double *D, float *Dbar, int64_t epad, int64_t E, cudaStream_t s);
cudaError_t launch_mg_jacobi(const DevMesh &m, const MgLevel &c, const OpCoef *op, float *Jd, const int32_t *ids,
                             int64_t e0, int64_t e1, bool atomic, cudaStream_t s);
cudaError_t launch_mg_jacobi_faces(const DevMesh &m, const MgLevel &c, const MatConst *mc, float cC, float *Jd,
                                   const int32_t *ids, int64_t f0, int64_t f1, bool atomic, cudaStream_t s);
// y_c += (kK K1 + mK M1) x_c (coefficients per material from op); dot: block partials of x_e . y_e
cudaError_t launch_mg_ebe(const DevMesh &m, const MgLevel &c, const OpCoef *op, const float *x, float *y,
                          const int32_t *ids, int64_t e0, int64_t e1, bool atomic, double *dot, const int32_t *skip,
                          cudaStream_t s);
cudaError_t launch_mg_faces(const DevMesh &m, const MgLevel &c, const MatConst *mc, float cC, const float *x, float *y,
                            const int32_t *ids, int64_t f0, int64_t f1, bool atomic, double *dot, const int32_t *skip,
                            cudaStream_t s);
// r_c = P^T (r / ||r||) and the start of the coarse PCG (3 partial sets into part)
cudaError_t launch_mg_restrict_init(const double *r, const CgScalars *so, const MgLevel &c, float *rc, float *zc,
                                    float *pc, float *xc, float *Apc, double *part, cudaStream_t s);
// x_in = P x_c, Ap_in = 0
cudaError_t launch_mg_prolong(const MgLevel &c, const float *xc, float *xin, float *Apin, int64_t N,
                              const CgScalars *so, cudaStream_t s);
// start of the fine inner PCG from x_in (Ap_in holds A x_in): 3 partial sets into part
cudaError_t launch_mg_fine_init(const double *r, const CgScalars *so, const float *J, float *rin, float *zin,
                                float *pin, float *Apin, int64_t N, double *part, cudaStream_t s);

// ------------------------------------------------------------------ k_vec.cu
cudaError_t launch_fill(double *x, double v, int64_t n, cudaStream_t s);
cudaError_t launch_negate_copy(double *dst, const double *src, int64_t n, cudaStream_t s);
cudaError_t launch_invert_blocks(const double *Jd, double *Jinv, float *Jinv32, int64_t N, int32_t *bad,
                                 cudaStream_t s);
int vec_blocks(int64_t n_nodes);  // fixed grid of the node-vector kernels (partials per block)
// r = b - Ap; z = Jinv r; p = z; block partials of b.b, r.r, r.z -> part[0..3*nb)
cudaError_t launch_cg_init(const double *b, const double *Ap, const double *Jinv, double *r, double *z, double *p,
                           int64_t N, double *part, cudaStream_t s, SegList sg = {});
#define NS_FIN_INIT 0
#define NS_FIN_PAP 1
#define NS_FIN_UPDATE 2
#define NS_FIN_FCG_INIT 3
#define NS_FIN_FCG_BETA 4
#define NS_FIN_FCG_UPDATE 6
// One block sums part[v*n .. v*n+n) for v < nvals in a fixed order and updates the CG scalars:
//  INIT: bb, rr, rz -> done (1 converged, 2 zero right-hand side); PAP: pAp, alpha = rz/pAp;
//  UPDATE: rr, rz -> iters++, done (1 converged, 3 iteration limit), beta = rz/rz_old.
// With members (M > 1) one block per member, summing the slots that pm assigns to it, each
// member updating its own scalars sc[m].  A member whose gate[m].done is set is marked done
// without reading its partials (the inner solve of a member whose outer solve converged).
cudaError_t launch_cg_final(const double *part, int n, int nvals, CgScalars *sc, int mode, double tol, int max_iter,
                            cudaStream_t s, int M = 1, PartMap pm = {}, const CgScalars *gate = nullptr);
// x += alpha p; r -= alpha Ap; z = Jinv r; partials r.r, r.z -> part[0..2*nb)
cudaError_t launch_cg_update(double *x, double *r, double *z, const double *p, const double *Ap, const double *Jinv,
                             int64_t N, double *part, const CgScalars *sc, cudaStream_t s, SegList sg = {});
// p = z + beta p; Ap = 0
cudaError_t launch_cg_pupdate(double *p, const double *z, double *Ap, int64_t N, const CgScalars *sc, cudaStream_t s,
                              SegList sg = {});
// flexible outer CG (FP64) with the inner FP32 PCG as preconditioner
cudaError_t launch_fcg_init(const double *b, const double *Ap, double *r, int64_t N, double *part, cudaStream_t s,
                            SegList sg = {});
cudaError_t launch_fcg_gamma(const float *xin, double *z, const double *Ap, int64_t N, double *part,
                             const CgScalars *so, cudaStream_t s, SegList sg = {});
cudaError_t launch_fcg_p(double *p, const double *z, const double *r, double *Ap, double *Kp, int64_t N,
                         double *part, const CgScalars *so, cudaStream_t s, SegList sg = {});
// alpha = (p.r)/(p.Ap): pr holds vector partials (member m: pmr), pap operator partials (pma)
cudaError_t launch_fcg_alpha(const double *pr, int npr, const double *pap, int npap, CgScalars *sc, cudaStream_t s,
                             int M = 1, PartMap pmr = {}, PartMap pma = {});
// (q, Kp non-null: q += alpha Kp as well -- K du accumulated during a solve from zero)
cudaError_t launch_fcg_update(double *x, double *r, const double *p, const double *Ap, double *q, const double *Kp,
                              int64_t N, double *part, const CgScalars *so, cudaStream_t s, SegList sg = {});
cudaError_t launch_in_init(const double *r, const CgScalars *so, const float *J, float *rin, float *zin, float *pin,
                           float *xin, float *Apin, int64_t N, double *part, cudaStream_t s, SegList sg = {});
cudaError_t launch_in_update(float *xin, float *rin, float *zin, const float *pin, const float *Apin, const float *J,
                             int64_t N, double *part, const CgScalars *si, const CgScalars *so, cudaStream_t s,
                             SegList sg = {});
cudaError_t launch_in_pupdate(float *pin, const float *zin, float *Apin, int64_t N, const CgScalars *si,
                              const CgScalars *so, cudaStream_t s, SegList sg = {});
cudaError_t launch_newmark(double *u, double *v, double *a, double *du_prev, const double *du, int64_t N, double dt,
                           cudaStream_t s);
cudaError_t launch_surface_gather(const int32_t *surf, int64_t Ns, const double *u, const double *v, const double *a,
                                  double *ou, double *ov, double *oa, cudaStream_t s);
cudaError_t launch_d_to_f32(const double *src, float *dst, int64_t n, cudaStream_t s);
cudaError_t launch_dot_partials(const double *x, const double *y, int64_t n, double *part, cudaStream_t s);

// ------------------------------------------------------------------ k_spring.cu
struct SpringTables {
  const double *q;    // [S][6]
  const float2 *q2;   // [S][6] the same as (hi, lo) float pairs
  const double *T;    // [S][21] w q q^T packed upper triangle (+ one row with their sum)
  const float2 *T2;   // [S][21] the same entries as (hi, lo) float pairs
  const double *pow;  // power tables: r[128], -ln r hi[128], lo[128], 2^(i/64)[64], ln2 hi/lo, ln2/64 hi/lo
  const float *powf;  // double-float power tables (df64.cuh, kPowFLen floats)
  int S;
  const uint2 *tfrag = nullptr;  // digits of T in MMA fragment order (tensor-core assembly)
  const double *tsc = nullptr;   // [21] 2^(et[ij] - 12): column scales of those digits
  int tc = 1;         // 1: assemble D on the tensor cores where the launch shape allows
  int tp = 0;         // integration points per block of the spring kernel (0: size heuristic)
  int minb = 1;       // register budget of the spring kernel: 1 (compiler's choice) or 4 blocks per SM
  // counters [kSpringCountSlots][3]: springs moved, reversals, roots on the FP64 path (nullptr: none)
  unsigned long long *cnt = nullptr;
};
// the spring kernel's default points per block for S springs, and whether tp is usable
int spring_tile_default(int S);
bool spring_tile_ok(int tp, int S);
constexpr int kPowTabLen = 452;
// Spring update of points [p0, p1) (point p = elem*4 + qp), strains from eps [P][12]
// (FP64, or float pairs when eps_pairs: the layout launch_strain_pairs writes);
// state arrays indexed relative to `base` point; D written to D[(qp*21 + k) * epad + elem]
// (element layout) or, if dpts != nullptr, to dpts[p - p0][21] (free points).
cudaError_t launch_springs(const SpringTables &tab, const MatConst *mc, const int32_t *mat_of_elem,
                           const int32_t *mat_of_point, const double *eps, SpringSoA st, int64_t base, int64_t p0,
                           int64_t p1, double *D, int64_t epad, double *dpts, cudaStream_t s,
                           bool eps_pairs = false);
// The autotuner's spring sample: the strain pairs of elements [e0, e0 + ne) moved one
// increment on (eps + deps, deps) into eps_out from element out_elem on, and the elements'
// materials into mat_out from out_elem on.
cudaError_t launch_tune_sample(const double *eps_pairs, const int32_t *mat_e, int64_t e0, int64_t ne, float2 *eps_out,
                               int32_t *mat_out, int64_t out_elem, cudaStream_t s);
// elastic tangent for elements [e0, e1)
cudaError_t launch_elastic_D(const SpringTables &tab, const MatConst *mc, const int32_t *mat, double *D, int64_t epad,
                             int64_t e0, int64_t e1, cudaStream_t s);
cudaError_t launch_D_to_f32(const double *D, float *D32, int64_t epad, int64_t E, cudaStream_t s);
// D16[j][e] = half2(D[2j][e], D[2j+1][e]) / G0[mat[e]] for the FP16 inner operator
cudaError_t launch_D_to_f16(const double *D, const int32_t *mat, const MatConst *mc, void *D16, int64_t epad,
                            int64_t E, cudaStream_t s);

// ------------------------------------------------------------------ context views (ns_api.cu)
// What the allocation-free spring entry point needs from a context.
struct SpringCtxView {
  SpringTables tab;
  const MatConst *mats;
  int nmat;
  cudaStream_t stream;
  int device;
};
int ctx_spring_view(ns_ctx *c, SpringCtxView *v);  // NS_OK once materials are set
void ctx_set_error(ns_ctx *c, const char *msg);
void ctx_count_launches(ns_ctx *c, int n);
int ctx_sync_main(ns_ctx *c);                       // bounded wait for the context's main stream
// Served batches (ns_server.cpp).  Copy member ms of src into member md of dst, device to
// device: node vectors u, v, a, q, du, tangent D and spring state (same element, node and
// spring counts; a context without members counts as member 0).  All state resident.
int ctx_copy_member(ns_ctx *dst, int md, ns_ctx *src, int ms);
// Input velocity of member m at the context's steps k = 0 .. n-1 (vin [n][3]); later steps
// take vin[n-1].  Call after ns_set_ground_motion (which fixes the record length).
int ctx_set_member_velocity(ns_ctx *c, int m, const double *vin, int64_t n);
// device bytes the context holds (its own allocations)
int64_t ctx_steps(ns_ctx *c);
// Member ranges of a disjoint union built by the caller itself (every element's nodes in its
// member's range by construction): ns_set_members without reading the mesh back to check it.
int ctx_set_members_built(ns_ctx *c, int32_t M, const int64_t *elem_off, const int64_t *node_off);

// ------------------------------------------------------------------ ns_host.cpp
int host_spring_directions(int S, double *q, double *w);
int host_colouring(int64_t E, int64_t N, const int32_t *conn, int32_t *colour, int32_t *nc);
// coarse (vertex) numbering and interpolation parents of every node; returns the coarse count or -1
int64_t host_coarse_map(int64_t E, int64_t N, const int32_t *conn, int32_t *cid, int32_t *par);
void host_material_constants(const ns_material &m, double f1, double f2, MatConst *out);
// outcrop input velocity: the trapezoidal integral of acc [n][3] from v(0) = 0, with one
// entry past the record (zero acceleration there): out [n + 1][3]
void host_input_velocity(const double *acc, int64_t n, double dt, double *out);
void host_pow_tables(double *out);   // kPowTabLen entries
void host_powf_tables(float *out);   // kPowFLen entries (df64.cuh)
// per-column exponents et[21] of the spring tables T [S][21] (max_k |T_k[ij]| 2^-et[ij] in
// [1/4, 1/2)) and their 7-bit digits in MMA fragment order, 7 x ceil(S/16) x 3 x 32 entries
// (k_spring.cu)
void host_spring_digits(int S, const double *T, uint2 *frag, int *et);

}  // namespace ns
