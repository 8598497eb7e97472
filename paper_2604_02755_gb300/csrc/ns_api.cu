// C ABI and runtime of the GB300 time stepper: context, uploads, the per-step
// driver (right-hand side, block-Jacobi set-up, PCG, Newmark update, multi-spring
// update with the host<->HBM state stream of Alg. 3), read-back and checkpoints.
#include <math.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include "kern_common.cuh"
#include "ns_internal.h"

using namespace ns;

namespace {

struct EventTimer {
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, int>> pending;  // (kind, first event index)
  size_t used = 0;
  cudaEvent_t get() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  void reset() {
    used = 0;
    pending.clear();
  }
  ~EventTimer() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

enum TimeKind { TK_RHS, TK_JAC, TK_SOLVE, TK_NEWMARK, TK_SPRINGS, TK_STEP, TK_EBE64, TK_EBE32, TK_SPRING, TK_N };

}  // namespace

struct ns_ctx {
  ns_config cfg{};
  std::string err;
  cudaStream_t s_main = nullptr, s_h2d = nullptr, s_d2h = nullptr;
  DevMesh m;
  double *xyz_d = nullptr;
  bool has_mesh = false, has_mat = false, has_bnd = false, has_motion = false;
  int nmat = 0;
  std::vector<MatConst> mats_h;
  MatConst *mats_d = nullptr;
  OpCoef *op_A = nullptr, *op_K = nullptr, *op_M = nullptr, *op_Cr = nullptr, *op_rhs = nullptr;
  double *q_d = nullptr, *T_d = nullptr, *pow_d = nullptr;
  float2 *q2_d = nullptr;
  float *powf_d = nullptr;
  float2 *T2_d = nullptr;
  uint2 *tfrag_d = nullptr;
  double *tsc_d = nullptr;
  SpringTables tab{};
  double *D = nullptr;
  float *D32 = nullptr;   // NS_PREC_FP64_IR: FP32 copy of D for the inner operator
  __half *D16 = nullptr;  // NS_PREC_FP64_IR16: FP16 pairs of D / G0
  dd *D2 = nullptr;       // pair_operator: D as float pairs, refreshed at the start of each step
  OpCoef *op_A16 = nullptr;  // op_A with kK scaled by G0 (reads D16)
  // spring state: resident elements [0, E_res) on the device, [E_res, E) in pinned host memory
  int64_t E_res = 0;
  SpringSoA st;                      // device, resident part
  SpringSoA hst;                     // pinned host, streamed part
  SpringSoA hst_dev;                 // the same arrays' device addresses (zero-copy mode)
  std::vector<SpringSoA> ring;       // device chunk buffers
  cudaEvent_t *ev_h2d = nullptr, *ev_comp = nullptr, *ev_d2h = nullptr;
  cudaEvent_t ev_d2h_all = nullptr, ev_stream_t0 = nullptr, ev_stream_t1 = nullptr, ev_strain = nullptr;
  bool prefetched = false;
  // node vectors
  double *u = nullptr, *v = nullptr, *a = nullptr, *q = nullptr, *du = nullptr, *b = nullptr, *r = nullptr,
         *z = nullptr, *p = nullptr, *Ap = nullptr, *Jd = nullptr, *Jinv = nullptr;
  float *Jinv32 = nullptr;
  float *rin = nullptr, *zin = nullptr, *pin = nullptr, *xin = nullptr, *Apin = nullptr;  // inner FP32 PCG
  CgScalars *sc_in = nullptr;
  // two-level preconditioner (cfg.multigrid): coarse level, its PCG scalars, coarse index of
  // every node (host, for the boundary faces)
  MgLevel mg;
  CgScalars *sc_c = nullptr;
  int32_t shared_nmat = 1;  // shared members: material-table entries per member
  // members with their own springs per point (ns_set_member_springs): per member the springs,
  // the first spring of its state, its spring tables and the device arrays behind them
  std::vector<int32_t> mS;
  std::vector<int64_t> spr_off;
  std::vector<SpringTables> mtab;
  std::vector<void *> mtab_mem;
  // their spring launches are spread over these streams (forked from and joined to the main one)
  static constexpr int kMemberStreams = 4;
  cudaStream_t s_mem[kMemberStreams] = {};
  cudaEvent_t ev_fork = nullptr, ev_mem[kMemberStreams] = {};
  std::vector<int32_t> cid_h;
  double *eps = nullptr;
  double *part = nullptr;
  int64_t part_pap_cap = 0;
  CgScalars *sc = nullptr, *sc_h = nullptr;
  int32_t *flag_d = nullptr, *flag_h = nullptr;
  double *vin_d = nullptr;
  int64_t n_vin = 0;
  double *surf_u = nullptr, *surf_v = nullptr, *surf_a = nullptr;
  int64_t ring_steps = 0;
  int64_t step = 0;
  cudaEvent_t ev_sync = nullptr, ev_adv0 = nullptr, ev_adv1 = nullptr, ev_join = nullptr;
  // batched members (ns_set_members): M independent sub-models of the uploaded mesh
  int32_t M = 1;
  std::vector<int64_t> moff_e, moff_n, moff_f;  // [M + 1] element / node / face ranges
  Seg *vseg_d = nullptr, *eseg_d = nullptr, *fseg_d = nullptr;
  int32_t *voff_d = nullptr, *eoff_d = nullptr, *foff_d = nullptr, *fmem_d = nullptr;
  int nvseg = 0, neseg = 0, nfseg = 0;
  std::vector<int32_t> member_iters;  // outer CG iterations of each member at the last step
  std::vector<int32_t> face_elem_h;   // element of each boundary face (host copy)
  // captured launch sequences (cfg.graphs): one outer flexible-CG iteration, one batch of
  // plain CG iterations; with the launches and FP32 operator applications each contains
  bool capturing = false;
  cudaGraphExec_t g_outer = nullptr, g_batch = nullptr;
  int64_t g_outer_cnt[3] = {0, 0, 0}, g_batch_cnt[3] = {0, 0, 0};
  int64_t cap_ebe32 = 0, cap_ebe64 = 0;
  ns_stats stats{};
  // fault injection (cfg.fault_*): pinned allocations and state-stream copies made so far
  int64_t n_pinned_allocs = 0, n_state_copies = 0;
  // spring-update counters [kSpringCountSlots][3] (moved, reversals, FP64 roots), summed by
  // the spring kernel since the last ns_reset_stats
  unsigned long long *spr_cnt = nullptr;
  EventTimer timer;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> tev;
};

#define NS_SET(ctx, code, msg) \
  do {                         \
    (ctx)->err = (msg);        \
    return (code);             \
  } while (0)

#define CKC(ctx, call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                     \
      return (e_ == cudaErrorMemoryAllocation) ? NS_ERR_OOM_DEVICE : NS_ERR_CUDA;          \
    }                                                                                      \
  } while (0)

#define LAUNCH(ctx, call)                                                    \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    (ctx)->stats.kernel_launches++;                                          \
    if (e_ != cudaSuccess) {                                                 \
      (ctx)->err = std::string("launch ") + #call + ": " + cudaGetErrorString(e_); \
      return NS_ERR_CUDA;                                                    \
    }                                                                        \
  } while (0)

namespace {

template <typename T>
int dalloc(ns_ctx *c, T **p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->err = "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed: " + cudaGetErrorString(e);
    return NS_ERR_OOM_DEVICE;
  }
  return NS_OK;
}

template <typename T>
void dfree(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <typename T>
int halloc(ns_ctx *c, T **p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  if (++c->n_pinned_allocs == c->cfg.fault_pinned_alloc) {
    c->err = "cudaHostAlloc of " + std::to_string(n * sizeof(T)) + " bytes failed (injected fault: pinned allocation " +
             std::to_string(c->n_pinned_allocs) + ")";
    return NS_ERR_OOM_PINNED;
  }
  cudaError_t e = cudaHostAlloc((void **)p, n * sizeof(T), cudaHostAllocDefault);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->err = "cudaHostAlloc of " + std::to_string(n * sizeof(T)) + " bytes failed: " + cudaGetErrorString(e);
    return NS_ERR_OOM_PINNED;
  }
  return NS_OK;
}

template <typename T>
void hfree(T *&p) {
  if (p) cudaFreeHost(p);
  p = nullptr;
}

int64_t pad64(int64_t n) { return ((n + 63) / 64) * 64; }

// Bounded wait: poll the event until it completes or the deadline passes.
int wait_event(ns_ctx *c, cudaEvent_t ev) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return NS_OK;
    if (e != cudaErrorNotReady) {
      c->err = std::string("device error: ") + cudaGetErrorString(e);
      return NS_ERR_CUDA;
    }
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > c->cfg.wait_timeout_s) {
      c->err = "timed out waiting for the device";
      return NS_ERR_TIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

int sync_stream(ns_ctx *c, cudaStream_t s) {
  CKC(c, cudaEventRecord(c->ev_sync, s));
  return wait_event(c, c->ev_sync);
}

int sync_all(ns_ctx *c) {
  int rc;
  if ((rc = sync_stream(c, c->s_main)) != NS_OK) return rc;
  if ((rc = sync_stream(c, c->s_h2d)) != NS_OK) return rc;
  return sync_stream(c, c->s_d2h);
}

void tbegin(ns_ctx *c, int kind, cudaStream_t s, cudaEvent_t *out) {
  if (kind == TK_EBE32 && c->capturing) c->cap_ebe32++;
  if (kind == TK_EBE64 && c->capturing) c->cap_ebe64++;
  if (!c->cfg.timing || c->capturing) return;
  *out = c->timer.get();
  cudaEventRecord(*out, s);
}

void tend(ns_ctx *c, int kind, cudaStream_t s, cudaEvent_t start) {
  if (!c->cfg.timing || c->capturing) return;
  cudaEvent_t e = c->timer.get();
  cudaEventRecord(e, s);
  c->tev.push_back({kind, {start, e}});
}

void flush_times(ns_ctx *c) {
  for (auto &t : c->tev) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, t.second.first, t.second.second) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    switch (t.first) {
      case TK_RHS: c->stats.ms_rhs += ms; break;
      case TK_JAC: c->stats.ms_jacobi += ms; break;
      case TK_SOLVE: c->stats.ms_solve += ms; break;
      case TK_NEWMARK: c->stats.ms_newmark += ms; break;
      case TK_SPRINGS: c->stats.ms_springs += ms; break;
      case TK_STEP: c->stats.ms_step += ms; break;
      case TK_EBE64: c->stats.ms_ebe64 += ms; c->stats.n_ebe64++; break;
      case TK_EBE32: c->stats.ms_ebe32 += ms; c->stats.n_ebe32++; break;
      case TK_SPRING: c->stats.ms_spring += ms; c->stats.n_spring++; break;
      default: break;
    }
  }
  c->tev.clear();
}

int nblk(int64_t n) { return (int)((n + kBlock - 1) / kBlock); }

// Launch cuts by member (empty lists with one member: the flat launches)
SegList vsegs(const ns_ctx *c) { return c->M > 1 ? SegList{c->vseg_d, c->nvseg, c->voff_d} : SegList{}; }
SegList esegs(const ns_ctx *c) { return c->M > 1 ? SegList{c->eseg_d, c->neseg, c->eoff_d} : SegList{}; }
SegList fsegs(const ns_ctx *c) { return c->M > 1 ? SegList{c->fseg_d, c->nfseg, c->foff_d} : SegList{}; }
int nvparts(const ns_ctx *c) { return c->M > 1 ? c->nvseg : vec_blocks(c->m.N); }
PartMap vmap(const ns_ctx *c) { return c->M > 1 ? PartMap{c->voff_d, nullptr, 0} : PartMap{}; }
// operator partials: element blocks first, then face blocks
PartMap opmap(const ns_ctx *c) { return c->M > 1 ? PartMap{c->eoff_d, c->foff_d, c->neseg} : PartMap{}; }

// ---------------------------------------------------------------- operator application helpers

// y += Op x over all elements (atomic) or colour by colour (plain adds). Returns the number
// of dot partials written (if dot != nullptr).  yk (with dot): K x also accumulates there.
int apply_elems64(ns_ctx *c, const OpCoef *op, const double *xm, const double *xk, double *y, double *dot,
                  const int32_t *skip, int *npart, double *yk = nullptr) {
  const bool atomic = c->cfg.scatter == NS_SCATTER_ATOMIC;
  int off = 0;
  if (atomic) {
    LAUNCH(c, launch_ebe64(c->m, c->D, op, xm, xk, y, nullptr, 0, c->m.E, true, dot, skip, c->s_main, esegs(c), c->D2,
                           yk));
    off = c->M > 1 ? c->neseg : nblk(c->m.E);
  } else {
    for (size_t k = 0; k + 1 < c->m.ecol_off.size(); ++k) {
      const int64_t e0 = c->m.ecol_off[k], e1 = c->m.ecol_off[k + 1];
      LAUNCH(c, launch_ebe64(c->m, c->D, op, xm, xk, y, c->m.ecol_ids, e0, e1, false, dot ? dot + off : nullptr, skip,
                             c->s_main, SegList{}, c->D2, yk));
      off += nblk(e1 - e0);
    }
  }
  if (npart) *npart = off;
  return NS_OK;
}

int apply_faces64(ns_ctx *c, double cC, const double *x, const double *vin, double *y, double *dot,
                  const int32_t *skip, int *npart) {
  const bool atomic = c->cfg.scatter == NS_SCATTER_ATOMIC;
  int off = 0;
  if (c->m.F > 0) {
    if (atomic) {
      LAUNCH(c, launch_faces64(c->m, c->mats_d, cC, x, vin, y, nullptr, 0, c->m.F, true, dot, skip, c->s_main,
                               fsegs(c), c->M > 1 ? c->fmem_d : nullptr, 3 * c->n_vin));
      off = c->M > 1 ? c->nfseg : nblk(c->m.F);
    } else {
      for (size_t k = 0; k + 1 < c->m.fcol_off.size(); ++k) {
        const int64_t f0 = c->m.fcol_off[k], f1 = c->m.fcol_off[k + 1];
        LAUNCH(c, launch_faces64(c->m, c->mats_d, cC, x, vin, y, c->m.fcol_ids, f0, f1, false,
                                 dot ? dot + off : nullptr, skip, c->s_main));
        off += nblk(f1 - f0);
      }
    }
  }
  if (npart) *npart = off;
  return NS_OK;
}

// y = A x (the matrix of Eq. 1), with the element-energy partials of x.A x if dot != nullptr
// (and K x accumulated into yk if yk != nullptr)
int apply_A(ns_ctx *c, const double *x, double *y, bool zero_y, double *dot, const int32_t *skip, int *npart,
            bool timed, double *yk = nullptr) {
  int rc;
  if (zero_y) CKC(c, cudaMemsetAsync(y, 0, sizeof(double) * 3 * c->m.N, c->s_main));
  cudaEvent_t t0 = nullptr;
  if (timed) tbegin(c, TK_EBE64, c->s_main, &t0);
  int ne = 0, nf = 0;
  if ((rc = apply_elems64(c, c->op_A, nullptr, x, y, dot, skip, &ne, yk)) != NS_OK) return rc;
  if (timed) tend(c, TK_EBE64, c->s_main, t0);
  if ((rc = apply_faces64(c, 2.0 / c->cfg.dt, x, nullptr, y, dot ? dot + ne : nullptr, skip, &nf)) != NS_OK) return rc;
  if (npart) *npart = ne + nf;
  return NS_OK;
}

// y = A x in FP32 (inner preconditioner solve), element-energy partials into dot
int apply_A32(ns_ctx *c, const float *x, float *y, double *dot, const int32_t *skip, int *npart) {
  const bool atomic = c->cfg.scatter == NS_SCATTER_ATOMIC;
  int off = 0;
  cudaEvent_t t0 = nullptr;
  tbegin(c, TK_EBE32, c->s_main, &t0);
  const bool h16 = c->cfg.precision == NS_PREC_FP64_IR16;
  auto elems = [&](const int32_t *ids, int64_t e0, int64_t e1, bool at, double *d, SegList sg) {
    // automatic: the per-warp staged kernel for the FP32 tangent; direct loads for the FP16
    // one (half the tangent bytes, where staging measured slower)
    const int st = c->cfg.stage_elements >= 0 ? c->cfg.stage_elements : (h16 ? 0 : 2);
    return h16 ? launch_ebe16(c->m, c->D16, c->op_A16, x, y, ids, e0, e1, at, d, skip, c->s_main, sg, st)
               : launch_ebe32(c->m, c->D32, c->op_A, x, y, ids, e0, e1, at, d, skip, c->s_main, sg, st);
  };
  if (atomic) {
    LAUNCH(c, elems(nullptr, 0, c->m.E, true, dot, esegs(c)));
    off = c->M > 1 ? c->neseg : nblk(c->m.E);
  } else {
    for (size_t k = 0; k + 1 < c->m.ecol_off.size(); ++k) {
      const int64_t e0 = c->m.ecol_off[k], e1 = c->m.ecol_off[k + 1];
      LAUNCH(c, elems(c->m.ecol_ids, e0, e1, false, dot + off, SegList{}));
      off += nblk(e1 - e0);
    }
  }
  tend(c, TK_EBE32, c->s_main, t0);
  if (c->m.F > 0) {
    const float cC = (float)(2.0 / c->cfg.dt);
    if (atomic) {
      LAUNCH(c, launch_faces32(c->m, c->mats_d, cC, x, y, nullptr, 0, c->m.F, true, dot + off, skip, c->s_main,
                               fsegs(c)));
      off += c->M > 1 ? c->nfseg : nblk(c->m.F);
    } else {
      for (size_t k = 0; k + 1 < c->m.fcol_off.size(); ++k) {
        const int64_t f0 = c->m.fcol_off[k], f1 = c->m.fcol_off[k + 1];
        LAUNCH(c, launch_faces32(c->m, c->mats_d, cC, x, y, c->m.fcol_ids, f0, f1, false, dot + off, skip,
                                 c->s_main));
        off += nblk(f1 - f0);
      }
    }
  }
  *npart = off;
  return NS_OK;
}

int fill_opcoefs(ns_ctx *c) {
  const double dt = c->cfg.dt;
  OpCoef A{}, K{}, M{}, Cr{}, R{};
  for (int i = 0; i < c->nmat; ++i) {
    const MatConst &m = c->mats_h[i];
    A.mK[i] = m.rho * (4.0 / (dt * dt) + 2.0 * m.ray_a / dt);
    A.kK[i] = 1.0 + 2.0 * m.ray_b / dt;
    K.kK[i] = 1.0;
    M.mK[i] = m.rho;
    Cr.mK[i] = m.rho * m.ray_a;
    Cr.kK[i] = m.ray_b;
    R.mM[i] = m.rho;                          // M a
    R.mK[i] = m.rho * (4.0 / dt + m.ray_a);   // M (4/dt + alpha) v
    R.kK[i] = m.ray_b;                        // beta K v
  }
  CKC(c, cudaMemcpy(c->op_A, &A, sizeof(OpCoef), cudaMemcpyHostToDevice));
  OpCoef A16 = A;
  for (int i = 0; i < c->nmat; ++i) A16.kK[i] = A.kK[i] * c->mats_h[i].G0;
  CKC(c, cudaMemcpy(c->op_A16, &A16, sizeof(OpCoef), cudaMemcpyHostToDevice));
  CKC(c, cudaMemcpy(c->op_K, &K, sizeof(OpCoef), cudaMemcpyHostToDevice));
  CKC(c, cudaMemcpy(c->op_M, &M, sizeof(OpCoef), cudaMemcpyHostToDevice));
  CKC(c, cudaMemcpy(c->op_Cr, &Cr, sizeof(OpCoef), cudaMemcpyHostToDevice));
  CKC(c, cudaMemcpy(c->op_rhs, &R, sizeof(OpCoef), cudaMemcpyHostToDevice));
  return NS_OK;
}

int alloc_soa(ns_ctx *c, SpringSoA &s, int64_t nspr, bool host) {
  int rc;
  if (host) {
    if ((rc = halloc(c, &s.tau, nspr)) || (rc = halloc(c, &s.gR, nspr)) || (rc = halloc(c, &s.tR, nspr)) ||
        (rc = halloc(c, &s.gmax, nspr)) || (rc = halloc(c, &s.dir, nspr)) || (rc = halloc(c, &s.mode, nspr)))
      return rc;
    memset(s.tau, 0, nspr * 8);
    memset(s.gR, 0, nspr * 8);
    memset(s.tR, 0, nspr * 8);
    memset(s.gmax, 0, nspr * 8);
    memset(s.dir, 0, nspr * 4);
    memset(s.mode, 0, nspr * 4);
  } else {
    if ((rc = dalloc(c, &s.tau, nspr)) || (rc = dalloc(c, &s.gR, nspr)) || (rc = dalloc(c, &s.tR, nspr)) ||
        (rc = dalloc(c, &s.gmax, nspr)) || (rc = dalloc(c, &s.dir, nspr)) || (rc = dalloc(c, &s.mode, nspr)))
      return rc;
    CKC(c, cudaMemsetAsync(s.tau, 0, nspr * 8, c->s_main));
    CKC(c, cudaMemsetAsync(s.gR, 0, nspr * 8, c->s_main));
    CKC(c, cudaMemsetAsync(s.tR, 0, nspr * 8, c->s_main));
    CKC(c, cudaMemsetAsync(s.gmax, 0, nspr * 8, c->s_main));
    CKC(c, cudaMemsetAsync(s.dir, 0, nspr * 4, c->s_main));
    CKC(c, cudaMemsetAsync(s.mode, 0, nspr * 4, c->s_main));
  }
  return NS_OK;
}

void free_soa(SpringSoA &s, bool host) {
  if (host) {
    hfree(s.tau); hfree(s.gR); hfree(s.tR); hfree(s.gmax); hfree(s.dir); hfree(s.mode);
  } else {
    dfree(s.tau); dfree(s.gR); dfree(s.tR); dfree(s.gmax); dfree(s.dir); dfree(s.mode);
  }
}

// copy springs [off, off + n) between two SoA sets
int copy_soa(ns_ctx *c, const SpringSoA &dst, int64_t doff, const SpringSoA &src, int64_t soff, int64_t n,
             cudaMemcpyKind kind, cudaStream_t s) {
  CKC(c, cudaMemcpyAsync(dst.tau + doff, src.tau + soff, n * 8, kind, s));
  CKC(c, cudaMemcpyAsync(dst.gR + doff, src.gR + soff, n * 8, kind, s));
  CKC(c, cudaMemcpyAsync(dst.tR + doff, src.tR + soff, n * 8, kind, s));
  CKC(c, cudaMemcpyAsync(dst.gmax + doff, src.gmax + soff, n * 8, kind, s));
  CKC(c, cudaMemcpyAsync(dst.dir + doff, src.dir + soff, n * 4, kind, s));
  CKC(c, cudaMemcpyAsync(dst.mode + doff, src.mode + soff, n * 4, kind, s));
  return NS_OK;
}

// A state-stream copy is about to be issued: the injected fault of cfg.fault_state_copy.
int state_copy_fault(ns_ctx *c) {
  if (++c->n_state_copies == c->cfg.fault_state_copy) {
    c->err = "cudaMemcpyAsync of a state chunk failed (injected fault: state copy " + std::to_string(c->n_state_copies) +
             ")";
    return NS_ERR_CUDA;
  }
  return NS_OK;
}

int64_t n_chunks(const ns_ctx *c) {
  const int64_t ns_el = c->m.E - c->E_res;
  return ns_el <= 0 ? 0 : (ns_el + c->cfg.chunk_elems - 1) / c->cfg.chunk_elems;
}

// H2D of streamed chunk k into ring slot k % R
int issue_h2d(ns_ctx *c, int64_t k) {
  const int R = c->cfg.ring_depth;
  const int slot = (int)(k % R);
  const int64_t S4 = 4 * (int64_t)c->tab.S;
  const int64_t e0 = c->E_res + k * c->cfg.chunk_elems;
  const int64_t e1 = std::min(c->m.E, e0 + c->cfg.chunk_elems);
  if (k >= R) CKC(c, cudaStreamWaitEvent(c->s_h2d, c->ev_d2h[slot], 0));
  if (int f = state_copy_fault(c)) return f;
  int rc = copy_soa(c, c->ring[slot], 0, c->hst, (e0 - c->E_res) * S4, (e1 - e0) * S4, cudaMemcpyHostToDevice,
                    c->s_h2d);
  if (rc) return rc;
  c->stats.h2d_bytes += (e1 - e0) * S4 * 40;
  CKC(c, cudaEventRecord(c->ev_h2d[slot], c->s_h2d));
  return NS_OK;
}

// Start the first ring-depth chunk transfers of a step at its beginning: they depend only
// on the previous step's write-back of the same ring slot, so they overlap this step's
// right-hand side, preconditioner set-up and solve.
int prefetch_state(ns_ctx *c) {
  const int64_t nc = n_chunks(c);
  if (nc == 0 || c->prefetched || c->cfg.stream_mode == NS_STREAM_ZERO_COPY) return NS_OK;
  const int64_t h0 = c->stats.h2d_bytes;
  for (int64_t k = 0; k < std::min<int64_t>(nc, c->cfg.ring_depth); ++k) {
    // slot k was last drained by the previous step's D2H of the last chunk it held,
    // which the copy stream orders after the D2H of chunk k itself
    CKC(c, cudaStreamWaitEvent(c->s_h2d, c->ev_d2h[k], 0));
    int rc = issue_h2d(c, k);
    if (rc) return rc;
  }
  c->stats.h2d_bytes_early += c->stats.h2d_bytes - h0;
  c->prefetched = true;
  return NS_OK;
}

// Multi-spring update (Alg. 3 pipeline for the streamed part).  Streamed chunk k goes
// H2D (copy stream) -> compute (main stream) -> D2H (second copy stream) through a ring
// of R device buffers; the resident elements are cut into slices that the main stream
// computes between chunks, so the copy engines stay busy while a chunk is in flight.
int spring_launch(ns_ctx *c, const SpringSoA &st, int64_t base_elem, int64_t e0, int64_t e1) {
  if (e1 <= e0) return NS_OK;
  cudaEvent_t t0 = nullptr;
  tbegin(c, TK_SPRING, c->s_main, &t0);
  LAUNCH(c, launch_springs(c->tab, c->mats_d, c->m.mat, nullptr, c->eps, st, 4 * base_elem, 4 * e0, 4 * e1, c->D,
                           c->m.epad, nullptr, c->s_main, true));
  tend(c, TK_SPRING, c->s_main, t0);
  return NS_OK;
}

int spring_phase(ns_ctx *c) {
  int rc;
  LAUNCH(c, launch_strain_pairs(c->m, c->u, c->du, c->eps, 0, c->m.E, c->s_main));
  if (!c->mS.empty()) {
    // members with their own springs: one launch per member, all state resident; the
    // launches go to kMemberStreams streams forked from the main one, so that small
    // members' updates run side by side, and are joined back before the step ends
    const int NS_ = ns_ctx::kMemberStreams;
    CKC(c, cudaEventRecord(c->ev_fork, c->s_main));
    for (int k = 0; k < NS_; ++k) CKC(c, cudaStreamWaitEvent(c->s_mem[k], c->ev_fork, 0));
    for (int m = 0; m < c->M; ++m) {
      const int64_t e0 = c->moff_e[m], e1 = c->moff_e[m + 1], o = c->spr_off[m];
      SpringSoA sm{c->st.tau + o, c->st.gR + o, c->st.tR + o, c->st.gmax + o, c->st.dir + o, c->st.mode + o};
      LAUNCH(c, launch_springs(c->mtab[m], c->mats_d, c->m.mat, nullptr, c->eps, sm, 4 * e0, 4 * e0, 4 * e1, c->D,
                               c->m.epad, nullptr, c->s_mem[m % NS_], true));
    }
    for (int k = 0; k < NS_; ++k) {
      CKC(c, cudaEventRecord(c->ev_mem[k], c->s_mem[k]));
      CKC(c, cudaStreamWaitEvent(c->s_main, c->ev_mem[k], 0));
    }
    return NS_OK;
  }
  const int64_t nc = n_chunks(c);
  if (nc == 0) return spring_launch(c, c->st, 0, 0, c->E_res);
  if (c->cfg.timing) CKC(c, cudaEventRecord(c->ev_stream_t0, c->s_main));
  if (c->cfg.stream_mode == NS_STREAM_ZERO_COPY) {
    // the streamed elements' springs are read and written in pinned host memory in place
    if ((rc = spring_launch(c, c->st, 0, 0, c->E_res)) != NS_OK) return rc;
    if ((rc = spring_launch(c, c->hst_dev, c->E_res, c->E_res, c->m.E)) != NS_OK) return rc;
    const int64_t b = (c->m.E - c->E_res) * 4 * (int64_t)c->tab.S * 40;
    c->stats.h2d_bytes += b;
    c->stats.d2h_bytes += b;
    if (c->cfg.timing) CKC(c, cudaEventRecord(c->ev_stream_t1, c->s_main));
    return NS_OK;
  }
  if ((rc = prefetch_state(c)) != NS_OK) return rc;
  const int R = c->cfg.ring_depth;
  const int64_t S4 = 4 * (int64_t)c->tab.S;
  auto slice = [&](int64_t k) { return c->E_res * k / (nc + 1); };  // resident slice k = [slice(k), slice(k+1))
  if ((rc = spring_launch(c, c->st, 0, slice(0), slice(1))) != NS_OK) return rc;
  for (int64_t k = 0; k < nc; ++k) {
    const int slot = (int)(k % R);
    const int64_t e0 = c->E_res + k * c->cfg.chunk_elems;
    const int64_t e1 = std::min(c->m.E, e0 + c->cfg.chunk_elems);
    CKC(c, cudaStreamWaitEvent(c->s_main, c->ev_h2d[slot], 0));
    if ((rc = spring_launch(c, c->ring[slot], e0, e0, e1)) != NS_OK) return rc;
    CKC(c, cudaEventRecord(c->ev_comp[slot], c->s_main));
    CKC(c, cudaStreamWaitEvent(c->s_d2h, c->ev_comp[slot], 0));
    if ((rc = state_copy_fault(c)) != NS_OK) return rc;
    if ((rc = copy_soa(c, c->hst, (e0 - c->E_res) * S4, c->ring[slot], 0, (e1 - e0) * S4, cudaMemcpyDeviceToHost,
                       c->s_d2h)))
      return rc;
    c->stats.d2h_bytes += (e1 - e0) * S4 * 40;
    CKC(c, cudaEventRecord(c->ev_d2h[slot], c->s_d2h));
    if (k + R < nc && (rc = issue_h2d(c, k + R)) != NS_OK) return rc;
    if ((rc = spring_launch(c, c->st, 0, slice(k + 1), slice(k + 2))) != NS_OK) return rc;
  }
  CKC(c, cudaEventRecord(c->ev_d2h_all, c->s_d2h));
  if (c->cfg.timing) CKC(c, cudaEventRecord(c->ev_stream_t1, c->s_d2h));
  c->prefetched = false;
  return NS_OK;
}

int read_scalars(ns_ctx *c) {
  const size_t n = 2 * (size_t)c->M + (c->cfg.multigrid ? 1 : 0);
  CKC(c, cudaMemcpyAsync(c->sc_h, c->sc, n * sizeof(CgScalars), cudaMemcpyDeviceToHost, c->s_main));
  return sync_stream(c, c->s_main);
}

// y_c (+)= Op_c x_c over the coarse elements and (cC != 0) faces, atomic or colour by colour;
// with dot the energy partials of the application (elements, then faces).
int apply_mg(ns_ctx *c, const OpCoef *op, float cC, const float *x, float *y, double *dot, const int32_t *skip,
             int *npart) {
  const bool atomic = c->cfg.scatter == NS_SCATTER_ATOMIC;
  int off = 0;
  if (op) {
    if (atomic) {
      LAUNCH(c, launch_mg_ebe(c->m, c->mg, op, x, y, nullptr, 0, c->m.E, true, dot, skip, c->s_main));
      off = nblk(c->m.E);
    } else {
      for (size_t k = 0; k + 1 < c->m.ecol_off.size(); ++k) {
        const int64_t e0 = c->m.ecol_off[k], e1 = c->m.ecol_off[k + 1];
        LAUNCH(c, launch_mg_ebe(c->m, c->mg, op, x, y, c->m.ecol_ids, e0, e1, false, dot ? dot + off : nullptr, skip,
                                c->s_main));
        off += nblk(e1 - e0);
      }
    }
  }
  if (cC != 0.0f && c->m.F > 0) {
    if (atomic) {
      LAUNCH(c, launch_mg_faces(c->m, c->mg, c->mats_d, cC, x, y, nullptr, 0, c->m.F, true, dot ? dot + off : nullptr,
                                skip, c->s_main));
      off += nblk(c->m.F);
    } else {
      for (size_t k = 0; k + 1 < c->m.fcol_off.size(); ++k) {
        const int64_t f0 = c->m.fcol_off[k], f1 = c->m.fcol_off[k + 1];
        LAUNCH(c, launch_mg_faces(c->m, c->mg, c->mats_d, cC, x, y, c->m.fcol_ids, f0, f1, false,
                                  dot ? dot + off : nullptr, skip, c->s_main));
        off += nblk(f1 - f0);
      }
    }
  }
  if (npart) *npart = off;
  return NS_OK;
}

// Two-level start of the inner solve of one outer iteration: the coarse PCG on
// P^T (r / ||r||) (at most coarse_max_iter iterations or to coarse_tol), its solution
// interpolated onto the quadratic nodes as the inner solve's first iterate, the residual
// of that iterate, and the inner scalars' initial reduction.
int mg_start_inner(ns_ctx *c, double *pv) {
  const int64_t N = c->m.N, Nc = c->mg.Nc;
  const int nbc = vec_blocks(Nc), nbv = vec_blocks(N);
  MgLevel &g = c->mg;
  LAUNCH(c, launch_mg_restrict_init(c->r, c->sc, g, g.r, g.z, g.p, g.x, g.Ap, pv, c->s_main));
  LAUNCH(c, launch_cg_final(pv, nbc, 3, c->sc_c, NS_FIN_INIT, c->cfg.coarse_tol, c->cfg.coarse_max_iter, c->s_main, 1,
                            {}, c->sc));
  const float cC = (float)(2.0 / c->cfg.dt);
  for (int it = 0; it < c->cfg.coarse_max_iter; ++it) {
    int np = 0, rc;
    if ((rc = apply_mg(c, c->op_A, cC, g.p, g.Ap, c->part, &c->sc_c->done, &np)) != NS_OK) return rc;
    LAUNCH(c, launch_cg_final(c->part, np, 1, c->sc_c, NS_FIN_PAP, c->cfg.coarse_tol, c->cfg.coarse_max_iter,
                              c->s_main));
    LAUNCH(c, launch_in_update(g.x, g.r, g.z, g.p, g.Ap, g.Jinv32, Nc, pv, c->sc_c, c->sc, c->s_main));
    LAUNCH(c, launch_cg_final(pv, nbc, 2, c->sc_c, NS_FIN_UPDATE, c->cfg.coarse_tol, c->cfg.coarse_max_iter,
                              c->s_main));
    LAUNCH(c, launch_in_pupdate(g.p, g.z, g.Ap, Nc, c->sc_c, c->sc, c->s_main));
  }
  LAUNCH(c, launch_mg_prolong(g, g.x, c->xin, c->Apin, N, c->sc, c->s_main));
  int np = 0, rc;
  if ((rc = apply_A32(c, c->xin, c->Apin, c->part, &c->sc->done, &np)) != NS_OK) return rc;
  LAUNCH(c, launch_mg_fine_init(c->r, c->sc, c->Jinv32, c->rin, c->zin, c->pin, c->Apin, N, pv, c->s_main));
  LAUNCH(c, launch_cg_final(pv, nbv, 3, c->sc_in, NS_FIN_INIT, c->cfg.inner_tol, c->cfg.inner_max_iter, c->s_main, 1,
                            {}, c->sc));
  return NS_OK;
}

// outer solve finished for every member (scalars read back)
bool outer_done(const ns_ctx *c) {
  for (int m = 0; m < c->M; ++m)
    if (c->sc_h[m].done == 0) return false;
  return true;
}

// members with a zero right-hand side take du = 0 (done == 2 after the initial reduction)
int zero_rhs_members(ns_ctx *c) {
  for (int m = 0; m < c->M; ++m)
    if (c->sc_h[m].done == 2) {
      const int64_t n0 = c->M > 1 ? c->moff_n[m] : 0, n1 = c->M > 1 ? c->moff_n[m + 1] : c->m.N;
      CKC(c, cudaMemsetAsync(c->du + 3 * n0, 0, sizeof(double) * 3 * (n1 - n0), c->s_main));
    }
  return NS_OK;
}

// Issue a fixed launch sequence on the main stream: directly, or (cfg.graphs) captured into
// a CUDA graph on first use and replayed afterwards.  Every pointer and launch shape in the
// sequence is fixed for the context's life; what varies (converged members, iteration
// counts) lives in device memory that the kernels read.
template <typename F>
int issue_fixed(ns_ctx *c, cudaGraphExec_t *ge, int64_t cnt[3], F &&issue) {
  if (!c->cfg.graphs) return issue();
  if (!*ge) {
    const int64_t k0 = c->stats.kernel_launches;
    c->cap_ebe32 = c->cap_ebe64 = 0;
    CKC(c, cudaStreamBeginCapture(c->s_main, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    int rc = issue();
    c->capturing = false;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->s_main, &g);
    if (rc == NS_OK && e != cudaSuccess) {
      c->err = std::string("stream capture: ") + cudaGetErrorString(e);
      rc = NS_ERR_CUDA;
    }
    if (rc == NS_OK) {
      const cudaError_t e2 = cudaGraphInstantiate(ge, g, 0);
      if (e2 != cudaSuccess) {
        c->err = std::string("graph instantiation: ") + cudaGetErrorString(e2);
        *ge = nullptr;
        rc = NS_ERR_CUDA;
      }
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    cnt[0] = c->stats.kernel_launches - k0;  // kernels, FP32 and FP64 operator launches of one replay
    cnt[1] = c->cap_ebe32;
    cnt[2] = c->cap_ebe64;
    c->stats.kernel_launches = k0;
    if (rc != NS_OK) return rc;
  }
  CKC(c, cudaGraphLaunch(*ge, c->s_main));
  c->stats.kernel_launches += cnt[0];
  c->stats.n_ebe32 += cnt[1];
  c->stats.n_ebe64 += cnt[2];
  return NS_OK;
}

// A solve from zero builds du = sum_k alpha_k p_k, so q^n = q^{n-1} + K du can be
// accumulated as q += alpha_k K p_k, K p_k coming out of the operator application that
// the iteration makes anyway (A = cK K + mass and damping terms) -- one FP64 element
// sweep per step fewer.  K p_k goes to b, which is dead once the initial residual is formed.
// Only the flexible solver does it: its few outer iterations pay for the extra scatter,
// the plain PCG's dozens of iterations would not (measured: +3% per step).
bool q_folded(const ns_ctx *c) { return !c->cfg.x0_prev && c->cfg.precision != NS_PREC_FP64; }

void destroy_graphs(ns_ctx *c) {
  if (c->g_outer) cudaGraphExecDestroy(c->g_outer);
  if (c->g_batch) cudaGraphExecDestroy(c->g_batch);
  c->g_outer = c->g_batch = nullptr;
}

// Flexible FP64 CG whose preconditioner is an FP32 block-Jacobi PCG on the same operator
// (the paper's precision policy: only the preconditioning is single precision).  With
// members every launch covers all of them and each member iterates on its own scalars.
int solve_ir(ns_ctx *c) {
  int rc;
  const int64_t N = c->m.N;
  const int nbv = nvparts(c), M = c->M;
  const SegList vs = vsegs(c);
  const PartMap vm = vmap(c), om = opmap(c);
  double *pv = c->part + c->part_pap_cap;
  double *Kp = q_folded(c) ? c->b : nullptr, *qf = q_folded(c) ? c->q : nullptr;
  if (c->cfg.x0_prev) {
    if ((rc = apply_A(c, c->du, c->Ap, true, nullptr, nullptr, nullptr, false)) != NS_OK) return rc;
  } else {  // from zero: A x0 = 0, no operator application
    CKC(c, cudaMemsetAsync(c->du, 0, sizeof(double) * 3 * N, c->s_main));
    CKC(c, cudaMemsetAsync(c->Ap, 0, sizeof(double) * 3 * N, c->s_main));
  }
  LAUNCH(c, launch_fcg_init(c->b, c->Ap, c->r, N, pv, c->s_main, vs));
  LAUNCH(c, launch_cg_final(pv, nbv, 2, c->sc, NS_FIN_FCG_INIT, c->cfg.cg_tol, c->cfg.cg_max_iter, c->s_main, M, vm));
  if ((rc = read_scalars(c)) != NS_OK) return rc;
  if ((rc = zero_rhs_members(c)) != NS_OK) return rc;
  int inner_total = 0;
  const int32_t *skip_in = &c->sc_in->done, *skip_out = &c->sc->done;
  // one outer iteration: inner FP32 solve A z ~= r from zero, then the flexible CG update
  auto outer_iteration = [&]() -> int {
    int rc;
    if (c->cfg.multigrid) {
      if ((rc = mg_start_inner(c, pv)) != NS_OK) return rc;
    } else {
      LAUNCH(c, launch_in_init(c->r, c->sc, c->Jinv32, c->rin, c->zin, c->pin, c->xin, c->Apin, N, pv, c->s_main,
                               vs));
      LAUNCH(c, launch_cg_final(pv, nbv, 3, c->sc_in, NS_FIN_INIT, c->cfg.inner_tol, c->cfg.inner_max_iter,
                                c->s_main, M, vm, c->sc));
    }
    for (int it = 0; it < c->cfg.inner_max_iter; ++it) {
      int np = 0;
      if ((rc = apply_A32(c, c->pin, c->Apin, c->part, skip_in, &np)) != NS_OK) return rc;
      LAUNCH(c, launch_cg_final(c->part, np, 1, c->sc_in, NS_FIN_PAP, c->cfg.inner_tol, c->cfg.inner_max_iter,
                                c->s_main, M, om));
      LAUNCH(c, launch_in_update(c->xin, c->rin, c->zin, c->pin, c->Apin, c->Jinv32, N, pv, c->sc_in, c->sc,
                                 c->s_main, vs));
      LAUNCH(c, launch_cg_final(pv, nbv, 2, c->sc_in, NS_FIN_UPDATE, c->cfg.inner_tol, c->cfg.inner_max_iter,
                                c->s_main, M, vm));
      LAUNCH(c, launch_in_pupdate(c->pin, c->zin, c->Apin, N, c->sc_in, c->sc, c->s_main, vs));
    }
    // outer flexible CG step
    LAUNCH(c, launch_fcg_gamma(c->xin, c->z, c->Ap, N, pv, c->sc, c->s_main, vs));
    LAUNCH(c, launch_cg_final(pv, nbv, 1, c->sc, NS_FIN_FCG_BETA, c->cfg.cg_tol, c->cfg.cg_max_iter, c->s_main, M, vm));
    LAUNCH(c, launch_fcg_p(c->p, c->z, c->r, c->Ap, Kp, N, pv, c->sc, c->s_main, vs));
    int np = 0;
    if ((rc = apply_A(c, c->p, c->Ap, false, c->part, skip_out, &np, true, Kp)) != NS_OK) return rc;
    LAUNCH(c, launch_fcg_alpha(pv, nbv, c->part, np, c->sc, c->s_main, M, vm, om));
    LAUNCH(c, launch_fcg_update(c->du, c->r, c->p, c->Ap, qf, Kp, N, pv, c->sc, c->s_main, vs));
    LAUNCH(c, launch_cg_final(pv, nbv, 1, c->sc, NS_FIN_FCG_UPDATE, c->cfg.cg_tol, c->cfg.cg_max_iter, c->s_main, M,
                              vm));
    return NS_OK;
  };
  while (!outer_done(c)) {
    if ((rc = issue_fixed(c, &c->g_outer, c->g_outer_cnt, outer_iteration)) != NS_OK)
      return rc;
    if ((rc = read_scalars(c)) != NS_OK) return rc;
    int most = 0;
    for (int m = 0; m < M; ++m) most = std::max(most, c->sc_h[M + m].iters);
    inner_total += most;
    if (c->cfg.multigrid) c->stats.coarse_iters_total += c->sc_h[2].iters;
  }
  c->stats.inner_iters_last = inner_total;
  c->stats.inner_iters_total += inner_total;
  return NS_OK;
}

// Plain FP64 block-Jacobi PCG; convergence read back every `batch` iterations (kernels of
// a converged member skip themselves in between).
int solve_pcg(ns_ctx *c) {
  int rc;
  const int64_t N = c->m.N;
  const int nbv = nvparts(c), M = c->M;
  const SegList vs = vsegs(c);
  const PartMap vm = vmap(c), om = opmap(c);
  double *pv = c->part + c->part_pap_cap;
  if (c->cfg.x0_prev) {
    if ((rc = apply_A(c, c->du, c->Ap, true, nullptr, nullptr, nullptr, false)) != NS_OK) return rc;
  } else {  // from zero: A x0 = 0, no operator application
    CKC(c, cudaMemsetAsync(c->du, 0, sizeof(double) * 3 * N, c->s_main));
    CKC(c, cudaMemsetAsync(c->Ap, 0, sizeof(double) * 3 * N, c->s_main));
  }
  LAUNCH(c, launch_cg_init(c->b, c->Ap, c->Jinv, c->r, c->z, c->p, N, pv, c->s_main, vs));
  LAUNCH(c, launch_cg_final(pv, nbv, 3, c->sc, NS_FIN_INIT, c->cfg.cg_tol, c->cfg.cg_max_iter, c->s_main, M, vm));
  if ((rc = read_scalars(c)) != NS_OK) return rc;
  if ((rc = zero_rhs_members(c)) != NS_OK) return rc;
  const int batch = 8;
  const int32_t *skip = &c->sc->done;
  if (!outer_done(c)) {
    CKC(c, cudaMemsetAsync(c->Ap, 0, sizeof(double) * 3 * N, c->s_main));
    auto iterations = [&]() -> int {
      int rc;
      for (int it = 0; it < batch; ++it) {
        int np = 0;
        if ((rc = apply_A(c, c->p, c->Ap, false, c->part, skip, &np, true)) != NS_OK) return rc;
        LAUNCH(c, launch_cg_final(c->part, np, 1, c->sc, NS_FIN_PAP, c->cfg.cg_tol, c->cfg.cg_max_iter, c->s_main, M,
                                  om));
        LAUNCH(c, launch_cg_update(c->du, c->r, c->z, c->p, c->Ap, c->Jinv, N, pv, c->sc, c->s_main, vs));
        LAUNCH(c, launch_cg_final(pv, nbv, 2, c->sc, NS_FIN_UPDATE, c->cfg.cg_tol, c->cfg.cg_max_iter, c->s_main, M,
                                  vm));
        LAUNCH(c, launch_cg_pupdate(c->p, c->z, c->Ap, N, c->sc, c->s_main, vs));
      }
      return NS_OK;
    };
    for (;;) {
      if ((rc = issue_fixed(c, &c->g_batch, c->g_batch_cnt, iterations)) != NS_OK)
        return rc;
      if ((rc = read_scalars(c)) != NS_OK) return rc;
      if (outer_done(c)) break;
    }
  }
  return NS_OK;
}

// One time step n = step + 1 (Eq. 1 and the updates below it, then the spring update).
int one_step(ns_ctx *c) {
  int rc;
  const double dt = c->cfg.dt;
  const int64_t N = c->m.N, n = c->step + 1;
  const bool atomic = c->cfg.scatter == NS_SCATTER_ATOMIC;
  cudaEvent_t tstep = nullptr, t0 = nullptr;
  tbegin(c, TK_STEP, c->s_main, &tstep);
  if ((rc = prefetch_state(c)) != NS_OK) return rc;

  // 3x3 block-Jacobi preconditioner from the diagonal node blocks of A^n (FP32 when it only
  // serves the inner single-precision solve)
  tbegin(c, TK_JAC, c->s_main, &t0);
  CKC(c, cudaMemsetAsync(c->flag_d, 0, sizeof(int32_t), c->s_main));
  if (c->D2) LAUNCH(c, launch_to_pairs(c->D, c->D2, 84 * c->m.epad, c->s_main));
  if (c->cfg.precision != NS_PREC_FP64) {
    // FP32 blocks from the inner operator's own copy of the tangent (FP32, or FP16 / G0)
    const bool h16 = c->cfg.precision == NS_PREC_FP64_IR16;
    float *Jd32 = (float *)c->Jd;  // the FP64 block buffer is reused for the FP32 blocks
    if (h16)
      LAUNCH(c, launch_D_to_f16(c->D, c->m.mat, c->mats_d, c->D16, c->m.epad, c->m.E, c->s_main));
    else
      LAUNCH(c, launch_D_to_f32(c->D, c->D32, c->m.epad, c->m.E, c->s_main));
    CKC(c, cudaMemsetAsync(Jd32, 0, sizeof(float) * 6 * N, c->s_main));
    auto jel = [&](const int32_t *ids, int64_t e0, int64_t e1, bool at) {
      return h16 ? launch_jacobi_elems16(c->m, c->D16, c->op_A16, Jd32, ids, e0, e1, at, c->s_main)
                 : launch_jacobi_elems32(c->m, c->D32, c->op_A, Jd32, ids, e0, e1, at, c->s_main);
    };
    if (atomic) {
      LAUNCH(c, jel(nullptr, 0, c->m.E, true));
      LAUNCH(c, launch_jacobi_faces32(c->m, c->mats_d, 2.0 / dt, Jd32, nullptr, 0, c->m.F, true, c->s_main));
    } else {
      for (size_t k = 0; k + 1 < c->m.ecol_off.size(); ++k)
        LAUNCH(c, jel(c->m.ecol_ids, c->m.ecol_off[k], c->m.ecol_off[k + 1], false));
      for (size_t k = 0; k + 1 < c->m.fcol_off.size(); ++k)
        LAUNCH(c, launch_jacobi_faces32(c->m, c->mats_d, 2.0 / dt, Jd32, c->m.fcol_ids, c->m.fcol_off[k],
                                        c->m.fcol_off[k + 1], false, c->s_main));
    }
    LAUNCH(c, launch_invert_blocks32(Jd32, c->Jinv32, N, c->flag_d, c->s_main));
    if (c->cfg.multigrid) {  // coarse tangent (four-point mean) and coarse block-Jacobi blocks
      MgLevel &g = c->mg;
      LAUNCH(c, launch_mg_dbar(c->D, g.Dbar, c->m.epad, c->m.E, c->s_main));
      CKC(c, cudaMemsetAsync(g.Jd32, 0, sizeof(float) * 6 * g.Nc, c->s_main));
      if (atomic) {
        LAUNCH(c, launch_mg_jacobi(c->m, g, c->op_A, g.Jd32, nullptr, 0, c->m.E, true, c->s_main));
        LAUNCH(c, launch_mg_jacobi_faces(c->m, g, c->mats_d, (float)(2.0 / dt), g.Jd32, nullptr, 0, c->m.F, true,
                                         c->s_main));
      } else {
        for (size_t k = 0; k + 1 < c->m.ecol_off.size(); ++k)
          LAUNCH(c, launch_mg_jacobi(c->m, g, c->op_A, g.Jd32, c->m.ecol_ids, c->m.ecol_off[k], c->m.ecol_off[k + 1],
                                     false, c->s_main));
        for (size_t k = 0; k + 1 < c->m.fcol_off.size(); ++k)
          LAUNCH(c, launch_mg_jacobi_faces(c->m, g, c->mats_d, (float)(2.0 / dt), g.Jd32, c->m.fcol_ids,
                                           c->m.fcol_off[k], c->m.fcol_off[k + 1], false, c->s_main));
      }
      LAUNCH(c, launch_invert_blocks32(g.Jd32, g.Jinv32, g.Nc, c->flag_d, c->s_main));
    }
  } else {
    CKC(c, cudaMemsetAsync(c->Jd, 0, sizeof(double) * 6 * N, c->s_main));
    if (atomic) {
      LAUNCH(c, launch_jacobi_elems(c->m, c->D, c->op_A, c->Jd, nullptr, 0, c->m.E, true, c->s_main));
      LAUNCH(c, launch_jacobi_faces(c->m, c->mats_d, 2.0 / dt, c->Jd, nullptr, 0, c->m.F, true, c->s_main));
    } else {
      for (size_t k = 0; k + 1 < c->m.ecol_off.size(); ++k)
        LAUNCH(c, launch_jacobi_elems(c->m, c->D, c->op_A, c->Jd, c->m.ecol_ids, c->m.ecol_off[k],
                                      c->m.ecol_off[k + 1], false, c->s_main));
      for (size_t k = 0; k + 1 < c->m.fcol_off.size(); ++k)
        LAUNCH(c, launch_jacobi_faces(c->m, c->mats_d, 2.0 / dt, c->Jd, c->m.fcol_ids, c->m.fcol_off[k],
                                      c->m.fcol_off[k + 1], false, c->s_main));
    }
    LAUNCH(c, launch_invert_blocks(c->Jd, c->Jinv, c->Jinv32, N, c->flag_d, c->s_main));
  }
  tend(c, TK_JAC, c->s_main, t0);

  // right-hand side of Eq. 1: f^n - q^{n-1} + C^n v^{n-1} + M (a^{n-1} + 4/dt v^{n-1})
  tbegin(c, TK_RHS, c->s_main, &t0);
  LAUNCH(c, launch_negate_copy(c->b, c->q, 3 * N, c->s_main));
  if ((rc = apply_elems64(c, c->op_rhs, c->a, c->v, c->b, nullptr, nullptr, nullptr)) != NS_OK) return rc;
  const double *vin = c->vin_d + 3 * std::min<int64_t>(n, c->n_vin - 1);
  if ((rc = apply_faces64(c, 1.0, c->v, vin, c->b, nullptr, nullptr, nullptr)) != NS_OK) return rc;
  tend(c, TK_RHS, c->s_main, t0);

  // PCG on A du = b, starting from the previous increment (or zero)
  tbegin(c, TK_SOLVE, c->s_main, &t0);
  CKC(c, cudaMemcpyAsync(c->flag_h, c->flag_d, sizeof(int32_t), cudaMemcpyDeviceToHost, c->s_main));
  if ((rc = (c->cfg.precision != NS_PREC_FP64) ? solve_ir(c) : solve_pcg(c)) != NS_OK) return rc;
  tend(c, TK_SOLVE, c->s_main, t0);
  if (*c->flag_h) NS_SET(c, NS_ERR_STATE, "block-Jacobi preconditioner has a non-positive diagonal block");
  int most = 0, lim = -1;
  double relres = 0.0;
  c->member_iters.assign(c->M, 0);
  for (int m = 0; m < c->M; ++m) {
    const CgScalars &sh = c->sc_h[m];
    c->member_iters[m] = sh.iters;
    most = std::max(most, sh.iters);
    if (sh.done == 3 && lim < 0) lim = m;
    if (sh.bb > 0) relres = std::max(relres, sqrt(sh.rr / sh.bb));
  }
  c->stats.cg_iters_last = most;
  if (lim >= 0)
    NS_SET(c, NS_ERR_NOT_CONVERGED,
           "CG reached the iteration limit at step " + std::to_string(n) +
               (c->M > 1 ? " (member " + std::to_string(lim) + ")" : std::string()));
  c->stats.cg_iters_total += most;
  c->stats.relres_last = relres;

  // q^n = q^{n-1} + K^n du (already accumulated by the solve when it started from zero);
  // u, v, a updates; surface record
  tbegin(c, TK_NEWMARK, c->s_main, &t0);
  if (!q_folded(c))
    if ((rc = apply_elems64(c, c->op_K, nullptr, c->du, c->q, nullptr, nullptr, nullptr)) != NS_OK) return rc;
  LAUNCH(c, launch_newmark(c->u, c->v, c->a, nullptr, c->du, N, dt, c->s_main));
  if (c->m.Ns > 0) {
    const int64_t slot = (n - 1) % c->ring_steps, off = slot * c->m.Ns * 3;
    LAUNCH(c, launch_surface_gather(c->m.surf, c->m.Ns, c->u, c->v, c->a, c->surf_u + off, c->surf_v + off,
                                    c->surf_a + off, c->s_main));
  }
  tend(c, TK_NEWMARK, c->s_main, t0);

  // multi-spring update -> D^n for the next step (lagged tangent, Alg. 4)
  tbegin(c, TK_SPRINGS, c->s_main, &t0);
  if ((rc = spring_phase(c)) != NS_OK) return rc;
  tend(c, TK_SPRINGS, c->s_main, t0);
  tend(c, TK_STEP, c->s_main, tstep);
  c->step = n;
  c->stats.steps = n;
  return NS_OK;
}

}  // namespace

// ============================================================================ context views

namespace ns {
int ctx_spring_view(ns_ctx *c, SpringCtxView *v) {
  if (!c || !c->has_mat) return NS_ERR_STATE;
  v->tab = c->tab;
  v->mats = c->mats_d;
  v->nmat = c->nmat;
  v->stream = c->s_main;
  v->device = c->cfg.device;
  return NS_OK;
}
void ctx_set_error(ns_ctx *c, const char *msg) { c->err = msg; }

int64_t ctx_steps(ns_ctx *c) { return c->step; }

int ctx_copy_member(ns_ctx *dst, int md, ns_ctx *src, int ms) {
  auto range = [](const ns_ctx *c, int m, const std::vector<int64_t> &off, int64_t all, int64_t &a0, int64_t &n) {
    if (c->M > 1) {
      a0 = off[m];
      n = off[m + 1] - off[m];
    } else {
      a0 = 0;
      n = all;
    }
  };
  if (!dst || !src || !dst->has_mat || !src->has_mat) return NS_ERR_STATE;
  if (dst->E_res < dst->m.E || src->E_res < src->m.E) NS_SET(dst, NS_ERR_STATE, "member copy needs resident state");
  int64_t en0s, ens, en0d, end_, nn0s, nns, nn0d, nnd;
  range(src, ms, src->moff_e, src->m.E, en0s, ens);
  range(dst, md, dst->moff_e, dst->m.E, en0d, end_);
  range(src, ms, src->moff_n, src->m.N, nn0s, nns);
  range(dst, md, dst->moff_n, dst->m.N, nn0d, nnd);
  const int Ss = src->mS.empty() ? src->tab.S : src->mS[ms], Sd = dst->mS.empty() ? dst->tab.S : dst->mS[md];
  if (ens != end_ || nns != nnd || Ss != Sd) NS_SET(dst, NS_ERR_INVALID_ARG, "member copy between different cases");
  const int64_t sps = src->mS.empty() ? en0s * 4 * Ss : src->spr_off[ms];
  const int64_t spd = dst->mS.empty() ? en0d * 4 * Sd : dst->spr_off[md];
  const int64_t nspr = ens * 4 * (int64_t)Ss;
  int rc;
  if ((rc = sync_all(src)) != NS_OK) return rc;
  if ((rc = sync_all(dst)) != NS_OK) return rc;
  cudaStream_t s = dst->s_main;
  const double *vs[5] = {src->u, src->v, src->a, src->q, src->du};
  double *vd[5] = {dst->u, dst->v, dst->a, dst->q, dst->du};
  for (int f = 0; f < 5; ++f)
    CKC(dst, cudaMemcpyAsync(vd[f] + 3 * nn0d, vs[f] + 3 * nn0s, 24 * nns, cudaMemcpyDeviceToDevice, s));
  for (int k = 0; k < 84; ++k)
    CKC(dst, cudaMemcpyAsync(dst->D + (size_t)k * dst->m.epad + en0d, src->D + (size_t)k * src->m.epad + en0s, 8 * ens,
                             cudaMemcpyDeviceToDevice, s));
  if ((rc = copy_soa(dst, dst->st, spd, src->st, sps, nspr, cudaMemcpyDeviceToDevice, s)) != NS_OK) return rc;
  return sync_stream(dst, s);
}

int ctx_set_member_velocity(ns_ctx *c, int m, const double *vin, int64_t n) {
  if (!c || !vin || n < 1) return NS_ERR_INVALID_ARG;
  if (!c->has_motion) NS_SET(c, NS_ERR_STATE, "set the ground motion first");
  if (m < 0 || m >= c->M) NS_SET(c, NS_ERR_INVALID_ARG, "member index out of range");
  std::vector<double> row(3 * (size_t)c->n_vin);
  for (int64_t k = 0; k < c->n_vin; ++k)
    for (int cc = 0; cc < 3; ++cc) row[3 * k + cc] = vin[3 * std::min(k, n - 1) + cc];
  CKC(c, cudaMemcpy(c->vin_d + (size_t)m * row.size(), row.data(), row.size() * 8, cudaMemcpyHostToDevice));
  return NS_OK;
}
void ctx_count_launches(ns_ctx *c, int n) { c->stats.kernel_launches += n; }
int ctx_sync_main(ns_ctx *c) { return sync_stream(c, c->s_main); }
}  // namespace ns

// ============================================================================ C ABI

extern "C" {

void ns_config_default(ns_config *cfg) {
  memset(cfg, 0, sizeof(*cfg));
  cfg->n_springs = 10;
  cfg->dt = 0.01;
  cfg->cg_tol = 1e-8;
  cfg->cg_max_iter = 10000;
  cfg->x0_prev = 1;
  cfg->precision = NS_PREC_FP64;
  cfg->scatter = NS_SCATTER_ATOMIC;
  cfg->chunk_elems = 100000;
  cfg->ring_depth = 3;
  cfg->device_state_budget = -1;
  cfg->rayleigh_f1 = 0.1;
  cfg->rayleigh_f2 = 2.5;
  cfg->surface_ring_steps = 64;
  cfg->device = 0;
  cfg->timing = 0;
  cfg->inner_max_iter = 45;
  cfg->inner_tol = 1e-4;
  cfg->wait_timeout_s = 120.0;
  cfg->graphs = 1;
  cfg->stage_elements = -1;
  cfg->stream_mode = NS_STREAM_RING;
  cfg->pair_operator = 0;
  cfg->l2_prefetch = 1;
  cfg->spring_tile_points = 0;
  cfg->spring_tile_blocks = 4;
  cfg->spring_tensor_cores = 0;
  cfg->fault_pinned_alloc = 0;
  cfg->fault_state_copy = 0;
  cfg->multigrid = 0;
  cfg->coarse_max_iter = 20;
  cfg->coarse_tol = 1e-2;
  cfg->shared_members = 0;
  cfg->local_gather = 0;
}

static thread_local std::string g_create_err;
static int setup_members(ns_ctx *c, int32_t M, const int64_t *elem_off, const int64_t *node_off);

const char *ns_last_error(ns_ctx *ctx) {
  if (!ctx) return g_create_err.c_str();
  return ctx->err.c_str();
}

int ns_create(ns_ctx **out, const ns_config *cfg) {
  if (!out || !cfg) {
    g_create_err = "null argument";
    return NS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (cfg->n_springs < 5 || !(cfg->dt > 0) || !(cfg->cg_tol > 0) || cfg->cg_max_iter < 1 || cfg->ring_depth < 2 ||
      cfg->chunk_elems < 1 || cfg->surface_ring_steps < 1 ||
      (cfg->precision != NS_PREC_FP64 && cfg->precision != NS_PREC_FP64_IR &&
       cfg->precision != NS_PREC_FP64_IR16) ||
      (cfg->scatter != NS_SCATTER_ATOMIC && cfg->scatter != NS_SCATTER_COLOUR) || !(cfg->wait_timeout_s > 0) ||
      cfg->inner_max_iter < 1 || !(cfg->inner_tol > 0) ||
      (cfg->stream_mode != NS_STREAM_RING && cfg->stream_mode != NS_STREAM_ZERO_COPY) ||
      (cfg->spring_tile_points != 0 && !spring_tile_ok(cfg->spring_tile_points, cfg->n_springs)) ||
      (cfg->spring_tile_blocks != 0 && cfg->spring_tile_blocks != 1 && cfg->spring_tile_blocks != 4) ||
      (cfg->multigrid != 0 && cfg->multigrid != 1) || (cfg->local_gather != 0 && cfg->local_gather != 1) ||
      cfg->l2_prefetch < 0 || cfg->l2_prefetch > 1 || cfg->stage_elements < -1 || cfg->stage_elements > 2 ||
      cfg->shared_members < 0 || cfg->shared_members > 65536 ||
      (cfg->shared_members > 1 && (cfg->scatter != NS_SCATTER_ATOMIC || cfg->multigrid)) ||
      (cfg->multigrid && (cfg->precision == NS_PREC_FP64 || cfg->coarse_max_iter < 1 || !(cfg->coarse_tol > 0)))) {
    g_create_err = "invalid configuration value";
    return NS_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
    cudaGetLastError();
    g_create_err = "no CUDA device " + std::to_string(cfg->device);
    return NS_ERR_CUDA;
  }
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    g_create_err = "cudaSetDevice failed";
    return NS_ERR_CUDA;
  }
  ns_ctx *c = new ns_ctx();
  c->cfg = *cfg;
  if (cudaStreamCreateWithFlags(&c->s_main, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->s_h2d, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->s_d2h, cudaStreamNonBlocking) != cudaSuccess) {
    g_create_err = "stream creation failed";
    ns_destroy(c);
    return NS_ERR_CUDA;
  }
  cudaEventCreateWithFlags(&c->ev_d2h_all, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&c->ev_sync, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  cudaEventCreate(&c->ev_adv0);
  cudaEventCreate(&c->ev_adv1);
  cudaEventCreate(&c->ev_stream_t0);
  cudaEventCreate(&c->ev_stream_t1);
  cudaEventCreateWithFlags(&c->ev_strain, cudaEventDisableTiming);
  const int R = cfg->ring_depth;
  c->ev_h2d = new cudaEvent_t[R];
  c->ev_comp = new cudaEvent_t[R];
  c->ev_d2h = new cudaEvent_t[R];
  for (int i = 0; i < R; ++i) {
    cudaEventCreateWithFlags(&c->ev_h2d[i], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&c->ev_comp[i], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&c->ev_d2h[i], cudaEventDisableTiming);
  }
  int arc = NS_OK;
  if ((arc = halloc(c, &c->sc_h, 3)) || (arc = halloc(c, &c->flag_h, 1)) || (arc = dalloc(c, &c->sc, 3)) ||
      (arc = dalloc(c, &c->flag_d, 1)) || (arc = dalloc(c, &c->op_A, 1)) || (arc = dalloc(c, &c->op_A16, 1)) ||
      (arc = dalloc(c, &c->op_K, 1)) || (arc = dalloc(c, &c->op_M, 1)) || (arc = dalloc(c, &c->op_Cr, 1)) ||
      (arc = dalloc(c, &c->op_rhs, 1)) || (arc = dalloc(c, &c->mats_d, kMaxMat)) ||
      (arc = dalloc(c, &c->spr_cnt, 3 * (size_t)kSpringCountSlots))) {
    g_create_err = c->err;  // the failing allocation's own code: pinned or device
    ns_destroy(c);
    return arc;
  }
  cudaMemsetAsync(c->sc, 0, 3 * sizeof(CgScalars), c->s_main);
  cudaMemsetAsync(c->spr_cnt, 0, 3 * kSpringCountSlots * sizeof(unsigned long long), c->s_main);
  cudaStreamSynchronize(c->s_main);
  c->sc_in = c->sc + 1;
  c->sc_c = c->sc + 2;
  *c->flag_h = 0;
  *out = c;
  return NS_OK;
}

int ns_upload_mesh(ns_ctx *c, int64_t N, const double *xyz, int64_t E, const int32_t *conn, const int32_t *mat) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (c->has_mesh) NS_SET(c, NS_ERR_INVALID_ARG, "mesh already uploaded");
  if (N <= 0 || E <= 0 || !xyz || !conn || !mat || N > INT32_MAX || E > INT32_MAX)
    NS_SET(c, NS_ERR_INVALID_ARG, "bad mesh sizes or null pointers");
  for (int64_t i = 0; i < E * 10; ++i)
    if (conn[i] < 0 || conn[i] >= N) NS_SET(c, NS_ERR_BAD_MESH, "connectivity index out of range");
  for (int64_t e = 0; e < E; ++e)
    if (mat[e] < 0 || mat[e] >= kMaxMat) NS_SET(c, NS_ERR_BAD_MESH, "material index out of range");
  int rc;
  cudaSetDevice(c->cfg.device);
  DevMesh &m = c->m;
  // members sharing this mesh: one copy of connectivity and geometry, per-member element
  // data and node vectors (member k's material of element e is table entry mat[e] + k nmb)
  const int32_t Ms = c->cfg.shared_members > 1 ? c->cfg.shared_members : 1;
  int32_t nmb = 1;
  for (int64_t e = 0; e < E; ++e) nmb = std::max(nmb, mat[e] + 1);
  if (Ms > 1 && (N * Ms > INT32_MAX || E * Ms > INT32_MAX))
    NS_SET(c, NS_ERR_INVALID_ARG, "shared members: too many nodes or elements in all");
  if (Ms > 1 && (int64_t)nmb * Ms > kMaxMat)
    NS_SET(c, NS_ERR_INVALID_ARG, "shared members: the material table would exceed " + std::to_string(kMaxMat));
  m.Msh = Ms;
  m.Eb = E;
  m.Nb = N;
  m.N = N * Ms;
  m.E = E * Ms;
  m.prefetch = (c->cfg.l2_prefetch && Ms == 1) ? 1 : 0;
  m.epg = pad64(E);
  m.epad = pad64(m.E);
  c->shared_nmat = nmb;
  std::vector<int32_t> soa((size_t)10 * m.epg, 0);
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < 10; ++a) soa[(size_t)a * m.epg + e] = conn[e * 10 + a];
  if ((rc = dalloc(c, &m.conn, soa.size())) || (rc = dalloc(c, &m.geom, 10 * m.epg)) ||
      (rc = dalloc(c, &m.geom32, 10 * m.epg)) || (rc = dalloc(c, &m.mat, m.epad)) || (rc = dalloc(c, &m.kerr, 1)) ||
      (rc = dalloc(c, &c->xyz_d, 3 * N)))
    return rc;
  CKC(c, cudaMemcpy(m.conn, soa.data(), soa.size() * 4, cudaMemcpyHostToDevice));
  if (Ms == 1) {
    CKC(c, cudaMemcpy(m.mat, mat, E * 4, cudaMemcpyHostToDevice));
  } else {
    std::vector<int32_t> mv((size_t)m.E);
    for (int32_t k = 0; k < Ms; ++k)
      for (int64_t e = 0; e < E; ++e) mv[(size_t)k * E + e] = mat[e] + k * nmb;
    CKC(c, cudaMemcpy(m.mat, mv.data(), mv.size() * 4, cudaMemcpyHostToDevice));
  }
  CKC(c, cudaMemcpy(c->xyz_d, xyz, N * 24, cudaMemcpyHostToDevice));
  CKC(c, cudaMemsetAsync(m.geom, 0, 10 * m.epg * 8, c->s_main));
  CKC(c, cudaMemsetAsync(m.geom32, 0, 10 * m.epg * 4, c->s_main));
  if (m.epad > m.E) CKC(c, cudaMemsetAsync(m.mat + m.E, 0, (m.epad - m.E) * 4, c->s_main));  // read by tile copies
  CKC(c, cudaMemsetAsync(m.kerr, 0, 4, c->s_main));
  CKC(c, cudaMemsetAsync(c->flag_d, 0, 4, c->s_main));
  LAUNCH(c, launch_geometry(m, c->xyz_d, c->flag_d, c->s_main));
  if (c->cfg.pair_operator) {
    if ((rc = dalloc(c, &m.geom2, 10 * (size_t)m.epg))) return rc;
    LAUNCH(c, launch_to_pairs(m.geom, m.geom2, 10 * m.epg, c->s_main));
  }
  CKC(c, cudaStreamSynchronize(c->s_main));
  int32_t bad = 0;
  CKC(c, cudaMemcpy(&bad, c->flag_d, 4, cudaMemcpyDeviceToHost));
  if (bad) NS_SET(c, NS_ERR_BAD_MESH, "element " + std::to_string(bad - 1) + " has a non-positive volume or a curved edge");
  // node vectors (every member's)
  const size_t n3 = 3 * (size_t)m.N;
  if ((rc = dalloc(c, &c->u, n3)) || (rc = dalloc(c, &c->v, n3)) || (rc = dalloc(c, &c->a, n3)) ||
      (rc = dalloc(c, &c->q, n3)) || (rc = dalloc(c, &c->du, n3)) || (rc = dalloc(c, &c->b, n3)) ||
      (rc = dalloc(c, &c->r, n3)) || (rc = dalloc(c, &c->z, n3)) || (rc = dalloc(c, &c->p, n3)) ||
      (rc = dalloc(c, &c->Ap, n3)) || (rc = dalloc(c, &c->Jd, 6 * (size_t)m.N)) ||
      (rc = dalloc(c, &c->Jinv, 6 * (size_t)m.N)) || (rc = dalloc(c, &c->Jinv32, 6 * (size_t)m.N)) ||
      (rc = dalloc(c, &c->eps, 48 * (size_t)m.E)))
    return rc;
  const size_t n4 = 4 * (size_t)m.N;  // inner FP32 vectors: [N][4] rows of 16 bytes
  if (c->cfg.precision != NS_PREC_FP64 &&
      ((rc = dalloc(c, &c->rin, n4)) || (rc = dalloc(c, &c->zin, n4)) || (rc = dalloc(c, &c->pin, n4)) ||
       (rc = dalloc(c, &c->xin, n4)) || (rc = dalloc(c, &c->Apin, n4))))
    return rc;
  for (double *x : {c->u, c->v, c->a, c->q, c->du}) CKC(c, cudaMemsetAsync(x, 0, n3 * 8, c->s_main));
  // colouring for the deterministic scatter
  int32_t nc = 0;
  if (c->cfg.scatter == NS_SCATTER_COLOUR) {
    std::vector<int32_t> col((size_t)E);
    if (host_colouring(E, N, conn, col.data(), &nc) != 0) NS_SET(c, NS_ERR_BAD_MESH, "more than 64 element colours");
    std::vector<int32_t> ids((size_t)E);
    m.ecol_off.assign(nc + 1, 0);
    for (int64_t e = 0; e < E; ++e) m.ecol_off[col[e] + 1]++;
    for (int k = 0; k < nc; ++k) m.ecol_off[k + 1] += m.ecol_off[k];
    std::vector<int64_t> fillp(m.ecol_off.begin(), m.ecol_off.end() - 1);
    for (int64_t e = 0; e < E; ++e) ids[fillp[col[e]]++] = (int32_t)e;
    if ((rc = dalloc(c, &m.ecol_ids, (size_t)E))) return rc;
    CKC(c, cudaMemcpy(m.ecol_ids, ids.data(), E * 4, cudaMemcpyHostToDevice));
  }
  c->part_pap_cap = nblk(m.E) + (int64_t)nc + 64 + nblk(1) * 2;
  if (c->cfg.local_gather && Ms == 1 && c->cfg.scatter == NS_SCATTER_ATOMIC) {
    // node lists of the locally gathered FP32 operator: per block of kBlock elements its
    // distinct nodes in first-use order, each element's nodes as indices into that list
    const int64_t nb = nblk(E);
    std::vector<int64_t> loff((size_t)nb + 1, 0);
    std::vector<int32_t> lnode;
    lnode.reserve((size_t)E * 4);
    std::vector<uint16_t> lc((size_t)10 * m.epg, 0);
    std::vector<int64_t> stamp((size_t)N, -1);
    std::vector<int32_t> local((size_t)N, 0);
    int32_t lmax = 0;
    for (int64_t b = 0; b < nb; ++b) {
      const int64_t e0 = b * kBlock, e1 = std::min<int64_t>(E, e0 + kBlock);
      int32_t k = 0;
      for (int64_t e = e0; e < e1 && k <= kLocalMaxNodes; ++e)
        for (int a = 0; a < 10; ++a) {
          const int32_t nd = conn[e * 10 + a];
          if (stamp[nd] != b) {
            stamp[nd] = b;
            local[nd] = k++;
            lnode.push_back(nd);
          }
          lc[(size_t)a * m.epg + e] = (uint16_t)local[nd];
        }
      lmax = std::max(lmax, k);
      loff[b + 1] = (int64_t)lnode.size();
      if (lmax > kLocalMaxNodes) break;
    }
    if (lmax <= kLocalMaxNodes) {
      if ((rc = dalloc(c, &m.lconn, lc.size())) || (rc = dalloc(c, &m.lnode, lnode.size())) ||
          (rc = dalloc(c, &m.loff, loff.size())))
        return rc;
      CKC(c, cudaMemcpy(m.lconn, lc.data(), lc.size() * 2, cudaMemcpyHostToDevice));
      CKC(c, cudaMemcpy(m.lnode, lnode.data(), lnode.size() * 4, cudaMemcpyHostToDevice));
      CKC(c, cudaMemcpy(m.loff, loff.data(), loff.size() * 8, cudaMemcpyHostToDevice));
      m.lmax = lmax;
    }  // else: node lists too long for shared memory (e.g. a shuffled numbering): direct gathers
  }
  if (c->cfg.multigrid) {  // coarse level of the two-level preconditioner
    MgLevel &g = c->mg;
    c->cid_h.assign((size_t)N, -1);
    std::vector<int32_t> par((size_t)2 * N);
    const int64_t Nc = host_coarse_map(E, N, conn, c->cid_h.data(), par.data());
    if (Nc <= 0) NS_SET(c, NS_ERR_BAD_MESH, "a node is a vertex of one element and an edge node of another");
    g.Nc = Nc;
    std::vector<int32_t> c1((size_t)4 * m.epad, 0);
    for (int64_t e = 0; e < E; ++e)
      for (int a = 0; a < 4; ++a) c1[(size_t)a * m.epad + e] = c->cid_h[conn[e * 10 + a]];
    // restriction lists: per coarse node the vertex itself, then its edge nodes in node order
    std::vector<int64_t> rptr((size_t)Nc + 1, 0);
    for (int64_t n = 0; n < N; ++n) {
      if (par[2 * n] < 0) NS_SET(c, NS_ERR_BAD_MESH, "node " + std::to_string(n) + " belongs to no element");
      rptr[par[2 * n] + 1]++;
      if (par[2 * n + 1] != par[2 * n]) rptr[par[2 * n + 1] + 1]++;
    }
    for (int64_t v = 0; v < Nc; ++v) rptr[v + 1] += rptr[v];
    std::vector<int32_t> rlist((size_t)rptr[Nc]);
    std::vector<int64_t> fill(rptr.begin(), rptr.end() - 1);
    for (int64_t n = 0; n < N; ++n) {
      if (par[2 * n] == par[2 * n + 1]) {
        rlist[fill[par[2 * n]]++] = (int32_t)n;
      } else {
        rlist[fill[par[2 * n]]++] = ~(int32_t)n;
        rlist[fill[par[2 * n + 1]]++] = ~(int32_t)n;
      }
    }
    if ((rc = dalloc(c, &g.conn1, c1.size())) || (rc = dalloc(c, &g.rptr, rptr.size())) ||
        (rc = dalloc(c, &g.rlist, std::max<size_t>(rlist.size(), 1))) || (rc = dalloc(c, &g.par, (size_t)N)) ||
        (rc = dalloc(c, &g.Dbar, 21 * (size_t)m.epad)) || (rc = dalloc(c, &g.Jd32, 6 * (size_t)Nc)) ||
        (rc = dalloc(c, &g.Jinv32, 6 * (size_t)Nc)) || (rc = dalloc(c, &g.x, 4 * (size_t)Nc)) ||
        (rc = dalloc(c, &g.r, 4 * (size_t)Nc)) || (rc = dalloc(c, &g.z, 4 * (size_t)Nc)) ||
        (rc = dalloc(c, &g.p, 4 * (size_t)Nc)) || (rc = dalloc(c, &g.Ap, 4 * (size_t)Nc)))
      return rc;
    CKC(c, cudaMemcpy(g.conn1, c1.data(), c1.size() * 4, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(g.rptr, rptr.data(), rptr.size() * 8, cudaMemcpyHostToDevice));
    if (!rlist.empty()) CKC(c, cudaMemcpy(g.rlist, rlist.data(), rlist.size() * 4, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(g.par, par.data(), par.size() * 4, cudaMemcpyHostToDevice));
    CKC(c, cudaMemsetAsync(g.Dbar, 0, 21 * m.epad * 4, c->s_main));
    for (float *x : {g.x, g.r, g.z, g.p, g.Ap}) CKC(c, cudaMemsetAsync(x, 0, 16 * Nc, c->s_main));
    CKC(c, cudaStreamSynchronize(c->s_main));
  }
  c->has_mesh = true;
  return NS_OK;
}

int ns_set_materials(ns_ctx *c, int32_t n, const ns_material *mats) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (!c->has_mesh) NS_SET(c, NS_ERR_STATE, "upload the mesh before the materials");
  if (n < 1 || n > kMaxMat || !mats) NS_SET(c, NS_ERR_INVALID_ARG, "bad material count");
  for (int i = 0; i < n; ++i) {
    const ns_material &m = mats[i];
    if (!(m.rho > 0) || !(m.vs > 0) || !(m.vp > m.vs * 1.1547005383792517) || !(m.gamma_ref > 0) || !(m.h_max > 0) ||
        !(m.h_max < 0.6) || !(m.rayleigh_h >= 0))
      NS_SET(c, NS_ERR_INVALID_ARG, "material " + std::to_string(i) + " has an invalid parameter");
  }
  std::vector<int32_t> mh((size_t)c->m.E);
  CKC(c, cudaMemcpy(mh.data(), c->m.mat, c->m.E * 4, cudaMemcpyDeviceToHost));
  for (int32_t x : mh)
    if (x >= n) NS_SET(c, NS_ERR_INVALID_ARG, "an element uses a material index beyond the table");
  // spring tables: q [S][6], T [S+1][21] = w q q^T (last row: their sum)
  const int S = c->cfg.n_springs;
  std::vector<double> qh(6 * (size_t)S), Th(21 * (size_t)(S + 1), 0.0);
  double w = 0;
  if (host_spring_directions(S, qh.data(), &w) != 0) NS_SET(c, NS_ERR_INVALID_ARG, "need at least 5 springs");
  for (int k = 0; k < S; ++k)
    for (int i = 0; i < 6; ++i)
      for (int j = i; j < 6; ++j) {
        const double t = w * qh[6 * k + i] * qh[6 * k + j];
        Th[21 * (size_t)k + sym6(i, j)] = t;
        Th[21 * (size_t)S + sym6(i, j)] += t;
      }
  c->nmat = n;
  c->mats_h.resize(n);
  for (int i = 0; i < n; ++i) host_material_constants(mats[i], c->cfg.rayleigh_f1, c->cfg.rayleigh_f2, &c->mats_h[i]);
  CKC(c, cudaMemcpy(c->mats_d, c->mats_h.data(), sizeof(MatConst) * n, cudaMemcpyHostToDevice));
  int rc;
  if ((rc = fill_opcoefs(c))) return rc;
  if (c->has_mat) return NS_OK;  // state already allocated: only the constants change
  std::vector<double> ph(kPowTabLen);
  host_pow_tables(ph.data());
  std::vector<float> pfh(kPowFLen);
  host_powf_tables(pfh.data());
  std::vector<float2> q2h(6 * (size_t)S);
  for (size_t i = 0; i < q2h.size(); ++i) {
    const float hi = (float)qh[i];
    q2h[i] = make_float2(hi, (float)(qh[i] - (double)hi));
  }
  std::vector<float2> T2h(21 * (size_t)S);
  for (size_t i = 0; i < T2h.size(); ++i) {
    const float hi = (float)Th[i];
    T2h[i] = make_float2(hi, (float)(Th[i] - (double)hi));
  }
  if ((rc = dalloc(c, &c->q_d, qh.size())) || (rc = dalloc(c, &c->T_d, Th.size())) ||
      (rc = dalloc(c, &c->pow_d, ph.size())) || (rc = dalloc(c, &c->T2_d, T2h.size())) ||
      (rc = dalloc(c, &c->powf_d, pfh.size())) || (rc = dalloc(c, &c->q2_d, q2h.size())))
    return rc;
  CKC(c, cudaMemcpy(c->T2_d, T2h.data(), T2h.size() * sizeof(float2), cudaMemcpyHostToDevice));
  {  // digits of T for the tensor-core tangent assembly
    std::vector<uint2> fr((size_t)7 * ((S + 15) / 16) * 3 * 32);
    int et[21];
    host_spring_digits(S, Th.data(), fr.data(), et);
    double tsc[21];
    for (int i = 0; i < 21; ++i) tsc[i] = ldexp(1.0, et[i] - 14);
    if ((rc = dalloc(c, &c->tfrag_d, fr.size())) || (rc = dalloc(c, &c->tsc_d, 21))) return rc;
    CKC(c, cudaMemcpy(c->tfrag_d, fr.data(), fr.size() * sizeof(uint2), cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(c->tsc_d, tsc, sizeof(tsc), cudaMemcpyHostToDevice));
    c->tab.tfrag = c->tfrag_d;
    c->tab.tsc = c->tsc_d;
    c->tab.tc = c->cfg.spring_tensor_cores ? 1 : 0;
  }
  CKC(c, cudaMemcpy(c->q2_d, q2h.data(), q2h.size() * sizeof(float2), cudaMemcpyHostToDevice));
  CKC(c, cudaMemcpy(c->q_d, qh.data(), qh.size() * 8, cudaMemcpyHostToDevice));
  CKC(c, cudaMemcpy(c->T_d, Th.data(), Th.size() * 8, cudaMemcpyHostToDevice));
  CKC(c, cudaMemcpy(c->pow_d, ph.data(), ph.size() * 8, cudaMemcpyHostToDevice));
  CKC(c, cudaMemcpy(c->powf_d, pfh.data(), pfh.size() * 4, cudaMemcpyHostToDevice));
  c->tab.q = c->q_d;
  c->tab.T = c->T_d;
  c->tab.pow = c->pow_d;
  c->tab.powf = c->powf_d;
  c->tab.T2 = c->T2_d;
  c->tab.q2 = c->q2_d;
  c->tab.S = S;
  c->tab.tp = c->cfg.spring_tile_points;
  c->tab.cnt = c->spr_cnt;
  c->tab.minb = c->cfg.spring_tile_blocks == 4 ? 4 : 1;
  // tangent D (element SoA [84][epad]) and spring state placement
  const int64_t E = c->m.E, epad = c->m.epad;
  if ((rc = dalloc(c, &c->D, 84 * (size_t)epad))) return rc;
  if (c->cfg.pair_operator && (rc = dalloc(c, &c->D2, 84 * (size_t)epad))) return rc;
  if (c->cfg.precision == NS_PREC_FP64_IR && (rc = dalloc(c, &c->D32, 84 * (size_t)epad))) return rc;
  if (c->cfg.precision == NS_PREC_FP64_IR16) {
    if ((rc = dalloc(c, &c->D16, 84 * (size_t)epad))) return rc;
    CKC(c, cudaMemsetAsync(c->D16, 0, 84 * epad * 2, c->s_main));
  }
  CKC(c, cudaMemsetAsync(c->D, 0, 84 * epad * 8, c->s_main));
  LAUNCH(c, launch_elastic_D(c->tab, c->mats_d, c->m.mat, c->D, epad, 0, E, c->s_main));
  const int64_t per_elem = ns_state_bytes(1, S);
  if (c->cfg.device_state_budget < 0)
    c->E_res = E;
  else
    c->E_res = std::min<int64_t>(E, c->cfg.device_state_budget / per_elem);
  const int64_t S4 = 4 * (int64_t)S;
  if ((rc = alloc_soa(c, c->st, std::max<int64_t>(1, c->E_res * S4), false))) return rc;
  if (c->E_res < E) {
    if ((rc = alloc_soa(c, c->hst, (E - c->E_res) * S4, true))) return rc;
    if (c->cfg.stream_mode == NS_STREAM_ZERO_COPY) {
      void *d = nullptr;
      auto dev_of = [&](void *h) -> void * {
        d = nullptr;
        return cudaHostGetDevicePointer(&d, h, 0) == cudaSuccess ? d : nullptr;
      };
      c->hst_dev.tau = (double *)dev_of(c->hst.tau);
      c->hst_dev.gR = (double *)dev_of(c->hst.gR);
      c->hst_dev.tR = (double *)dev_of(c->hst.tR);
      c->hst_dev.gmax = (double *)dev_of(c->hst.gmax);
      c->hst_dev.dir = (int32_t *)dev_of(c->hst.dir);
      c->hst_dev.mode = (int32_t *)dev_of(c->hst.mode);
      if (!c->hst_dev.tau || !c->hst_dev.gR || !c->hst_dev.tR || !c->hst_dev.gmax || !c->hst_dev.dir ||
          !c->hst_dev.mode) {
        cudaGetLastError();
        NS_SET(c, NS_ERR_CUDA, "pinned state has no device address (zero-copy unavailable)");
      }
    } else {
      c->ring.resize(c->cfg.ring_depth);
      for (auto &rb : c->ring)
        if ((rc = alloc_soa(c, rb, std::min<int64_t>(c->cfg.chunk_elems, E - c->E_res) * S4, false))) return rc;
    }
  }
  c->stats.resident_elems = c->E_res;
  c->stats.streamed_elems = E - c->E_res;
  CKC(c, cudaStreamSynchronize(c->s_main));
  c->has_mat = true;
  return NS_OK;
}

int ns_set_boundary(ns_ctx *c, int64_t F, const int32_t *faces, const int32_t *face_elem, const int32_t *face_kind,
                    int64_t Ns, const int32_t *surf) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (!c->has_mesh) NS_SET(c, NS_ERR_STATE, "upload the mesh before the boundary");
  if (c->has_bnd) NS_SET(c, NS_ERR_INVALID_ARG, "boundary already set");
  if (F < 0 || Ns < 0 || (F > 0 && (!faces || !face_elem || !face_kind)) || (Ns > 0 && !surf))
    NS_SET(c, NS_ERR_INVALID_ARG, "bad boundary sizes or null pointers");
  DevMesh &m = c->m;
  for (int64_t i = 0; i < F * 6; ++i)
    if (faces[i] < 0 || faces[i] >= m.Nb) NS_SET(c, NS_ERR_BAD_MESH, "face node index out of range");
  for (int64_t f = 0; f < F; ++f)
    if (face_elem[f] < 0 || face_elem[f] >= m.Eb || (face_kind[f] != 0 && face_kind[f] != 1))
      NS_SET(c, NS_ERR_BAD_MESH, "bad face element or kind");
  for (int64_t i = 0; i < Ns; ++i)
    if (surf[i] < 0 || surf[i] >= m.Nb) NS_SET(c, NS_ERR_BAD_MESH, "surface node index out of range");
  int rc;
  // with shared members: one copy of the faces' nodes, geometry and kinds; their materials
  // and surface nodes per member, member after member
  const int32_t Ms = m.Msh;
  m.Fb = F;
  m.F = F * Ms;
  m.fpg = pad64(std::max<int64_t>(F, 1));
  m.fpad = pad64(std::max<int64_t>(m.F, 1));
  m.Ns = Ns * Ms;
  std::vector<int32_t> mh((size_t)m.E);
  CKC(c, cudaMemcpy(mh.data(), m.mat, m.E * 4, cudaMemcpyDeviceToHost));
  std::vector<int32_t> soa((size_t)6 * m.fpg, 0), fm((size_t)std::max<int64_t>(m.F, 1), 0);
  c->face_elem_h.assign((size_t)m.F, 0);
  for (int64_t f = 0; f < F; ++f)
    for (int a = 0; a < 6; ++a) soa[(size_t)a * m.fpg + f] = faces[f * 6 + a];
  for (int32_t k = 0; k < Ms; ++k)
    for (int64_t f = 0; f < F; ++f) {
      c->face_elem_h[(size_t)k * F + f] = (int32_t)(k * m.Eb + face_elem[f]);
      fm[(size_t)k * F + f] = mh[(size_t)k * m.Eb + face_elem[f]];
    }
  std::vector<int32_t> sv((size_t)std::max<int64_t>(m.Ns, 1), 0);
  for (int32_t k = 0; k < Ms; ++k)
    for (int64_t i = 0; i < Ns; ++i) sv[(size_t)k * Ns + i] = (int32_t)(surf[i] + k * m.Nb);
  if ((rc = dalloc(c, &m.fnode, soa.size())) || (rc = dalloc(c, &m.fgeom, 4 * (size_t)m.fpg)) ||
      (rc = dalloc(c, &m.fmat, fm.size())) || (rc = dalloc(c, &m.fkind, (size_t)std::max<int64_t>(F, 1))) ||
      (rc = dalloc(c, &m.surf, sv.size())))
    return rc;
  CKC(c, cudaMemcpy(m.fnode, soa.data(), soa.size() * 4, cudaMemcpyHostToDevice));
  CKC(c, cudaMemcpy(m.fmat, fm.data(), fm.size() * 4, cudaMemcpyHostToDevice));
  if (F > 0) CKC(c, cudaMemcpy(m.fkind, face_kind, F * 4, cudaMemcpyHostToDevice));
  if (m.Ns > 0) CKC(c, cudaMemcpy(m.surf, sv.data(), m.Ns * 4, cudaMemcpyHostToDevice));
  LAUNCH(c, launch_face_geometry(m, c->xyz_d, c->s_main));
  if (c->cfg.multigrid) {
    std::vector<int32_t> cf((size_t)3 * m.fpad, 0);
    for (int64_t f = 0; f < F; ++f)
      for (int a = 0; a < 3; ++a) {
        const int32_t v = c->cid_h[faces[f * 6 + a]];
        if (v < 0) NS_SET(c, NS_ERR_BAD_MESH, "a boundary face vertex is an edge node of the mesh");
        cf[(size_t)a * m.fpad + f] = v;
      }
    if ((rc = dalloc(c, &c->mg.cfnode, cf.size()))) return rc;
    CKC(c, cudaMemcpy(c->mg.cfnode, cf.data(), cf.size() * 4, cudaMemcpyHostToDevice));
  }
  CKC(c, cudaStreamSynchronize(c->s_main));
  if (c->cfg.scatter == NS_SCATTER_COLOUR && F > 0) {
    // greedy colouring of the faces (6 nodes each) in face order (no shared members here)
    std::vector<uint64_t> used((size_t)m.N, 0);
    std::vector<int32_t> col((size_t)F);
    int nc = 0;
    for (int64_t f = 0; f < F; ++f) {
      uint64_t taken = 0;
      for (int a = 0; a < 6; ++a) taken |= used[faces[f * 6 + a]];
      if (~taken == 0) NS_SET(c, NS_ERR_BAD_MESH, "more than 64 face colours");
      const int k = __builtin_ctzll(~taken);
      col[f] = k;
      nc = std::max(nc, k + 1);
      for (int a = 0; a < 6; ++a) used[faces[f * 6 + a]] |= 1ull << k;
    }
    m.fcol_off.assign(nc + 1, 0);
    for (int64_t f = 0; f < F; ++f) m.fcol_off[col[f] + 1]++;
    for (int k = 0; k < nc; ++k) m.fcol_off[k + 1] += m.fcol_off[k];
    std::vector<int64_t> fillp(m.fcol_off.begin(), m.fcol_off.end() - 1);
    std::vector<int32_t> ids((size_t)F);
    for (int64_t f = 0; f < F; ++f) ids[fillp[col[f]]++] = (int32_t)f;
    if ((rc = dalloc(c, &m.fcol_ids, (size_t)F))) return rc;
    CKC(c, cudaMemcpy(m.fcol_ids, ids.data(), F * 4, cudaMemcpyHostToDevice));
    c->part_pap_cap += nblk(F) + nc;
  } else {
    c->part_pap_cap += nblk(std::max<int64_t>(m.F, 1));
  }
  c->ring_steps = c->cfg.surface_ring_steps;
  const size_t rs = (size_t)c->ring_steps * 3 * (size_t)std::max<int64_t>(m.Ns, 1);
  if ((rc = dalloc(c, &c->surf_u, rs)) || (rc = dalloc(c, &c->surf_v, rs)) || (rc = dalloc(c, &c->surf_a, rs)))
    return rc;
  if ((rc = dalloc(c, &c->part, (size_t)(c->part_pap_cap + 3 * vec_blocks(m.N))))) return rc;
  c->has_bnd = true;
  if (Ms > 1) {  // the members are implied: member k owns elements [k Eb, (k+1) Eb) and nodes [k Nb, (k+1) Nb)
    std::vector<int64_t> eo(Ms + 1), no(Ms + 1);
    for (int32_t k = 0; k <= Ms; ++k) {
      eo[k] = k * m.Eb;
      no[k] = k * m.Nb;
    }
    if ((rc = setup_members(c, Ms, eo.data(), no.data())) != NS_OK) return rc;
  }
  return NS_OK;
}

int ns_set_ground_motion(ns_ctx *c, int64_t ns_, double dt, const double *acc) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (ns_ < 1 || !acc) NS_SET(c, NS_ERR_INVALID_ARG, "need at least one acceleration sample");
  if (!(fabs(dt - c->cfg.dt) <= 1e-12 * c->cfg.dt)) NS_SET(c, NS_ERR_INVALID_ARG, "record dt differs from the step dt");
  // trapezoidal input velocity, v(0) = 0; one extra entry for the first step past the record
  std::vector<double> vin(3 * (size_t)(ns_ + 1), 0.0);
  host_input_velocity(acc, ns_, dt, vin.data());
  int rc;
  dfree(c->vin_d);
  // [M][n_vin][3]: every member starts with this record
  if ((rc = dalloc(c, &c->vin_d, vin.size() * (size_t)c->M))) return rc;
  for (int m = 0; m < c->M; ++m)
    CKC(c, cudaMemcpy(c->vin_d + (size_t)m * vin.size(), vin.data(), vin.size() * 8, cudaMemcpyHostToDevice));
  c->n_vin = ns_ + 1;
  c->has_motion = true;
  return NS_OK;
}

int ns_set_member_ground_motion(ns_ctx *c, int32_t member, int64_t ns_, double dt, const double *acc) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (!c->has_motion) NS_SET(c, NS_ERR_STATE, "set the common record (ns_set_ground_motion) first");
  if (member < 0 || member >= c->M) NS_SET(c, NS_ERR_INVALID_ARG, "member index out of range");
  if (ns_ + 1 != c->n_vin || !acc) NS_SET(c, NS_ERR_INVALID_ARG, "member records must have the common record's length");
  if (!(fabs(dt - c->cfg.dt) <= 1e-12 * c->cfg.dt)) NS_SET(c, NS_ERR_INVALID_ARG, "record dt differs from the step dt");
  std::vector<double> vin(3 * (size_t)(ns_ + 1), 0.0);
  host_input_velocity(acc, ns_, dt, vin.data());
  CKC(c, cudaMemcpy(c->vin_d + (size_t)member * vin.size(), vin.data(), vin.size() * 8, cudaMemcpyHostToDevice));
  return NS_OK;
}

int ns_set_members(ns_ctx *c, int32_t M, const int64_t *elem_off, const int64_t *node_off) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (!c->has_mesh || !c->has_bnd) NS_SET(c, NS_ERR_STATE, "upload the mesh and the boundary before the members");
  if (c->has_motion || c->step > 0 || c->M > 1) NS_SET(c, NS_ERR_STATE, "members must be set before the ground motion");
  if (c->cfg.scatter != NS_SCATTER_ATOMIC) NS_SET(c, NS_ERR_INVALID_ARG, "members need the atomic scatter");
  if (c->cfg.multigrid) NS_SET(c, NS_ERR_INVALID_ARG, "the two-level preconditioner serves one member only");
  if (c->m.Msh > 1) NS_SET(c, NS_ERR_STATE, "the members of a shared mesh are already set");
  if (M < 1 || M > 65536 || !elem_off || !node_off) NS_SET(c, NS_ERR_INVALID_ARG, "bad member count");
  const DevMesh &m = c->m;
  if (elem_off[0] != 0 || elem_off[M] != m.E || node_off[0] != 0 || node_off[M] != m.N)
    NS_SET(c, NS_ERR_INVALID_ARG, "member ranges must cover all elements and nodes");
  for (int k = 0; k < M; ++k)
    if (elem_off[k + 1] <= elem_off[k] || node_off[k + 1] <= node_off[k])
      NS_SET(c, NS_ERR_INVALID_ARG, "every member needs elements and nodes");
  // every element's nodes in its member's node range
  std::vector<int32_t> conn((size_t)10 * m.epad);
  CKC(c, cudaMemcpy(conn.data(), m.conn, conn.size() * 4, cudaMemcpyDeviceToHost));
  for (int k = 0; k < M; ++k)
    for (int64_t e = elem_off[k]; e < elem_off[k + 1]; ++e)
      for (int a = 0; a < 10; ++a) {
        const int64_t nd = conn[(size_t)a * m.epad + e];
        if (nd < node_off[k] || nd >= node_off[k + 1])
          NS_SET(c, NS_ERR_BAD_MESH, "element " + std::to_string(e) + " uses a node of another member");
      }
  return setup_members(c, M, elem_off, node_off);
}

// Member ranges (already validated): launch cuts, per-member CG scalars and partial sums.
static int setup_members(ns_ctx *c, int32_t M, const int64_t *elem_off, const int64_t *node_off) {
  const DevMesh &m = c->m;
  // faces ordered by member
  std::vector<int32_t> fmem((size_t)std::max<int64_t>(m.F, 1), 0);
  std::vector<int64_t> foff(M + 1, 0);
  for (int64_t f = 0; f < m.F; ++f) {
    const int64_t e = c->face_elem_h[f];
    const int k = (int)(std::upper_bound(elem_off, elem_off + M + 1, e) - elem_off) - 1;
    if (f > 0 && k < fmem[f - 1]) NS_SET(c, NS_ERR_INVALID_ARG, "boundary faces must be ordered by member");
    fmem[f] = k;
    foff[k + 1]++;
  }
  for (int k = 0; k < M; ++k) foff[k + 1] += foff[k];
  c->moff_e.assign(elem_off, elem_off + M + 1);
  c->moff_n.assign(node_off, node_off + M + 1);
  c->moff_f = foff;
  // launch cuts: element and face blocks of kBlock, node-vector blocks in proportion to size
  std::vector<Seg> es, fs, vs;
  std::vector<int32_t> eo(M + 1, 0), fo(M + 1, 0), vo(M + 1, 0);
  const int vcap = 152 * 8;
  for (int k = 0; k < M; ++k) {
    for (int64_t a = elem_off[k]; a < elem_off[k + 1]; a += kBlock)
      es.push_back(Seg{a, std::min<int64_t>(a + kBlock, elem_off[k + 1]), k, 0});
    for (int64_t a = foff[k]; a < foff[k + 1]; a += kBlock)
      fs.push_back(Seg{a, std::min<int64_t>(a + kBlock, foff[k + 1]), k, 0});
    const int64_t nk = node_off[k + 1] - node_off[k];
    int64_t bk = std::min<int64_t>((nk + kBlock - 1) / kBlock, 1 + (int64_t)((double)vcap * nk / m.N));
    bk = std::max<int64_t>(bk, 1);
    for (int64_t b = 0; b < bk; ++b)
      vs.push_back(Seg{node_off[k] + nk * b / bk, node_off[k] + nk * (b + 1) / bk, k, 0});
    eo[k + 1] = (int32_t)es.size();
    fo[k + 1] = (int32_t)fs.size();
    vo[k + 1] = (int32_t)vs.size();
  }
  int rc;
  auto up = [&](auto **dst, const auto &src) -> int {
    dfree(*dst);
    int r = dalloc(c, dst, std::max<size_t>(src.size(), 1));
    if (r) return r;
    if (!src.empty()) {
      cudaError_t e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(src[0]), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        c->err = cudaGetErrorString(e);
        return NS_ERR_CUDA;
      }
    }
    return NS_OK;
  };
  if ((rc = up(&c->eseg_d, es)) || (rc = up(&c->fseg_d, fs)) || (rc = up(&c->vseg_d, vs)) ||
      (rc = up(&c->eoff_d, eo)) || (rc = up(&c->foff_d, fo)) || (rc = up(&c->voff_d, vo)) ||
      (rc = up(&c->fmem_d, fmem)))
    return rc;
  c->neseg = (int)es.size();
  c->nfseg = (int)fs.size();
  c->nvseg = (int)vs.size();
  c->m.eseg32 = true;
  for (const Seg &sgm : es) c->m.eseg32 = c->m.eseg32 && (sgm.a0 % 32 == 0);
  // per-member CG scalars (outer [0, M), inner [M, 2M)) and partial-sum space
  destroy_graphs(c);
  dfree(c->sc);
  hfree(c->sc_h);
  if ((rc = dalloc(c, &c->sc, 2 * (size_t)M)) || (rc = halloc(c, &c->sc_h, 2 * (size_t)M))) return rc;
  CKC(c, cudaMemsetAsync(c->sc, 0, 2 * M * sizeof(CgScalars), c->s_main));
  c->sc_in = c->sc + M;
  c->part_pap_cap = std::max<int64_t>(c->part_pap_cap, (int64_t)c->neseg + c->nfseg + 64);
  dfree(c->part);
  if ((rc = dalloc(c, &c->part, (size_t)(c->part_pap_cap + 3 * std::max(c->nvseg, vec_blocks(m.N)))))) return rc;
  CKC(c, cudaStreamSynchronize(c->s_main));
  c->M = M;
  c->member_iters.assign(M, 0);
  return NS_OK;
}

int ns_set_member_springs(ns_ctx *c, int32_t M, const int32_t *S) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (!c->has_mat || !c->has_bnd || c->M < 2 || c->m.Msh > 1)
    NS_SET(c, NS_ERR_STATE, "set the materials and the members (ns_set_members) first");
  if (c->step > 0 || !c->mS.empty()) NS_SET(c, NS_ERR_STATE, "member springs are set once, before the first step");
  if (c->E_res < c->m.E) NS_SET(c, NS_ERR_INVALID_ARG, "members with their own springs keep all state resident");
  if (M != c->M || !S) NS_SET(c, NS_ERR_INVALID_ARG, "one spring count per member");
  for (int m = 0; m < M; ++m)
    if (S[m] < 5 || !spring_tile_ok(spring_tile_default(S[m]), S[m]))
      NS_SET(c, NS_ERR_INVALID_ARG, "member " + std::to_string(m) + ": bad spring count");
  int rc;
  if ((rc = sync_all(c)) != NS_OK) return rc;
  std::vector<int64_t> off(M + 1, 0);
  for (int m = 0; m < M; ++m) off[m + 1] = off[m] + 4 * (c->moff_e[m + 1] - c->moff_e[m]) * (int64_t)S[m];
  std::vector<SpringTables> tabs(M);
  std::vector<void *> mem;
  auto up = [&](const void *src, size_t bytes) -> void * {
    void *d = nullptr;
    if (cudaMalloc(&d, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    mem.push_back(d);
    if (cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
    return d;
  };
  for (int m = 0; m < M && rc == NS_OK; ++m) {
    const int Sm = S[m];
    std::vector<double> qh(6 * (size_t)Sm), Th(21 * (size_t)(Sm + 1), 0.0);
    double w = 0;
    host_spring_directions(Sm, qh.data(), &w);
    for (int k = 0; k < Sm; ++k)
      for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) {
          const double t = w * qh[6 * k + i] * qh[6 * k + j];
          Th[21 * (size_t)k + sym6(i, j)] = t;
          Th[21 * (size_t)Sm + sym6(i, j)] += t;
        }
    std::vector<float2> q2h(6 * (size_t)Sm), T2h(21 * (size_t)Sm);
    for (size_t i = 0; i < q2h.size(); ++i) q2h[i] = make_float2((float)qh[i], (float)(qh[i] - (double)(float)qh[i]));
    for (size_t i = 0; i < T2h.size(); ++i) T2h[i] = make_float2((float)Th[i], (float)(Th[i] - (double)(float)Th[i]));
    SpringTables t = c->tab;  // power tables, launch shape and counters as the context's
    t.S = Sm;
    t.tc = 0;  // the tangent in double-float sums
    t.tfrag = nullptr;
    t.tsc = nullptr;
    t.tp = 0;  // the size heuristic for this spring count
    t.q = (const double *)up(qh.data(), qh.size() * 8);
    t.T = (const double *)up(Th.data(), Th.size() * 8);
    t.q2 = (const float2 *)up(q2h.data(), q2h.size() * sizeof(float2));
    t.T2 = (const float2 *)up(T2h.data(), T2h.size() * sizeof(float2));
    if (!t.q || !t.T || !t.q2 || !t.T2) {
      c->err = "allocation of the member spring tables failed";
      rc = NS_ERR_OOM_DEVICE;
    }
    tabs[m] = t;
  }
  SpringSoA st;
  if (rc == NS_OK) rc = alloc_soa(c, st, std::max<int64_t>(1, off[M]), false);
  if (rc != NS_OK) {
    for (void *p : mem) cudaFree(p);
    return rc;
  }
  for (int k = 0; k < ns_ctx::kMemberStreams; ++k) {
    if (!c->s_mem[k]) CKC(c, cudaStreamCreateWithFlags(&c->s_mem[k], cudaStreamNonBlocking));
    if (!c->ev_mem[k]) CKC(c, cudaEventCreateWithFlags(&c->ev_mem[k], cudaEventDisableTiming));
  }
  if (!c->ev_fork) CKC(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  free_soa(c->st, false);
  c->st = st;
  c->mS.assign(S, S + M);
  c->spr_off = off;
  c->mtab = tabs;
  c->mtab_mem = mem;
  for (int m = 0; m < M; ++m)  // elastic tangent of each member's spring set
    LAUNCH(c, launch_elastic_D(c->mtab[m], c->mats_d, c->m.mat, c->D, c->m.epad, c->moff_e[m], c->moff_e[m + 1],
                               c->s_main));
  c->stats.resident_elems = c->m.E;
  return sync_stream(c, c->s_main);
}

int ns_get_member_iters(ns_ctx *c, int32_t M, int32_t *iters) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (M != c->M || !iters) NS_SET(c, NS_ERR_INVALID_ARG, "member count differs from the context's");
  for (int k = 0; k < M; ++k) iters[k] = k < (int)c->member_iters.size() ? c->member_iters[k] : 0;
  return NS_OK;
}

int ns_advance(ns_ctx *c, int64_t nsteps) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (!c->has_mesh || !c->has_mat || !c->has_bnd || !c->has_motion)
    NS_SET(c, NS_ERR_STATE, "mesh, materials, boundary and ground motion must be set before advancing");
  if (nsteps < 0) NS_SET(c, NS_ERR_INVALID_ARG, "negative step count");
  cudaSetDevice(c->cfg.device);
  CKC(c, cudaEventRecord(c->ev_adv0, c->s_main));
  for (int64_t k = 0; k < nsteps; ++k) {
    c->timer.reset();
    c->tev.clear();
    int rc = one_step(c);
    if (rc != NS_OK) {
      sync_all(c);
      c->prefetched = false;  // chunks loaded for the failed step are loaded again
      return rc;
    }
    if ((rc = sync_all(c)) != NS_OK) return rc;
    if (c->cfg.timing) {
      flush_times(c);
      if (n_chunks(c) > 0) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, c->ev_stream_t0, c->ev_stream_t1) == cudaSuccess) c->stats.ms_stream_wall += ms;
        cudaGetLastError();
      }
    }
  }
  // join the copy streams into the main stream so the end event covers all device work
  CKC(c, cudaEventRecord(c->ev_join, c->s_h2d));
  CKC(c, cudaStreamWaitEvent(c->s_main, c->ev_join, 0));
  CKC(c, cudaEventRecord(c->ev_join, c->s_d2h));
  CKC(c, cudaStreamWaitEvent(c->s_main, c->ev_join, 0));
  CKC(c, cudaEventRecord(c->ev_adv1, c->s_main));
  int rc2 = wait_event(c, c->ev_adv1);
  if (rc2 != NS_OK) return rc2;
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, c->ev_adv0, c->ev_adv1) == cudaSuccess) c->stats.ms_advance += ms;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) NS_SET(c, NS_ERR_CUDA, std::string("device error: ") + cudaGetErrorString(e));
  {
    unsigned long long cnt[3 * kSpringCountSlots];
    CKC(c, cudaMemcpy(cnt, c->spr_cnt, sizeof(cnt), cudaMemcpyDeviceToHost));
    int64_t tot[3] = {0, 0, 0};
    for (int i = 0; i < kSpringCountSlots; ++i)
      for (int k = 0; k < 3; ++k) tot[k] += (int64_t)cnt[3 * i + k];
    c->stats.spring_moved = tot[0];
    c->stats.spring_reversals = tot[1];
    c->stats.spring_fp64_roots = tot[2];
  }
  int32_t kerr = 0;
  CKC(c, cudaMemcpy(&kerr, c->m.kerr, 4, cudaMemcpyDeviceToHost));
  if (kerr) NS_SET(c, NS_ERR_TIMEOUT, "a kernel's bounded wait for its shared-memory copies gave up");
  return NS_OK;
}

int ns_read_surface(ns_ctx *c, int64_t step0, int64_t nsteps, double *u, double *v, double *a) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (!c->has_bnd) NS_SET(c, NS_ERR_STATE, "no boundary set");
  if (nsteps < 0 || step0 < 1 || step0 + nsteps - 1 > c->step || step0 <= c->step - c->ring_steps)
    NS_SET(c, NS_ERR_INVALID_ARG, "requested steps are not in the surface ring");
  int rc;
  if ((rc = sync_all(c)) != NS_OK) return rc;
  const int64_t blk = c->m.Ns * 3;
  for (int64_t k = 0; k < nsteps; ++k) {
    const int64_t slot = (step0 + k - 1) % c->ring_steps;
    if (u) CKC(c, cudaMemcpy(u + k * blk, c->surf_u + slot * blk, blk * 8, cudaMemcpyDeviceToHost));
    if (v) CKC(c, cudaMemcpy(v + k * blk, c->surf_v + slot * blk, blk * 8, cudaMemcpyDeviceToHost));
    if (a) CKC(c, cudaMemcpy(a + k * blk, c->surf_a + slot * blk, blk * 8, cudaMemcpyDeviceToHost));
  }
  return NS_OK;
}

namespace {
struct SpringRec {
  double tau, gR, tR, gmax;
  int32_t dir, mode;
};
static_assert(sizeof(SpringRec) == 40, "40-byte spring record");

// gather springs [s0, s0 + n) of the global order into host SoA buffers
int state_to_host(ns_ctx *c, int64_t s0, int64_t n, SpringSoA &h) {
  const int64_t res_n = c->E_res * 4 * (int64_t)c->tab.S;
  for (int64_t s = s0; s < s0 + n;) {
    const int64_t off = s - s0;
    if (s < res_n) {
      const int64_t cnt = std::min(s0 + n, res_n) - s;
      int rc = copy_soa(c, h, off, c->st, s, cnt, cudaMemcpyDeviceToHost, c->s_main);
      if (rc) return rc;
      s += cnt;
    } else {
      const int64_t cnt = s0 + n - s;
      memcpy(h.tau + off, c->hst.tau + (s - res_n), cnt * 8);
      memcpy(h.gR + off, c->hst.gR + (s - res_n), cnt * 8);
      memcpy(h.tR + off, c->hst.tR + (s - res_n), cnt * 8);
      memcpy(h.gmax + off, c->hst.gmax + (s - res_n), cnt * 8);
      memcpy(h.dir + off, c->hst.dir + (s - res_n), cnt * 4);
      memcpy(h.mode + off, c->hst.mode + (s - res_n), cnt * 4);
      s += cnt;
    }
  }
  return sync_stream(c, c->s_main);
}

int state_from_host(ns_ctx *c, int64_t s0, int64_t n, const SpringSoA &h) {
  const int64_t res_n = c->E_res * 4 * (int64_t)c->tab.S;
  for (int64_t s = s0; s < s0 + n;) {
    const int64_t off = s - s0;
    if (s < res_n) {
      const int64_t cnt = std::min(s0 + n, res_n) - s;
      int rc = copy_soa(c, c->st, s, h, off, cnt, cudaMemcpyHostToDevice, c->s_main);
      if (rc) return rc;
      s += cnt;
    } else {
      const int64_t cnt = s0 + n - s;
      memcpy(c->hst.tau + (s - res_n), h.tau + off, cnt * 8);
      memcpy(c->hst.gR + (s - res_n), h.gR + off, cnt * 8);
      memcpy(c->hst.tR + (s - res_n), h.tR + off, cnt * 8);
      memcpy(c->hst.gmax + (s - res_n), h.gmax + off, cnt * 8);
      memcpy(c->hst.dir + (s - res_n), h.dir + off, cnt * 4);
      memcpy(c->hst.mode + (s - res_n), h.mode + off, cnt * 4);
      s += cnt;
    }
  }
  return sync_stream(c, c->s_main);
}

struct HostSoA {
  std::vector<double> tau, gR, tR, gmax;
  std::vector<int32_t> dir, mode;
  SpringSoA view;
  explicit HostSoA(int64_t n) : tau(n), gR(n), tR(n), gmax(n), dir(n), mode(n) {
    view.tau = tau.data(); view.gR = gR.data(); view.tR = tR.data(); view.gmax = gmax.data();
    view.dir = dir.data(); view.mode = mode.data();
  }
};

void unpack_D(const std::vector<double> &Dsoa, int64_t epad_src, int64_t e_local, int64_t e_src, double *out36x4) {
  for (int q = 0; q < 4; ++q)
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) out36x4[q * 36 + i * 6 + j] = Dsoa[(size_t)(q * 21 + sym6(i, j)) * epad_src + e_local];
  (void)e_src;
}
}  // namespace

int ns_read_state(ns_ctx *c, int64_t e0, int64_t n, void *theta, double *D) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (!c->has_mat) NS_SET(c, NS_ERR_STATE, "no state yet");
  if (!c->mS.empty() && theta) NS_SET(c, NS_ERR_STATE, "members with their own springs: spring state not readable");
  if (e0 < 0 || n < 0 || e0 + n > c->m.E) NS_SET(c, NS_ERR_INVALID_ARG, "element range out of bounds");
  int rc;
  if ((rc = sync_all(c)) != NS_OK) return rc;
  const int64_t S4 = 4 * (int64_t)c->tab.S;
  if (theta && n > 0) {
    HostSoA h(n * S4);
    if ((rc = state_to_host(c, e0 * S4, n * S4, h.view))) return rc;
    SpringRec *out = (SpringRec *)theta;
    for (int64_t i = 0; i < n * S4; ++i) out[i] = {h.tau[i], h.gR[i], h.tR[i], h.gmax[i], h.dir[i], h.mode[i]};
  }
  if (D && n > 0) {
    std::vector<double> tmp((size_t)84 * n);
    for (int k = 0; k < 84; ++k)
      CKC(c, cudaMemcpy(tmp.data() + (size_t)k * n, c->D + (size_t)k * c->m.epad + e0, n * 8, cudaMemcpyDeviceToHost));
    for (int64_t e = 0; e < n; ++e) unpack_D(tmp, n, e, e0 + e, D + e * 144);
  }
  return NS_OK;
}

int ns_write_state(ns_ctx *c, int64_t e0, int64_t n, const void *theta, const double *D) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (!c->has_mat) NS_SET(c, NS_ERR_STATE, "no state yet");
  if (!c->mS.empty() && theta) NS_SET(c, NS_ERR_STATE, "members with their own springs: spring state not writable");
  if (e0 < 0 || n < 0 || e0 + n > c->m.E) NS_SET(c, NS_ERR_INVALID_ARG, "element range out of bounds");
  int rc;
  if ((rc = sync_all(c)) != NS_OK) return rc;
  const int64_t S4 = 4 * (int64_t)c->tab.S;
  if (theta && n > 0) {
    HostSoA h(n * S4);
    const SpringRec *in = (const SpringRec *)theta;
    for (int64_t i = 0; i < n * S4; ++i) {
      h.tau[i] = in[i].tau; h.gR[i] = in[i].gR; h.tR[i] = in[i].tR; h.gmax[i] = in[i].gmax;
      h.dir[i] = in[i].dir; h.mode[i] = in[i].mode;
    }
    if ((rc = state_from_host(c, e0 * S4, n * S4, h.view))) return rc;
  }
  if (D && n > 0) {
    std::vector<double> tmp((size_t)84 * n);
    for (int64_t e = 0; e < n; ++e)
      for (int q = 0; q < 4; ++q)
        for (int i = 0; i < 6; ++i)
          for (int j = i; j < 6; ++j) tmp[(size_t)(q * 21 + sym6(i, j)) * n + e] = D[e * 144 + q * 36 + i * 6 + j];
    for (int k = 0; k < 84; ++k)
      CKC(c, cudaMemcpy(c->D + (size_t)k * c->m.epad + e0, tmp.data() + (size_t)k * n, n * 8, cudaMemcpyHostToDevice));
  }
  return NS_OK;
}

static double *field_ptr(ns_ctx *c, int32_t f) {
  switch (f) {
    case NS_FIELD_U: return c->u;
    case NS_FIELD_V: return c->v;
    case NS_FIELD_A: return c->a;
    case NS_FIELD_Q: return c->q;
    case NS_FIELD_DU: return c->du;
    default: return nullptr;
  }
}

int ns_read_nodal(ns_ctx *c, int32_t field, double *out) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (!c->has_mesh) NS_SET(c, NS_ERR_STATE, "no mesh");
  double *src = field_ptr(c, field);
  if (!src || !out) NS_SET(c, NS_ERR_INVALID_ARG, "bad field or null output");
  int rc;
  if ((rc = sync_all(c)) != NS_OK) return rc;
  CKC(c, cudaMemcpy(out, src, 3 * c->m.N * 8, cudaMemcpyDeviceToHost));
  return NS_OK;
}

int ns_write_nodal(ns_ctx *c, int32_t field, const double *in) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (!c->has_mesh) NS_SET(c, NS_ERR_STATE, "no mesh");
  double *dst = field_ptr(c, field);
  if (!dst || !in) NS_SET(c, NS_ERR_INVALID_ARG, "bad field or null input");
  int rc;
  if ((rc = sync_all(c)) != NS_OK) return rc;
  CKC(c, cudaMemcpy(dst, in, 3 * c->m.N * 8, cudaMemcpyHostToDevice));
  return NS_OK;
}

int ns_apply_operator(ns_ctx *c, int32_t op, const double *x, double *y) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (!c->has_mesh || !c->has_mat || !c->has_bnd) NS_SET(c, NS_ERR_STATE, "mesh, materials and boundary required");
  if (!x || !y || op < 0 || op > 4) NS_SET(c, NS_ERR_INVALID_ARG, "bad operator or null buffer");
  int rc;
  if ((rc = sync_all(c)) != NS_OK) return rc;
  const size_t n3 = 3 * (size_t)c->m.N;
  CKC(c, cudaMemcpy(c->p, x, n3 * 8, cudaMemcpyHostToDevice));
  CKC(c, cudaMemsetAsync(c->Ap, 0, n3 * 8, c->s_main));
  if (c->D2) LAUNCH(c, launch_to_pairs(c->D, c->D2, 84 * c->m.epad, c->s_main));  // D may have been written
  switch (op) {
    case NS_OP_K: rc = apply_elems64(c, c->op_K, nullptr, c->p, c->Ap, nullptr, nullptr, nullptr); break;
    case NS_OP_M: rc = apply_elems64(c, c->op_M, nullptr, c->p, c->Ap, nullptr, nullptr, nullptr); break;
    case NS_OP_CB: rc = apply_faces64(c, 1.0, c->p, nullptr, c->Ap, nullptr, nullptr, nullptr); break;
    case NS_OP_A: rc = apply_A(c, c->p, c->Ap, false, nullptr, nullptr, nullptr, false); break;
    case NS_OP_CR: rc = apply_elems64(c, c->op_Cr, nullptr, c->p, c->Ap, nullptr, nullptr, nullptr); break;
  }
  if (rc) return rc;
  if ((rc = sync_stream(c, c->s_main)) != NS_OK) return rc;
  CKC(c, cudaMemcpy(y, c->Ap, n3 * 8, cudaMemcpyDeviceToHost));
  return NS_OK;
}

int ns_apply_coarse_operator(ns_ctx *c, int32_t op, int64_t nc, const double *xc, double *yc) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (!c->has_mesh || !c->has_mat || !c->has_bnd) NS_SET(c, NS_ERR_STATE, "mesh, materials and boundary required");
  if (!c->cfg.multigrid) NS_SET(c, NS_ERR_STATE, "the context has no coarse level (cfg.multigrid = 0)");
  if (!xc || !yc || nc != c->mg.Nc || (op != NS_OP_K && op != NS_OP_M && op != NS_OP_CB && op != NS_OP_A))
    NS_SET(c, NS_ERR_INVALID_ARG, "bad operator, coarse size or null buffer");
  int rc;
  if ((rc = sync_all(c)) != NS_OK) return rc;
  std::vector<float> x4((size_t)4 * nc, 0.0f), y4((size_t)4 * nc);
  for (int64_t i = 0; i < nc; ++i)
    for (int k = 0; k < 3; ++k) x4[4 * i + k] = (float)xc[3 * i + k];
  MgLevel &g = c->mg;
  CKC(c, cudaMemcpy(g.p, x4.data(), x4.size() * 4, cudaMemcpyHostToDevice));
  CKC(c, cudaMemsetAsync(g.Ap, 0, x4.size() * 4, c->s_main));
  LAUNCH(c, launch_mg_dbar(c->D, g.Dbar, c->m.epad, c->m.E, c->s_main));  // D may have been written
  const OpCoef *oc = op == NS_OP_K ? c->op_K : op == NS_OP_M ? c->op_M : op == NS_OP_A ? c->op_A : nullptr;
  const float cC = op == NS_OP_CB ? 1.0f : op == NS_OP_A ? (float)(2.0 / c->cfg.dt) : 0.0f;
  if ((rc = apply_mg(c, oc, cC, g.p, g.Ap, nullptr, nullptr, nullptr)) != NS_OK) return rc;
  if ((rc = sync_stream(c, c->s_main)) != NS_OK) return rc;
  CKC(c, cudaMemcpy(y4.data(), g.Ap, y4.size() * 4, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < nc; ++i)
    for (int k = 0; k < 3; ++k) yc[3 * i + k] = y4[4 * i + k];
  return NS_OK;
}

int ns_spring_points(ns_ctx *c, int64_t npts, const int32_t *mat, const double *eps, const double *deps, void *theta,
                     double *D) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (!c->has_mat) NS_SET(c, NS_ERR_STATE, "materials required");
  if (npts < 0 || (npts > 0 && (!mat || !eps || !deps || !theta || !D))) NS_SET(c, NS_ERR_INVALID_ARG, "bad arguments");
  if (npts == 0) return NS_OK;
  for (int64_t i = 0; i < npts; ++i)
    if (mat[i] < 0 || mat[i] >= c->nmat) NS_SET(c, NS_ERR_INVALID_ARG, "material index out of range");
  const int S = c->tab.S;
  const int64_t nspr = npts * S;
  int rc;
  std::vector<double> e12((size_t)npts * 12);
  for (int64_t i = 0; i < npts; ++i)
    for (int k = 0; k < 6; ++k) {
      e12[i * 12 + k] = eps[i * 6 + k];
      e12[i * 12 + 6 + k] = deps[i * 6 + k];
    }
  HostSoA h(nspr);
  SpringRec *rec = (SpringRec *)theta;
  for (int64_t i = 0; i < nspr; ++i) {
    h.tau[i] = rec[i].tau; h.gR[i] = rec[i].gR; h.tR[i] = rec[i].tR; h.gmax[i] = rec[i].gmax;
    h.dir[i] = rec[i].dir; h.mode[i] = rec[i].mode;
  }
  SpringSoA d;
  double *eps_d = nullptr, *dp = nullptr;
  int32_t *mat_d = nullptr;
  rc = alloc_soa(c, d, nspr, false);
  if (!rc) rc = dalloc(c, &eps_d, e12.size());
  if (!rc) rc = dalloc(c, &dp, 21 * (size_t)npts);
  if (!rc) rc = dalloc(c, &mat_d, (size_t)npts);
  if (!rc) rc = copy_soa(c, d, 0, h.view, 0, nspr, cudaMemcpyHostToDevice, c->s_main);
  if (!rc) {
    cudaMemcpyAsync(eps_d, e12.data(), e12.size() * 8, cudaMemcpyHostToDevice, c->s_main);
    cudaMemcpyAsync(mat_d, mat, npts * 4, cudaMemcpyHostToDevice, c->s_main);
    cudaError_t e = launch_springs(c->tab, c->mats_d, nullptr, mat_d, eps_d, d, 0, 0, npts, nullptr, 0, dp, c->s_main);
    c->stats.kernel_launches++;
    if (e != cudaSuccess) {
      c->err = std::string("spring kernel: ") + cudaGetErrorString(e);
      rc = NS_ERR_CUDA;
    }
  }
  if (!rc) rc = copy_soa(c, h.view, 0, d, 0, nspr, cudaMemcpyDeviceToHost, c->s_main);
  std::vector<double> dh(21 * (size_t)npts);
  if (!rc && cudaMemcpyAsync(dh.data(), dp, dh.size() * 8, cudaMemcpyDeviceToHost, c->s_main) != cudaSuccess)
    rc = NS_ERR_CUDA;
  if (!rc) rc = sync_stream(c, c->s_main);
  free_soa(d, false);
  dfree(eps_d);
  dfree(dp);
  dfree(mat_d);
  if (rc) return rc;
  for (int64_t i = 0; i < nspr; ++i) rec[i] = {h.tau[i], h.gR[i], h.tR[i], h.gmax[i], h.dir[i], h.mode[i]};
  for (int64_t p = 0; p < npts; ++p)
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) D[p * 36 + i * 6 + j] = dh[p * 21 + sym6(i, j)];
  return NS_OK;
}

int ns_autotune_steps(ns_ctx *c, int32_t nsteps, ns_tuning *out) {
  if (!c || !out) return NS_ERR_INVALID_ARG;
  if (!c->mS.empty()) NS_SET(c, NS_ERR_STATE, "members with their own springs keep the default launch shape");
  memset(out, 0, sizeof(*out));
  struct Shape {
    int tp, minb;
  };
  std::vector<Shape> cand;
  const int tiles[7] = {4, 8, 16, 24, 32, 64, 128};
  for (int minb : {4, 1})
    for (int tp : tiles)
      if (spring_tile_ok(tp, c->tab.S)) cand.push_back({tp, minb});
  if (cand.empty()) NS_SET(c, NS_ERR_STATE, "no spring launch shape fits this spring count");
  if (nsteps < (int32_t)cand.size()) NS_SET(c, NS_ERR_INVALID_ARG, "need at least one step per launch shape");
  // every step runs in full (the launch shape changes no sum), its spring launches timed
  const int32_t timing = c->cfg.timing;
  const int tp0 = c->tab.tp, minb0 = c->tab.minb;
  c->cfg.timing = 1;
  std::vector<float> best(cand.size(), 1e30f);
  int rc = NS_OK;
  for (int32_t i = 0; i < nsteps && rc == NS_OK; ++i) {
    const size_t k = (size_t)i % cand.size();
    c->tab.tp = cand[k].tp;
    c->tab.minb = cand[k].minb;
    const double ms0 = c->stats.ms_spring;
    rc = ns_advance(c, 1);
    if (rc == NS_OK) best[k] = std::min(best[k], (float)(c->stats.ms_spring - ms0));
  }
  c->cfg.timing = timing;
  size_t kb = 0;
  for (size_t k = 0; k < cand.size(); ++k) {
    out->tile_points[k] = cand[k].tp;
    out->tile_blocks[k] = cand[k].minb;
    out->tile_ms[k] = best[k];
    if (best[k] < best[kb]) kb = k;
  }
  out->n_tile = (int32_t)cand.size();
  if (rc == NS_OK) {
    c->tab.tp = cand[kb].tp;
    c->tab.minb = cand[kb].minb;
  } else {
    c->tab.tp = tp0;
    c->tab.minb = minb0;
  }
  out->chosen_tile_points = c->tab.tp;
  out->chosen_tile_blocks = c->tab.minb;
  return rc;
}

int ns_autotune(ns_ctx *c, ns_tuning *out) {
  if (!c || !out) return NS_ERR_INVALID_ARG;
  if (!c->has_mat || !c->has_bnd || c->step < 1) NS_SET(c, NS_ERR_STATE, "autotune after at least one step");
  if (!c->mS.empty()) NS_SET(c, NS_ERR_STATE, "members with their own springs keep the default launch shape");
  memset(out, 0, sizeof(*out));
  const int S = c->tab.S;
  int rc = NS_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CKC(c, cudaEventCreate(&e0));
  CKC(c, cudaEventCreate(&e1));
  auto timed = [&](cudaStream_t s, auto &&work, float *ms) -> int {
    CKC(c, cudaEventRecord(e0, s));
    int r = work();
    if (r) return r;
    CKC(c, cudaEventRecord(e1, s));
    if ((r = sync_stream(c, s)) != NS_OK) return r;
    CKC(c, cudaEventElapsedTime(ms, e0, e1));
    return NS_OK;
  };
  // 1. spring kernel block shape on a copy of the state of 131,072 resident elements taken
  //    as eight slices spread over the model (its layers load the springs differently),
  //    packed into one sample that one launch covers.  The state is already at this
  //    step's strains, so the sample moves it one increment further along the same path
  //    (strain eps + deps, increment deps): the springs take a root solve of the size the
  //    next step's would take, not a solve that starts at its root.
  const int64_t ne = std::min<int64_t>(c->E_res, 131072);
  const int nsl = ne == 131072 ? 8 : 1;
  const int64_t nes = ne / nsl;
  if (ne > 0 && c->eps) {
    // the sample is a model of its own for the launch: packed state, strains, materials of
    // its elements and a tangent array in the production layout, so that the timed launch
    // takes the production path (element materials, the [84][epad] tangent)
    const int64_t nel = nes * nsl, np = 4 * nel, nspr = np * S, epad_s = (nel + 63) / 64 * 64;
    SpringSoA scr;
    double *D_s = nullptr, *eps_s = nullptr;
    int32_t *mat_s = nullptr;
    if ((rc = alloc_soa(c, scr, nspr, false)) == NS_OK && (rc = dalloc(c, &D_s, 84 * (size_t)epad_s)) == NS_OK &&
        (rc = dalloc(c, &eps_s, 12 * (size_t)np)) == NS_OK && (rc = dalloc(c, &mat_s, (size_t)nel)) == NS_OK) {
      auto slice0 = [&](int j) { return nsl == 1 ? (int64_t)0 : j * ((c->E_res - nes) / (nsl - 1)); };
      for (int j = 0; j < nsl && rc == NS_OK; ++j) {  // (no early return: the scratch is freed below)
        const cudaError_t e = launch_tune_sample(c->eps, c->m.mat, slice0(j), nes, reinterpret_cast<float2 *>(eps_s),
                                                 mat_s, j * nes, c->s_main);
        c->stats.kernel_launches++;
        if (e != cudaSuccess) {
          c->err = std::string("autotune sample: ") + cudaGetErrorString(e);
          rc = NS_ERR_CUDA;
        }
      }
      const int cands[8] = {4, 8, 16, 24, 32, 64, 128, 256};  // at most 16 shapes: ns_tuning's arrays
      float best = 1e30f;
      int chosen = spring_tile_default(S), chosen_b = 1;
      for (int kk = 0; kk < 16 && rc == NS_OK; ++kk) {
        const int k = kk % 8, minb = kk < 8 ? 1 : 4;
        if (!spring_tile_ok(cands[k], S)) continue;
        SpringTables tb = c->tab;
        tb.tp = cands[k];
        tb.minb = minb;
        float ms_best = 1e30f;
        for (int rep = 0; rep < 3 && rc == NS_OK; ++rep) {
          for (int j = 0; j < nsl && rc == NS_OK; ++j)
            rc = copy_soa(c, scr, j * nes * 4 * S, c->st, slice0(j) * 4 * S, nes * 4 * S, cudaMemcpyDeviceToDevice,
                          c->s_main);
          if (rc != NS_OK) break;
          float ms = 0.0f;
          rc = timed(c->s_main, [&]() -> int {
            LAUNCH(c, launch_springs(tb, c->mats_d, mat_s, nullptr, eps_s, scr, 0, 0, np, D_s, epad_s, nullptr,
                                     c->s_main, true));
            return NS_OK;
          }, &ms);
          ms_best = std::min(ms_best, ms);
        }
        if (rc != NS_OK) break;
        out->tile_points[out->n_tile] = cands[k];
        out->tile_blocks[out->n_tile] = minb;
        out->tile_ms[out->n_tile] = ms_best;
        out->n_tile++;
        if (ms_best < best) {
          best = ms_best;
          chosen = cands[k];
          chosen_b = minb;
        }
      }
      if (rc == NS_OK) {
        c->tab.tp = chosen;
        c->tab.minb = chosen_b;
        out->chosen_tile_points = chosen;
        out->chosen_tile_blocks = chosen_b;
      }
    }
    free_soa(scr, false);
    dfree(D_s);
    dfree(eps_s);
    dfree(mat_s);
  }
  // 2. chunk size of the streamed state: H2D of a ring's worth of chunks and D2H of the same
  //    bytes back to where they came from (the host state is left as it was)
  const int64_t nstream = c->m.E - c->E_res;
  if (rc == NS_OK && nstream > 0 && c->cfg.stream_mode == NS_STREAM_RING && !c->ring.empty()) {
    const int64_t cap = std::min<int64_t>(c->cfg.chunk_elems, nstream);  // ring buffers hold this many
    const int64_t S4 = 4 * (int64_t)S;
    const int R = (int)c->ring.size();
    int64_t cands[6] = {cap / 8, cap / 4, cap / 2, cap, 0, 0};
    double best = 0.0;
    int64_t chosen = c->cfg.chunk_elems;
    for (int k = 0; k < 4 && rc == NS_OK; ++k) {
      const int64_t ch = cands[k];
      if (ch < 1) continue;
      const int64_t nch = std::min<int64_t>((nstream + ch - 1) / ch, 2 * (int64_t)R);
      float ms = 0.0f;
      int64_t bytes = 0;
      rc = timed(c->s_h2d, [&]() -> int {
        for (int64_t j = 0; j < nch; ++j) {
          const int slot = (int)(j % R);
          const int64_t a = j * ch, n = std::min(ch, nstream - a);
          if (n <= 0) break;
          if (j >= R) CKC(c, cudaStreamWaitEvent(c->s_h2d, c->ev_d2h[slot], 0));
          int r = copy_soa(c, c->ring[slot], 0, c->hst, a * S4, n * S4, cudaMemcpyHostToDevice, c->s_h2d);
          if (r) return r;
          CKC(c, cudaEventRecord(c->ev_h2d[slot], c->s_h2d));
          CKC(c, cudaStreamWaitEvent(c->s_d2h, c->ev_h2d[slot], 0));
          if ((r = copy_soa(c, c->hst, a * S4, c->ring[slot], 0, n * S4, cudaMemcpyDeviceToHost, c->s_d2h))) return r;
          CKC(c, cudaEventRecord(c->ev_d2h[slot], c->s_d2h));
          bytes += 2 * n * S4 * 40;
        }
        // the measured window ends when the last D2H has landed
        CKC(c, cudaEventRecord(c->ev_join, c->s_d2h));
        CKC(c, cudaStreamWaitEvent(c->s_h2d, c->ev_join, 0));
        return NS_OK;
      }, &ms);
      if (rc != NS_OK) break;
      const double gbps = bytes / (ms / 1e3) / 1e9;
      out->chunk_elems[out->n_chunk] = ch;
      out->chunk_gbps[out->n_chunk] = (float)gbps;
      out->n_chunk++;
      if (gbps > best) {
        best = gbps;
        chosen = ch;
      }
    }
    if (rc == NS_OK) {
      int r = sync_stream(c, c->s_d2h);
      if (r) rc = r;
      c->cfg.chunk_elems = chosen;
      out->chosen_chunk_elems = chosen;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == NS_OK) CKC(c, cudaStreamSynchronize(c->s_main));
  return rc;
}

int ns_get_stats(ns_ctx *c, ns_stats *st) {
  if (!c || !st) return NS_ERR_INVALID_ARG;
  *st = c->stats;
  return NS_OK;
}

int ns_reset_stats(ns_ctx *c) {
  if (!c) return NS_ERR_INVALID_ARG;
  const int64_t steps = c->stats.steps, launches = c->stats.kernel_launches, re = c->stats.resident_elems,
                se = c->stats.streamed_elems;
  c->stats = ns_stats{};
  c->stats.steps = steps;
  c->stats.kernel_launches = launches;
  c->stats.resident_elems = re;
  c->stats.streamed_elems = se;
  int rc;
  if ((rc = sync_all(c)) != NS_OK) return rc;
  CKC(c, cudaMemset(c->spr_cnt, 0, 3 * kSpringCountSlots * sizeof(unsigned long long)));
  return NS_OK;
}

namespace {
struct CkptHeader {
  char magic[8];
  int64_t version, step, N, E, S;
};
}  // namespace

int ns_checkpoint_size(ns_ctx *c, int64_t *bytes) {
  if (!c || !bytes) return NS_ERR_INVALID_ARG;
  if (!c->has_mat) NS_SET(c, NS_ERR_STATE, "no state yet");
  if (!c->mS.empty()) NS_SET(c, NS_ERR_STATE, "members with their own springs: no checkpoint");
  *bytes = (int64_t)sizeof(CkptHeader) + 5 * 3 * c->m.N * 8 + c->m.E * 144 * 8 + ns_state_bytes(c->m.E, c->tab.S);
  return NS_OK;
}

int ns_checkpoint(ns_ctx *c, void *buf, int64_t bytes) {
  int64_t need = 0;
  int rc = ns_checkpoint_size(c, &need);
  if (rc) return rc;
  if (!buf || bytes < need) NS_SET(c, NS_ERR_INVALID_ARG, "checkpoint buffer too small");
  char *p = (char *)buf;
  CkptHeader h{};
  memcpy(h.magic, "NSCKPT01", 8);
  h.version = 1;
  h.step = c->step;
  h.N = c->m.N;
  h.E = c->m.E;
  h.S = c->tab.S;
  memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  for (int f = 0; f < 5; ++f) {
    if ((rc = ns_read_nodal(c, f, (double *)p))) return rc;
    p += 3 * c->m.N * 8;
  }
  if ((rc = ns_read_state(c, 0, c->m.E, p + c->m.E * 144 * 8, (double *)p))) return rc;
  return NS_OK;
}

int ns_restore(ns_ctx *c, const void *buf, int64_t bytes) {
  int64_t need = 0;
  int rc = ns_checkpoint_size(c, &need);
  if (rc) return rc;
  if (!buf || bytes < need) NS_SET(c, NS_ERR_INVALID_ARG, "checkpoint buffer too small");
  const char *p = (const char *)buf;
  CkptHeader h;
  memcpy(&h, p, sizeof(h));
  if (memcmp(h.magic, "NSCKPT01", 8) != 0 || h.N != c->m.N || h.E != c->m.E || h.S != c->tab.S)
    NS_SET(c, NS_ERR_INVALID_ARG, "checkpoint does not match this model");
  p += sizeof(h);
  for (int f = 0; f < 5; ++f) {
    if ((rc = ns_write_nodal(c, f, (const double *)p))) return rc;
    p += 3 * c->m.N * 8;
  }
  if ((rc = ns_write_state(c, 0, c->m.E, p + c->m.E * 144 * 8, (const double *)p))) return rc;
  c->step = h.step;
  c->stats.steps = h.step;
  return NS_OK;
}

void ns_destroy(ns_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->cfg.device);
  if (c->s_main) cudaStreamSynchronize(c->s_main);
  if (c->s_h2d) cudaStreamSynchronize(c->s_h2d);
  if (c->s_d2h) cudaStreamSynchronize(c->s_d2h);
  DevMesh &m = c->m;
  dfree(m.conn); dfree(m.geom); dfree(m.geom32); dfree(m.mat); dfree(m.kerr); dfree(m.geom2); dfree(m.fnode); dfree(m.fgeom); dfree(m.fmat);
  dfree(m.fkind); dfree(m.surf); dfree(m.ecol_ids); dfree(m.fcol_ids);
  dfree(m.lconn); dfree(m.lnode); dfree(m.loff);
  dfree(c->xyz_d); dfree(c->mats_d); dfree(c->op_A); dfree(c->op_K); dfree(c->op_M); dfree(c->op_Cr);
  dfree(c->op_rhs); dfree(c->q_d); dfree(c->T_d); dfree(c->pow_d); dfree(c->powf_d); dfree(c->T2_d); dfree(c->tfrag_d); dfree(c->tsc_d); dfree(c->q2_d); dfree(c->D); dfree(c->D32);
  dfree(c->D16); dfree(c->op_A16); dfree(c->D2);
  destroy_graphs(c);
  dfree(c->vseg_d); dfree(c->eseg_d); dfree(c->fseg_d); dfree(c->voff_d); dfree(c->eoff_d); dfree(c->foff_d);
  dfree(c->fmem_d);
  free_soa(c->st, false);
  free_soa(c->hst, true);
  for (auto &rb : c->ring) free_soa(rb, false);
  dfree(c->u); dfree(c->v); dfree(c->a); dfree(c->q); dfree(c->du); dfree(c->b); dfree(c->r); dfree(c->z);
  dfree(c->p); dfree(c->Ap); dfree(c->Jd); dfree(c->Jinv); dfree(c->eps); dfree(c->part); dfree(c->vin_d);
  dfree(c->surf_u); dfree(c->surf_v); dfree(c->surf_a);
  dfree(c->Jinv32);
  dfree(c->rin); dfree(c->zin); dfree(c->pin); dfree(c->xin); dfree(c->Apin);
  dfree(c->sc);
  dfree(c->spr_cnt);
  dfree(c->mg.conn1); dfree(c->mg.cfnode); dfree(c->mg.rptr); dfree(c->mg.rlist); dfree(c->mg.par);
  dfree(c->mg.Dbar); dfree(c->mg.Jd32); dfree(c->mg.Jinv32);
  dfree(c->mg.x); dfree(c->mg.r); dfree(c->mg.z); dfree(c->mg.p); dfree(c->mg.Ap);
  for (void *p : c->mtab_mem) cudaFree(p);
  dfree(c->flag_d);
  hfree(c->sc_h);
  hfree(c->flag_h);
  if (c->ev_h2d) {
    for (int i = 0; i < c->cfg.ring_depth; ++i) {
      cudaEventDestroy(c->ev_h2d[i]);
      cudaEventDestroy(c->ev_comp[i]);
      cudaEventDestroy(c->ev_d2h[i]);
    }
    delete[] c->ev_h2d;
    delete[] c->ev_comp;
    delete[] c->ev_d2h;
  }
  if (c->ev_d2h_all) cudaEventDestroy(c->ev_d2h_all);
  if (c->ev_sync) cudaEventDestroy(c->ev_sync);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_adv0) cudaEventDestroy(c->ev_adv0);
  if (c->ev_adv1) cudaEventDestroy(c->ev_adv1);
  if (c->ev_stream_t0) cudaEventDestroy(c->ev_stream_t0);
  if (c->ev_stream_t1) cudaEventDestroy(c->ev_stream_t1);
  if (c->ev_strain) cudaEventDestroy(c->ev_strain);
  if (c->s_main) cudaStreamDestroy(c->s_main);
  if (c->s_h2d) cudaStreamDestroy(c->s_h2d);
  if (c->s_d2h) cudaStreamDestroy(c->s_d2h);
  for (int k = 0; k < ns_ctx::kMemberStreams; ++k) {
    if (c->s_mem[k]) cudaStreamSynchronize(c->s_mem[k]), cudaStreamDestroy(c->s_mem[k]);
    if (c->ev_mem[k]) cudaEventDestroy(c->ev_mem[k]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  delete c;
}

// ---------------------------------------------------------------- host-only helpers

int ns_spring_directions(int32_t S, double *q, double *w) {
  if (!q || !w) return NS_ERR_INVALID_ARG;
  return host_spring_directions(S, q, w) == 0 ? NS_OK : NS_ERR_INVALID_ARG;
}

int ns_colour_elements(int64_t E, int64_t N, const int32_t *conn, int32_t *colour, int32_t *nc) {
  if (E < 0 || N <= 0 || !conn || !colour || !nc) return NS_ERR_INVALID_ARG;
  for (int64_t i = 0; i < 10 * E; ++i)
    if (conn[i] < 0 || conn[i] >= N) return NS_ERR_BAD_MESH;
  return host_colouring(E, N, conn, colour, nc) == 0 ? NS_OK : NS_ERR_BAD_MESH;
}

int64_t ns_state_bytes(int64_t E, int32_t S) { return E * 4 * (int64_t)S * 40; }

int ns_coarse_map(int64_t E, int64_t N, const int32_t *conn, int32_t *cid, int32_t *par, int64_t *nc) {
  if (E < 0 || N <= 0 || !conn || !cid || !par || !nc) return NS_ERR_INVALID_ARG;
  for (int64_t i = 0; i < 10 * E; ++i)
    if (conn[i] < 0 || conn[i] >= N) return NS_ERR_BAD_MESH;
  const int64_t r = host_coarse_map(E, N, conn, cid, par);
  if (r < 0) return NS_ERR_BAD_MESH;
  *nc = r;
  return NS_OK;
}

}  // extern "C"

namespace ns {
int ctx_set_members_built(ns_ctx *c, int32_t M, const int64_t *elem_off, const int64_t *node_off) {
  if (!c || !c->has_mesh || !c->has_bnd || c->has_motion || c->step > 0 || c->M > 1 || c->m.Msh > 1 ||
      c->cfg.scatter != NS_SCATTER_ATOMIC || c->cfg.multigrid || M < 1 || !elem_off || !node_off)
    return NS_ERR_STATE;
  if (elem_off[0] != 0 || elem_off[M] != c->m.E || node_off[0] != 0 || node_off[M] != c->m.N)
    return NS_ERR_INVALID_ARG;
  return setup_members(c, M, elem_off, node_off);
}
}  // namespace ns
