// Served ensemble runtime (include/ns_server.h): a first-come-first-served queue of
// independent cases, admitted into concurrent slots by device and pinned-host memory;
// each admitted case runs in a context of its own driven by its own host thread, or --
// continuous batching -- as a member of the batched context of its solver class, which a
// worker thread per class re-forms whenever a member arrives or finishes.
#include "../../include/ns_server.h"

#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ns_internal.h"

namespace {

int64_t pad64(int64_t n) { return ((n + 63) / 64) * 64; }

struct CaseRec {
  // copies of the submitted arrays
  std::vector<double> xyz, acc;
  std::vector<int32_t> conn, mat, faces, face_elem, face_kind, surf;
  std::vector<ns_material> mats;
  ns_config cfg{};
  int64_t n_nodes = 0, n_elems = 0, n_faces = 0, n_surf = 0, n_samples = 0, n_steps = 0;
  int32_t n_mat = 0;
  // admission
  int64_t dev_resident = 0, state_bytes = 0, dev_streamed = 0, reserved_dev = 0, reserved_pin = 0;
  ns_case_stats st{};
  std::string err;
  std::vector<double> ru, rv, ra;
  std::thread th;
  // batched: input velocity of the whole record ([n_samples + 1][3]) and steps done
  std::vector<double> vin;
  int64_t done = 0;
  double ms_share = 0.0, launch_share = 0.0;
};

// Solver class of a case: the settings that one batched context shares among its members.
struct ClassKey {
  int32_t precision, x0_prev, cg_max_iter, inner_max_iter, graphs, pair_operator;
  double dt, cg_tol, inner_tol, f1, f2;
  bool operator<(const ClassKey &o) const { return memcmp(this, &o, sizeof(ClassKey)) < 0; }
};
ClassKey class_of(const ns_config &c) {
  ClassKey k;
  memset(&k, 0, sizeof(k));
  k.precision = c.precision;
  k.x0_prev = c.x0_prev;
  k.cg_max_iter = c.cg_max_iter;
  k.inner_max_iter = c.inner_max_iter;
  k.graphs = c.graphs;
  k.pair_operator = c.pair_operator;
  k.dt = c.dt;
  k.cg_tol = c.cg_tol;
  k.inner_tol = c.inner_tol;
  k.f1 = c.rayleigh_f1;
  k.f2 = c.rayleigh_f2;
  return k;
}

struct ClassWorker {
  std::vector<CaseRec *> pending;  // admitted, not yet in the batch
  std::thread th;
  bool running = false;
};

}  // namespace

struct ns_server {
  ns_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int64_t> queue;
  std::map<int64_t, std::unique_ptr<CaseRec>> cases;
  int64_t next_id = 1;
  int active = 0;
  int64_t dev_used = 0, pin_used = 0;
  bool stop = false;
  std::thread sched;
  std::map<ClassKey, ClassWorker> classes;  // continuous batching (cfg.batch)
  std::chrono::steady_clock::time_point t0;

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

namespace {

// Head of the queue admissible now?  Decides resident or streamed placement.
bool can_admit(ns_server *s, CaseRec &r) {
  if (s->active >= s->cfg.max_active) return false;
  const int64_t dev_cap = s->cfg.batch ? s->cfg.device_budget / 2 : s->cfg.device_budget;
  if (s->dev_used + r.dev_resident <= dev_cap) {
    r.st.streamed = 0;
    r.reserved_dev = r.dev_resident;
    r.reserved_pin = 0;
    return true;
  }
  if (s->dev_used + r.dev_streamed <= s->cfg.device_budget && s->pin_used + r.state_bytes <= s->cfg.pinned_budget) {
    r.st.streamed = 1;
    r.reserved_dev = r.dev_streamed;
    r.reserved_pin = r.state_bytes;
    return true;
  }
  return false;
}

void run_case(ns_server *s, CaseRec *r) {
  int rc = NS_OK;
  ns_ctx *ctx = nullptr;
  ns_config cfg = r->cfg;
  cfg.device = s->cfg.device;
  cfg.surface_ring_steps = std::max<int64_t>(1, r->n_steps);
  cfg.device_state_budget = r->st.streamed ? 0 : -1;
  cudaSetDevice(s->cfg.device);
  rc = ns_create(&ctx, &cfg);
  if (rc == NS_OK) rc = ns_upload_mesh(ctx, r->n_nodes, r->xyz.data(), r->n_elems, r->conn.data(), r->mat.data());
  if (rc == NS_OK) rc = ns_set_materials(ctx, r->n_mat, r->mats.data());
  if (rc == NS_OK)
    rc = ns_set_boundary(ctx, r->n_faces, r->faces.data(), r->face_elem.data(), r->face_kind.data(), r->n_surf,
                         r->surf.data());
  if (rc == NS_OK) rc = ns_set_ground_motion(ctx, r->n_samples, cfg.dt, r->acc.data());
  int64_t done = 0;
  const int64_t q = std::max(1, s->cfg.quantum_steps);
  while (rc == NS_OK && done < r->n_steps) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->stop) {
        rc = NS_ERR_STATE;
        r->err = "server stopped";
        break;
      }
    }
    const int64_t k = std::min(q, r->n_steps - done);
    rc = ns_advance(ctx, k);
    if (rc == NS_OK) done += k;
  }
  if (rc == NS_OK) {
    const size_t n = (size_t)r->n_steps * (size_t)r->n_surf * 3;
    r->ru.assign(n, 0.0);
    r->rv.assign(n, 0.0);
    r->ra.assign(n, 0.0);
    if (r->n_surf > 0 && r->n_steps > 0)
      rc = ns_read_surface(ctx, 1, r->n_steps, r->ru.data(), r->rv.data(), r->ra.data());
  }
  ns_stats st{};
  if (ctx && ns_get_stats(ctx, &st) == NS_OK) {
    r->st.ms_device = st.ms_advance;
    r->st.kernel_launches = st.kernel_launches;
  }
  if (rc != NS_OK && ctx && r->err.empty()) r->err = ns_last_error(ctx);
  if (rc != NS_OK && !ctx && r->err.empty()) r->err = ns_last_error(nullptr);
  if (ctx) ns_destroy(ctx);
  std::lock_guard<std::mutex> lk(s->mu);
  r->st.error = rc;
  r->st.state = rc == NS_OK ? NS_CASE_DONE : NS_CASE_FAILED;
  r->st.t_done = s->now();
  s->dev_used -= r->reserved_dev;
  s->pin_used -= r->reserved_pin;
  s->active--;
  s->cv.notify_all();
}

// ------------------------------------------------------------------ continuous batching

void finish_case(ns_server *s, CaseRec *r, int rc) {  // with s->mu held
  r->st.error = rc;
  r->st.state = rc == NS_OK ? NS_CASE_DONE : NS_CASE_FAILED;
  r->st.t_done = s->now();
  r->st.ms_device = r->ms_share;
  r->st.kernel_launches = (int64_t)(r->launch_share + 0.5);
  s->dev_used -= r->reserved_dev;
  s->pin_used -= r->reserved_pin;
  s->active--;
  s->cv.notify_all();
}

// A batched context for the members, in order: the disjoint union of their meshes, their
// material tables one after another, their springs per point, and each member's input
// velocity from its own step on.  *surf_off receives the members' surface-row ranges.
int form_batch(ns_server *s, const std::vector<CaseRec *> &mem, ns_ctx **out, std::vector<int64_t> &surf_off) {
  *out = nullptr;
  const int M = (int)mem.size();
  std::vector<int64_t> eo(M + 1, 0), no(M + 1, 0), fo(M + 1, 0), so(M + 1, 0);
  int32_t nmat = 0;
  for (int m = 0; m < M; ++m) {
    eo[m + 1] = eo[m] + mem[m]->n_elems;
    no[m + 1] = no[m] + mem[m]->n_nodes;
    fo[m + 1] = fo[m] + mem[m]->n_faces;
    so[m + 1] = so[m] + mem[m]->n_surf;
    nmat += mem[m]->n_mat;
  }
  if (nmat > 1024) return NS_ERR_INVALID_ARG;
  std::vector<double> xyz(3 * (size_t)no[M]);
  std::vector<int32_t> conn(10 * (size_t)eo[M]), mat((size_t)eo[M]), faces(6 * (size_t)fo[M]), fe((size_t)fo[M]),
      fk((size_t)fo[M]), surf((size_t)so[M]);
  std::vector<ns_material> mats;
  std::vector<int32_t> S(M);
  int64_t horizon = 0;
  int32_t mo = 0;
  for (int m = 0; m < M; ++m) {
    const CaseRec &r = *mem[m];
    std::copy(r.xyz.begin(), r.xyz.end(), xyz.begin() + 3 * no[m]);
    for (int64_t i = 0; i < 10 * r.n_elems; ++i) conn[10 * eo[m] + i] = r.conn[i] + (int32_t)no[m];
    for (int64_t e = 0; e < r.n_elems; ++e) mat[eo[m] + e] = r.mat[e] + mo;
    for (int64_t i = 0; i < 6 * r.n_faces; ++i) faces[6 * fo[m] + i] = r.faces[i] + (int32_t)no[m];
    for (int64_t f = 0; f < r.n_faces; ++f) {
      fe[fo[m] + f] = r.face_elem[f] + (int32_t)eo[m];
      fk[fo[m] + f] = r.face_kind[f];
    }
    for (int64_t i = 0; i < r.n_surf; ++i) surf[so[m] + i] = r.surf[i] + (int32_t)no[m];
    mats.insert(mats.end(), r.mats.begin(), r.mats.end());
    mo += r.n_mat;
    S[m] = r.cfg.n_springs;
    horizon = std::max(horizon, r.n_steps - r.done);
  }
  ns_config cfg = mem[0]->cfg;
  cfg.device = s->cfg.device;
  cfg.surface_ring_steps = std::max(1, s->cfg.quantum_steps);
  cfg.device_state_budget = -1;
  cfg.scatter = NS_SCATTER_ATOMIC;
  cfg.shared_members = 0;
  cfg.multigrid = 0;
  cfg.spring_tile_points = 0;
  cudaSetDevice(s->cfg.device);
  ns_ctx *c = nullptr;
  int rc = ns_create(&c, &cfg);
  if (rc == NS_OK) rc = ns_upload_mesh(c, no[M], xyz.data(), eo[M], conn.data(), mat.data());
  if (rc == NS_OK) rc = ns_set_materials(c, nmat, mats.data());
  if (rc == NS_OK)
    rc = ns_set_boundary(c, fo[M], faces.data(), fe.data(), fk.data(), so[M], surf.data());
  if (rc == NS_OK && M > 1) rc = ns::ctx_set_members_built(c, M, eo.data(), no.data());
  if (rc == NS_OK && M > 1) rc = ns_set_member_springs(c, M, S.data());
  if (rc == NS_OK) {  // a zero record of the batch's length, then each member's own velocity
    std::vector<double> zero(3 * (size_t)(horizon + 1), 0.0);
    rc = ns_set_ground_motion(c, horizon + 1, cfg.dt, zero.data());
  }
  for (int m = 0; m < M && rc == NS_OK; ++m) {
    const CaseRec &r = *mem[m];
    const int64_t k0 = std::min<int64_t>(r.done, r.n_samples);
    rc = ns::ctx_set_member_velocity(c, m, r.vin.data() + 3 * k0, r.n_samples + 1 - k0);
  }
  if (rc != NS_OK) {
    if (c) ns_destroy(c);
    return rc;
  }
  surf_off = so;
  *out = c;
  return NS_OK;
}

// Worker of one solver class: keeps its admitted cases in one batched context, re-formed
// when a case arrives, and advances it a quantum at a time.  A case that finishes is
// finalised at once; while the finished members hold at most a quarter of the batch's
// elements they stay in it, parked (still stepped, their output ignored), until the next
// re-formation drops them -- which saves a re-formation per departure.
void class_worker(ns_server *s, ClassKey key) {
  struct Slot {
    CaseRec *r;       // nullptr: parked (finished)
    int64_t n_elems;
  };
  std::vector<Slot> mem;
  ns_ctx *ctx = nullptr;
  std::vector<int64_t> soff;
  auto active_cases = [&]() {
    std::vector<CaseRec *> v;
    for (const Slot &sl : mem)
      if (sl.r) v.push_back(sl.r);
    return v;
  };
  // a new context for `next` (continuing cases first, in their current order); the
  // continuing ones take their state from the current context
  auto reform = [&](const std::vector<CaseRec *> &next) -> int {
    const auto tf0 = std::chrono::steady_clock::now();
    ns_ctx *nc = nullptr;
    std::vector<int64_t> so;
    int rc = next.empty() ? NS_OK : form_batch(s, next, &nc, so);
    for (size_t m = 0, j = 0; m < mem.size() && rc == NS_OK && ctx; ++m)
      if (mem[m].r && j < next.size() && mem[m].r == next[j]) rc = ns::ctx_copy_member(nc, (int)j++, ctx, (int)m);
    if (ctx) ns_destroy(ctx);
    ctx = nullptr;
    mem.clear();
    if (rc != NS_OK) {
      std::string e = nc ? ns_last_error(nc) : "batch formation failed";
      if (nc) ns_destroy(nc);
      std::lock_guard<std::mutex> lk(s->mu);
      for (CaseRec *r : next) {
        r->err = e;
        finish_case(s, r, rc);
      }
      return rc;
    }
    ctx = nc;
    soff = so;
    const double tf = std::chrono::duration<double>(std::chrono::steady_clock::now() - tf0).count();
    for (CaseRec *r : next) {
      mem.push_back(Slot{r, r->n_elems});
      r->st.batches++;
      r->st.t_reform += tf;
    }
    return NS_OK;
  };
  for (;;) {
    std::vector<CaseRec *> arrived;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      ClassWorker &w = s->classes[key];
      if (active_cases().empty()) s->cv.wait(lk, [&] { return s->stop || !w.pending.empty(); });
      if (s->stop) {
        for (const Slot &sl : mem)
          if (sl.r) {
            sl.r->err = "server stopped";
            finish_case(s, sl.r, NS_ERR_STATE);
          }
        for (CaseRec *r : w.pending) {
          r->err = "server stopped";
          finish_case(s, r, NS_ERR_STATE);
        }
        w.pending.clear();
        w.running = false;
        break;
      }
      arrived.swap(w.pending);
    }
    if (!arrived.empty() || !ctx) {  // re-form: continuing cases first, then the arrivals (parked ones dropped)
      std::vector<CaseRec *> next = active_cases();
      next.insert(next.end(), arrived.begin(), arrived.end());
      if (reform(next) != NS_OK || !ctx) continue;
    }
    // one quantum, no further than the nearest finishing case
    int64_t q = s->cfg.quantum_steps;
    for (const Slot &sl : mem)
      if (sl.r) q = std::min(q, sl.r->n_steps - sl.r->done);
    ns_stats st0{}, st1{};
    ns_get_stats(ctx, &st0);
    int rc = ns_advance(ctx, q);
    ns_get_stats(ctx, &st1);
    int64_t Etot = 0;
    for (const Slot &sl : mem) Etot += sl.n_elems;
    if (rc == NS_OK) {
      const int64_t ns_all = soff.back(), step1 = ns::ctx_steps(ctx) - q + 1;
      std::vector<double> u(3 * (size_t)ns_all * q), v(u.size()), a(u.size());
      if (ns_all > 0) rc = ns_read_surface(ctx, step1, q, u.data(), v.data(), a.data());
      for (size_t m = 0; m < mem.size() && rc == NS_OK; ++m) {
        CaseRec *r = mem[m].r;
        if (!r) continue;
        const int64_t k = soff[m + 1] - soff[m];
        for (int64_t t = 0; t < q; ++t) {
          const size_t dst = ((size_t)(r->done + t) * r->n_surf) * 3, src = ((size_t)t * ns_all + soff[m]) * 3;
          std::copy(u.begin() + src, u.begin() + src + 3 * k, r->ru.begin() + dst);
          std::copy(v.begin() + src, v.begin() + src + 3 * k, r->rv.begin() + dst);
          std::copy(a.begin() + src, a.begin() + src + 3 * k, r->ra.begin() + dst);
        }
        const double share = (double)r->n_elems / (double)std::max<int64_t>(Etot, 1);
        r->ms_share += share * (st1.ms_advance - st0.ms_advance);
        r->launch_share += share * (double)(st1.kernel_launches - st0.kernel_launches);
        r->done += q;
      }
    }
    int64_t parked = 0;
    bool left = false;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (rc != NS_OK) {
        const std::string e = ns_last_error(ctx);
        for (Slot &sl : mem)
          if (sl.r) {
            sl.r->err = e;
            finish_case(s, sl.r, rc);
            sl.r = nullptr;
          }
      } else {
        for (Slot &sl : mem)
          if (sl.r && sl.r->done >= sl.r->n_steps) {
            finish_case(s, sl.r, NS_OK);
            sl.r = nullptr;
            left = true;
          }
      }
      for (const Slot &sl : mem)
        if (!sl.r) parked += sl.n_elems;
    }
    if (rc != NS_OK) {
      ns_destroy(ctx);
      ctx = nullptr;
      mem.clear();
    } else if (left && (active_cases().empty() || 4 * parked > Etot)) {
      reform(active_cases());  // too much finished work in the batch (or none left): re-form or close
    }
  }
  if (ctx) ns_destroy(ctx);
}

void scheduler(ns_server *s) {
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv.wait(lk, [&] { return s->stop || (!s->queue.empty() && can_admit(s, *s->cases[s->queue.front()])); });
    if (s->stop) return;
    const int64_t id = s->queue.front();
    s->queue.pop_front();
    CaseRec *r = s->cases[id].get();
    r->st.state = NS_CASE_RUNNING;
    r->st.t_admit = s->now();
    r->st.device_bytes = r->reserved_dev;
    s->dev_used += r->reserved_dev;
    s->pin_used += r->reserved_pin;
    s->active++;
    if (s->cfg.batch && !r->st.streamed) {  // a member of its class's batch
      const size_t n = (size_t)r->n_steps * (size_t)r->n_surf * 3;
      r->ru.assign(n, 0.0);
      r->rv.assign(n, 0.0);
      r->ra.assign(n, 0.0);
      r->vin.assign(3 * (size_t)(r->n_samples + 1), 0.0);
      ns::host_input_velocity(r->acc.data(), r->n_samples, r->cfg.dt, r->vin.data());
      const ClassKey key = class_of(r->cfg);
      ClassWorker &w = s->classes[key];
      w.pending.push_back(r);
      if (!w.running) {
        if (w.th.joinable()) w.th.join();
        w.running = true;
        w.th = std::thread(class_worker, s, key);
      }
      s->cv.notify_all();
    } else {
      r->th = std::thread(run_case, s, r);
    }
  }
}

}  // namespace

extern "C" {

int ns_case_bytes(const ns_case *c, int64_t *device_bytes, int64_t *state_bytes, int64_t *streamed_device_bytes) {
  if (!c || c->n_elems <= 0 || c->n_nodes <= 0 || c->n_steps < 0 || c->n_surf < 0 || c->n_faces < 0)
    return NS_ERR_INVALID_ARG;
  const int64_t E = c->n_elems, N = c->n_nodes, F = c->n_faces, S = c->cfg.n_springs;
  const int64_t epad = pad64(E), fpad = pad64(std::max<int64_t>(F, 1));
  const int prec = c->cfg.precision;
  int64_t b = epad * (40 + 80 + 40 + 4) + 24 * N;  // connectivity, geometry (FP64, FP32), material, xyz
  b += fpad * (24 + 32 + 4 + 4);                   // faces
  b += N * (10 * 24 + 48 + 48 + 24);               // node vectors, block-Jacobi blocks
  b += 384 * E;                                    // strains at the points
  if (prec != NS_PREC_FP64) b += 5 * 16 * N;       // inner FP32 vectors
  b += 672 * epad;                                 // tangent D
  if (prec == NS_PREC_FP64_IR) b += 336 * epad;
  if (prec == NS_PREC_FP64_IR16) b += 168 * epad;
  b += 3 * 24 * std::max<int64_t>(c->n_surf, 1) * std::max<int64_t>(c->n_steps, 1);  // surface record
  b += 3 * 8 * (c->n_samples + 1);                 // input velocity
  b += (int64_t)64 << 20;                          // partial sums, scalars, tables, graphs
  const int64_t st = E * 4 * S * 40;
  const int64_t ring = (int64_t)std::max(2, c->cfg.ring_depth) * std::min<int64_t>(c->cfg.chunk_elems, E) * 4 * S * 40;
  if (device_bytes) *device_bytes = b + st;
  if (state_bytes) *state_bytes = st;
  if (streamed_device_bytes) *streamed_device_bytes = b + ring;
  return NS_OK;
}

int ns_server_create(ns_server **out, const ns_server_config *cfg) {
  if (!out || !cfg || cfg->max_active < 1 || cfg->device_budget <= 0 || cfg->pinned_budget < 0 || cfg->device < 0 ||
      (cfg->batch != 0 && cfg->batch != 1))
    return NS_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device >= ndev) {
    cudaGetLastError();
    return NS_ERR_CUDA;
  }
  ns_server *s = new ns_server();
  s->cfg = *cfg;
  if (s->cfg.quantum_steps < 1) s->cfg.quantum_steps = 16;
  s->t0 = std::chrono::steady_clock::now();
  s->sched = std::thread(scheduler, s);
  *out = s;
  return NS_OK;
}

int ns_server_submit(ns_server *s, const ns_case *c, int64_t *id) {
  if (!s || !c || !id) return NS_ERR_INVALID_ARG;
  if (c->n_elems <= 0 || c->n_nodes <= 0 || !c->xyz || !c->conn || !c->mat || c->n_mat < 1 || !c->mats ||
      c->n_steps < 1 || c->n_samples < 1 || !c->acc || c->n_faces < 0 || c->n_surf < 0 ||
      (c->n_faces > 0 && (!c->faces || !c->face_elem || !c->face_kind)) || (c->n_surf > 0 && !c->surf))
    return NS_ERR_INVALID_ARG;
  auto r = std::make_unique<CaseRec>();
  if (ns_case_bytes(c, &r->dev_resident, &r->state_bytes, &r->dev_streamed) != NS_OK) return NS_ERR_INVALID_ARG;
  if (r->dev_resident > s->cfg.device_budget &&
      (r->dev_streamed > s->cfg.device_budget || r->state_bytes > s->cfg.pinned_budget))
    return NS_ERR_OOM_DEVICE;  // would never fit, even alone
  r->n_nodes = c->n_nodes;
  r->n_elems = c->n_elems;
  r->n_faces = c->n_faces;
  r->n_surf = c->n_surf;
  r->n_samples = c->n_samples;
  r->n_steps = c->n_steps;
  r->n_mat = c->n_mat;
  r->cfg = c->cfg;
  r->xyz.assign(c->xyz, c->xyz + 3 * c->n_nodes);
  r->conn.assign(c->conn, c->conn + 10 * c->n_elems);
  r->mat.assign(c->mat, c->mat + c->n_elems);
  r->mats.assign(c->mats, c->mats + c->n_mat);
  if (c->n_faces > 0) {
    r->faces.assign(c->faces, c->faces + 6 * c->n_faces);
    r->face_elem.assign(c->face_elem, c->face_elem + c->n_faces);
    r->face_kind.assign(c->face_kind, c->face_kind + c->n_faces);
  }
  if (c->n_surf > 0) r->surf.assign(c->surf, c->surf + c->n_surf);
  r->acc.assign(c->acc, c->acc + 3 * c->n_samples);
  r->st.state = NS_CASE_QUEUED;
  r->st.error = NS_OK;
  r->st.state_bytes = r->state_bytes;
  r->st.elem_steps = c->n_elems * c->n_steps;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return NS_ERR_STATE;
  r->st.t_submit = s->now();
  *id = s->next_id++;
  s->cases[*id] = std::move(r);
  s->queue.push_back(*id);
  s->cv.notify_all();
  return NS_OK;
}

int ns_server_status(ns_server *s, int64_t id, ns_case_stats *st) {
  if (!s || !st) return NS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->cases.find(id);
  if (it == s->cases.end()) return NS_ERR_INVALID_ARG;
  *st = it->second->st;
  return NS_OK;
}

int ns_server_wait(ns_server *s, int64_t id, double timeout_s) {
  if (!s) return NS_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->cases.find(id);
  if (it == s->cases.end()) return NS_ERR_INVALID_ARG;
  CaseRec *r = it->second.get();
  const bool ok = s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
    return r->st.state == NS_CASE_DONE || r->st.state == NS_CASE_FAILED;
  });
  return ok ? NS_OK : NS_ERR_TIMEOUT;
}

int ns_server_result(ns_server *s, int64_t id, double *u, double *v, double *a) {
  if (!s) return NS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->cases.find(id);
  if (it == s->cases.end()) return NS_ERR_INVALID_ARG;
  CaseRec *r = it->second.get();
  if (r->st.state == NS_CASE_FAILED) return r->st.error;
  if (r->st.state != NS_CASE_DONE) return NS_ERR_STATE;
  if (u) std::copy(r->ru.begin(), r->ru.end(), u);
  if (v) std::copy(r->rv.begin(), r->rv.end(), v);
  if (a) std::copy(r->ra.begin(), r->ra.end(), a);
  return NS_OK;
}

int ns_server_release(ns_server *s, int64_t id) {
  if (!s) return NS_ERR_INVALID_ARG;
  std::unique_ptr<CaseRec> r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->cases.find(id);
    if (it == s->cases.end()) return NS_ERR_INVALID_ARG;
    if (it->second->st.state != NS_CASE_DONE && it->second->st.state != NS_CASE_FAILED) return NS_ERR_STATE;
    r = std::move(it->second);
    s->cases.erase(it);
  }
  if (r->th.joinable()) r->th.join();
  return NS_OK;
}

void ns_server_destroy(ns_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (int64_t id : s->queue) {
      CaseRec *r = s->cases[id].get();
      r->st.state = NS_CASE_FAILED;
      r->st.error = NS_ERR_STATE;
      r->err = "server stopped before admission";
    }
    s->queue.clear();
    s->cv.notify_all();
  }
  if (s->sched.joinable()) s->sched.join();
  for (auto &kv : s->cases)
    if (kv.second->th.joinable()) kv.second->th.join();
  for (auto &kv : s->classes)
    if (kv.second.th.joinable()) kv.second.th.join();
  delete s;
}

}  // extern "C"
