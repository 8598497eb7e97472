// Served ensemble runtime (include/ns_server.h): a first-come-first-served queue of
// independent cases, admitted into concurrent slots by device and pinned-host memory,
// each slot one context of the time stepper driven by its own host thread.
#include "../../include/ns_server.h"

#include <cuda_runtime.h>

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
  std::chrono::steady_clock::time_point t0;

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

namespace {

// Head of the queue admissible now?  Decides resident or streamed placement.
bool can_admit(ns_server *s, CaseRec &r) {
  if (s->active >= s->cfg.max_active) return false;
  if (s->dev_used + r.dev_resident <= s->cfg.device_budget) {
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
    r->th = std::thread(run_case, s, r);
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
  if (!out || !cfg || cfg->max_active < 1 || cfg->device_budget <= 0 || cfg->pinned_budget < 0 || cfg->device < 0)
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
  delete s;
}

}  // extern "C"
