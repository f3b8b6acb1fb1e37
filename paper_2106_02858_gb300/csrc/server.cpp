// Serving runtime: continuous batching of CMCG requests.
//
// A server owns registered models (a mesh with its materials, frequency and
// order) and a queue of requests (one source each).  Worker threads, each with
// its own CUDA stream, take the model of the oldest queued request, wait at
// most max_wait_ms for more of that model, and run a pooled batch handle of it
// as slots (cmcg_slot_*): every round advances each busy slot by one step of its
// solve, and between rounds requests of that model that have arrived meanwhile
// take the slots that finished requests left free, while the other slots keep
// iterating.  The worker keeps the handle while it has busy slots or queued
// requests of its model; several handles run concurrently on different streams.  Handles
// are created lazily and kept (no cudaFree while serving); a new handle is
// created only if the server's device-memory total stays within the HBM
// budget, otherwise the batch waits for a pooled handle to come back.  All
// handles of a model use the kernel form chosen once when the model is
// registered, so a request's result does not depend on which other requests
// share its batch (the batched arithmetic per problem is that of a solve
// alone).
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/cmcg.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Model {
  int order = 1, np = 4, capacity = 1, form = 0;
  std::vector<double> verts, eps, mu;
  std::vector<int32_t> tets;
  std::vector<uint8_t> tags;
  double omega = 0;
  cmcg_mesh mesh{};
  int64_t nt = 0;
  int64_t handle_bytes = 0;
  std::vector<cmcg_handle*> idle;
};

struct Request {
  int64_t ticket = 0;
  int model = 0;
  std::vector<double> jre, jim, ere, eim, hre, him;
  bool has_im = false;
  bool done = false;
  bool claimed = false;  // a poll is waiting on it or has taken its result
  int status = CMCG_OK;
  cmcg_info info{};
  Clock::time_point t_submit, t_start, t_end;
};

}  // namespace

struct cmcg_server {
  cmcg_server_options opt{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_handle;
  std::vector<std::unique_ptr<Model>> models;
  std::deque<Request*> queue;
  std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
  int64_t next_ticket = 1;
  int64_t bytes_in_use = 0;
  int nhandles = 0;
  int64_t completed = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<cmcg_handle*> all_handles;
};

namespace {

cmcg_options model_options(const cmcg_server* s, const Model& m, int form) {
  cmcg_options o;
  cmcg_default_options(&o);
  o.order = m.order;
  o.precision = s->opt.precision;
  o.device = s->opt.device;
  o.stage_variant = form;
  return o;
}

int create_handle(const cmcg_server* s, const Model& m, int form, cmcg_handle** out) {
  std::vector<cmcg_problem> probs(m.capacity, cmcg_problem{&m.mesh, m.eps.data(), m.mu.data(), m.omega});
  cmcg_options o = model_options(s, m, form);
  return cmcg_create_batch(m.capacity, probs.data(), &o, out);
}

void worker_main(cmcg_server* s) {
  cudaSetDevice(s->opt.device);
  cudaStream_t stream = nullptr;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  const auto window = std::chrono::microseconds(int64_t(s->opt.max_wait_ms * 1000.0));
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
    if (s->queue.empty()) {
      if (s->stop) break;
      continue;
    }
    Request* first = s->queue.front();
    const int mid = first->model;
    Model& m = *s->models[mid];
    // Micro-batching window before the first round: wait for more requests of this model.
    auto count = [&] {
      int c = 0;
      for (Request* r : s->queue)
        if (r->model == mid) ++c;
      return c;
    };
    const auto deadline = first->t_submit + window;
    while (!s->stop && count() < m.capacity && Clock::now() < deadline) s->cv_work.wait_until(lk, deadline);
    if (s->queue.empty() || s->queue.front() != first) continue;  // another worker took it
    // A handle: pooled, or new within the HBM budget, or wait for one to come back.
    cmcg_handle* h = nullptr;
    int rc = CMCG_OK;
    for (;;) {
      if (!m.idle.empty()) {
        h = m.idle.back();
        m.idle.pop_back();
        break;
      }
      const int64_t budget = s->opt.hbm_budget_bytes;
      if (budget <= 0 || s->bytes_in_use + m.handle_bytes <= budget) {
        s->bytes_in_use += m.handle_bytes;  // reserve
        lk.unlock();
        rc = create_handle(s, m, m.form, &h);
        lk.lock();
        if (rc == CMCG_OK) {
          s->bytes_in_use += cmcg_device_bytes(h) - m.handle_bytes;
          s->nhandles++;
          s->all_handles.push_back(h);
        } else {
          s->bytes_in_use -= m.handle_bytes;
        }
        break;
      }
      if (s->nhandles == 0) {  // nothing will ever come back
        rc = CMCG_ERR_OUT_OF_MEMORY;
        break;
      }
      s->cv_handle.wait(lk);
    }
    if (rc != CMCG_OK) {  // the oldest request of this model fails; the others wait for a handle
      for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
        if (*it == first) {
          s->queue.erase(it);
          break;
        }
      first->status = rc;
      first->t_start = first->t_end = Clock::now();
      first->done = true;
      s->completed++;
      s->cv_done.notify_all();
      continue;
    }
    cmcg_set_stream(h, stream);
    // Slot loop: requests of this model are admitted into free slots between rounds while the
    // others iterate; each round advances every busy slot (cmcg_slot_round).
    std::vector<Request*> slot(size_t(m.capacity), nullptr);
    int busy = 0;
    bool broken = false;
    for (;;) {
      std::vector<int> admit;
      for (int sl = 0; sl < m.capacity; ++sl) {
        if (slot[size_t(sl)]) continue;
        auto it = s->queue.begin();
        while (it != s->queue.end() && (*it)->model != mid) ++it;
        if (it == s->queue.end()) break;
        Request* r = *it;
        s->queue.erase(it);
        r->t_start = Clock::now();
        slot[size_t(sl)] = r;
        admit.push_back(sl);
        ++busy;
      }
      if (busy == 0) break;
      lk.unlock();
      std::vector<std::pair<int, int>> failed;  // (slot, status)
      for (int sl : admit) {
        Request* r = slot[size_t(sl)];
        const int arc = cmcg_slot_admit(h, sl, r->jre.data(), r->has_im ? r->jim.data() : nullptr);
        if (arc) failed.emplace_back(sl, arc);
      }
      std::vector<int> done(size_t(m.capacity), 0);
      int rrc = failed.size() == admit.size() && !admit.empty() && busy == int(admit.size())
                    ? CMCG_OK
                    : cmcg_slot_round(h, s->opt.tol, s->opt.max_iter, done.data());
      std::vector<std::pair<int, int>> finished;  // (slot, status)
      if (rrc == CMCG_OK) {
        for (int sl = 0; sl < m.capacity; ++sl) {
          if (!done[size_t(sl)]) continue;
          Request* r = slot[size_t(sl)];
          const size_t len = size_t(m.nt) * 3 * m.np;
          r->ere.resize(len);
          r->eim.resize(len);
          r->hre.resize(len);
          r->him.resize(len);
          const int st = cmcg_slot_take(h, sl, r->ere.data(), r->eim.data(), r->hre.data(), r->him.data(), &r->info);
          finished.emplace_back(sl, st);
        }
      }
      lk.lock();
      auto complete = [&](int sl, int st) {
        Request* r = slot[size_t(sl)];
        if (!r) return;
        r->status = st;
        r->t_end = Clock::now();
        r->done = true;
        r->jre.clear();
        r->jim.clear();
        slot[size_t(sl)] = nullptr;
        --busy;
        s->completed++;
      };
      for (auto& f : failed) complete(f.first, f.second);
      for (auto& f : finished) complete(f.first, f.second);
      if (rrc != CMCG_OK) {  // the handle's state is unknown: fail what it holds and drop it
        for (int sl = 0; sl < m.capacity; ++sl) complete(sl, rrc);
        broken = true;
      }
      if (!failed.empty() || !finished.empty() || broken) s->cv_done.notify_all();
      if (broken) break;
    }
    if (broken) {
      s->bytes_in_use -= cmcg_device_bytes(h);
      s->nhandles--;
      for (auto it = s->all_handles.begin(); it != s->all_handles.end(); ++it)
        if (*it == h) {
          s->all_handles.erase(it);
          break;
        }
      lk.unlock();
      cmcg_destroy(h);
      lk.lock();
    } else {
      m.idle.push_back(h);
    }
    s->cv_handle.notify_all();
  }
  lk.unlock();
  cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

void cmcg_server_default_options(cmcg_server_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = CMCG_FP32;
  o->max_batch = 8;
  o->workers = 2;
  o->max_wait_ms = 2.0;
  o->tol = 1e-6;
  o->max_iter = 1000;
}

int cmcg_server_create(const cmcg_server_options* opt, cmcg_server** out) {
  if (!out) return CMCG_ERR_INVALID_ARG;
  *out = nullptr;
  cmcg_server_options o;
  if (opt) o = *opt;
  else cmcg_server_default_options(&o);
  if (o.max_batch < 1 || o.workers < 1 || o.workers > 64 || !(o.max_wait_ms >= 0) || !(o.tol >= 0) || o.max_iter < 0)
    return CMCG_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return CMCG_ERR_NO_DEVICE;
  if (o.device < 0 || o.device >= ndev) return CMCG_ERR_INVALID_ARG;
  cmcg_server* s = new cmcg_server();
  s->opt = o;
  for (int i = 0; i < o.workers; ++i) s->workers.emplace_back(worker_main, s);
  *out = s;
  return CMCG_OK;
}

int cmcg_server_add_model(cmcg_server* s, const cmcg_mesh* mesh, const double* eps, const double* mu, double omega,
                          int order, int max_batch, int* model) {
  if (!s || !mesh || !eps || !mu || !model || order < 1 || order > 3 || max_batch < 0) return CMCG_ERR_INVALID_ARG;
  if (!mesh->verts || !mesh->tets || !mesh->face_tags || mesh->nt <= 0 || mesh->nv <= 0) return CMCG_ERR_INVALID_ARG;
  auto m = std::make_unique<Model>();
  m->order = order;
  m->np = (order + 1) * (order + 2) * (order + 3) / 6;
  m->capacity = max_batch > 0 ? max_batch : s->opt.max_batch;
  m->verts.assign(mesh->verts, mesh->verts + 3 * mesh->nv);
  m->tets.assign(mesh->tets, mesh->tets + 4 * mesh->nt);
  m->tags.assign(mesh->face_tags, mesh->face_tags + 4 * mesh->nt);
  m->eps.assign(eps, eps + mesh->nt);
  m->mu.assign(mu, mu + mesh->nt);
  m->omega = omega;
  m->nt = mesh->nt;
  m->mesh = cmcg_mesh{mesh->nv, m->verts.data(), mesh->nt, m->tets.data(), m->tags.data()};
  // First handle: validates the model, chooses the kernel form for all its handles, joins the pool.
  cmcg_handle* h = nullptr;
  int rc = create_handle(s, *m, s->opt.stage_variant, &h);
  if (rc != CMCG_OK) return rc;
  int form = 0;
  cmcg_get_tuning(h, &form, nullptr);
  m->form = form + 1;
  m->handle_bytes = cmcg_device_bytes(h);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->opt.hbm_budget_bytes > 0 && s->bytes_in_use + m->handle_bytes > s->opt.hbm_budget_bytes) {
    cmcg_destroy(h);
    return CMCG_ERR_OUT_OF_MEMORY;
  }
  s->bytes_in_use += m->handle_bytes;
  s->nhandles++;
  s->all_handles.push_back(h);
  m->idle.push_back(h);
  *model = int(s->models.size());
  s->models.push_back(std::move(m));
  return CMCG_OK;
}

int cmcg_server_submit(cmcg_server* s, int model, const double* j_re, const double* j_im, int64_t* ticket) {
  if (!s || !j_re || !ticket) return CMCG_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (model < 0 || model >= int(s->models.size()) || s->stop) return CMCG_ERR_INVALID_ARG;
  const Model& m = *s->models[model];
  const size_t len = size_t(m.nt) * 3 * m.np;
  auto r = std::make_unique<Request>();
  r->ticket = s->next_ticket++;
  r->model = model;
  r->jre.assign(j_re, j_re + len);
  if (j_im) {
    r->jim.assign(j_im, j_im + len);
    r->has_im = true;
  }
  r->t_submit = Clock::now();
  *ticket = r->ticket;
  s->queue.push_back(r.get());
  s->reqs.emplace(r->ticket, std::move(r));
  s->cv_work.notify_all();
  return CMCG_OK;
}

int cmcg_server_poll(cmcg_server* s, int64_t ticket, int wait, double* e_re, double* e_im, double* h_re,
                     double* h_im, cmcg_info* info, double* latency_ms) {
  if (!s) return CMCG_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return CMCG_ERR_INVALID_ARG;
  Request* r = it->second.get();
  // One poll per ticket takes the result: a second poll of a ticket that another thread is
  // already waiting on is refused here, before it could wait on a request the first poll frees.
  if (r->claimed) return CMCG_ERR_INVALID_ARG;
  if (!r->done) {
    if (!wait) return CMCG_PENDING;
    r->claimed = true;
    s->cv_done.wait(lk, [&] { return r->done; });
  }
  r->claimed = true;
  const size_t len = r->ere.size();
  if (r->status >= 0) {
    if (e_re) std::memcpy(e_re, r->ere.data(), len * 8);
    if (e_im) std::memcpy(e_im, r->eim.data(), len * 8);
    if (h_re) std::memcpy(h_re, r->hre.data(), len * 8);
    if (h_im) std::memcpy(h_im, r->him.data(), len * 8);
  }
  if (info) *info = r->info;
  if (latency_ms) {
    latency_ms[0] = std::chrono::duration<double, std::milli>(r->t_end - r->t_submit).count();
    latency_ms[1] = std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count();
  }
  const int st = r->status;
  s->reqs.erase(it);
  return st;
}

int cmcg_server_stats(cmcg_server* s, int64_t* completed, int64_t* queued, int64_t* bytes_in_use, int* handles) {
  if (!s) return CMCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (completed) *completed = s->completed;
  if (queued) *queued = int64_t(s->queue.size());
  if (bytes_in_use) *bytes_in_use = s->bytes_in_use;
  if (handles) *handles = s->nhandles;
  return CMCG_OK;
}

void cmcg_server_destroy(cmcg_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_handle.notify_all();
  for (auto& t : s->workers) t.join();
  for (cmcg_handle* h : s->all_handles) cmcg_destroy(h);
  delete s;
}

}  // extern "C"
