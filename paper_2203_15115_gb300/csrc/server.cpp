// Serving runtime: solves of different mesh sizes admitted continuously under
// a device-memory budget, each in its own slot (worker thread + CUDA stream),
// so that the kernels of the requests in flight overlap on the GPU.  Built on
// the public mesh API of afd.h only.
//
// Meshes live in a server-wide pool: a finished request leaves its mesh
// (vectors, coarse factor, tuned stencil shape) resident and idle, the next
// request of the same size takes it without allocating, and idle meshes are
// destroyed least-recently-used first only when the budget needs the room.
// A session (a client's successive level-set iterations) keeps its own mesh;
// when its loads and supports are unchanged the next solve starts from the
// previous solution.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/afd.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  int64_t session = 0;       // 0: none
  int nx = 0, ny = 0, nz = 0;
  std::vector<double> E, f;
  std::vector<uint8_t> fixed;
  double tol = 1e-6;
  size_t bytes = 0;
  Clock::time_point submitted;
  // result
  bool done = false;
  int status = AFD_OK;
  afd_stats stats{};
  double J = 0.0;
  double latency_ms = 0.0;
  std::vector<double> u;
  std::string error;
};

// A resident mesh of the pool.
struct PoolMesh {
  afd_mesh* m = nullptr;      // null while being created
  int nx = 0, ny = 0, nz = 0;
  size_t bytes = 0;
  int64_t session = 0;        // owner session (0: shared by size)
  bool busy = false;
  uint64_t last_used = 0;
  // session meshes: the loads and supports of the last solve (warm start when unchanged)
  std::vector<double> f_last;
  std::vector<uint8_t> fixed_last;
  bool has_solution = false;
};

struct Slot {
  std::thread th;
  cudaStream_t stream = nullptr;
};

}  // namespace

struct afd_server {
  afd_server_config cfg;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<int64_t, std::shared_ptr<Request>> all;
  std::vector<std::unique_ptr<PoolMesh>> pool;
  int64_t next_id = 1;
  uint64_t tick = 0;
  double in_use = 0.0;        // bytes of all resident meshes (busy, idle or being created)
  bool stopping = false;
  std::vector<std::unique_ptr<Slot>> slots;
};

namespace {

bool same_dims(const PoolMesh& p, const Request& r) { return p.nx == r.nx && p.ny == r.ny && p.nz == r.nz; }

// Remove pool entry i (the caller destroys its mesh outside the lock).
afd_mesh* pool_remove(afd_server* S, size_t i) {
  afd_mesh* m = S->pool[i]->m;
  S->in_use -= (double)S->pool[i]->bytes;
  S->pool.erase(S->pool.begin() + (long)i);
  return m;
}

// Admission of the queue head (lock held).  Returns the pool entry to solve
// on (busy, possibly still to be created: m == null), or null when the head
// has to wait.  Idle meshes to destroy are appended to `drop`.
PoolMesh* admit(afd_server* S, const Request& h, std::vector<afd_mesh*>& drop) {
  if (h.session) {
    for (auto& p : S->pool)
      if (p->session == h.session) {
        if (p->busy) return nullptr;               // the session's previous request is still running
        if (same_dims(*p, h)) {
          p->busy = true;
          return p.get();
        }
        p->busy = true;                            // resized session: replace its mesh below
        for (size_t i = 0; i < S->pool.size(); ++i)
          if (S->pool[i].get() == p.get()) {
            drop.push_back(pool_remove(S, i));
            break;
          }
        break;
      }
  } else {
    PoolMesh* best = nullptr;
    for (auto& p : S->pool)
      if (!p->busy && p->session == 0 && p->m && same_dims(*p, h) && (!best || p->last_used > best->last_used))
        best = p.get();
    if (best) {
      best->busy = true;
      return best;
    }
  }
  // a new mesh: make room by destroying idle meshes, least recently used first
  while (S->in_use + (double)h.bytes > S->cfg.budget_bytes) {
    size_t victim = S->pool.size();
    for (size_t i = 0; i < S->pool.size(); ++i)
      if (!S->pool[i]->busy && S->pool[i]->m &&
          (victim == S->pool.size() || S->pool[i]->last_used < S->pool[victim]->last_used))
        victim = i;
    if (victim == S->pool.size()) return nullptr;   // everything resident is in use: wait
    drop.push_back(pool_remove(S, victim));
  }
  S->pool.emplace_back(new PoolMesh());
  PoolMesh* p = S->pool.back().get();
  p->nx = h.nx;
  p->ny = h.ny;
  p->nz = h.nz;
  p->bytes = h.bytes;
  p->session = h.session;
  p->busy = true;
  S->in_use += (double)h.bytes;
  return p;
}

// One slot: take the head of the queue when admission allows, solve it on a
// pooled mesh with the slot's stream, give the mesh back to the pool.
void worker(afd_server* S, Slot* slot) {
  cudaSetDevice(S->device);
  cudaStreamCreateWithFlags(&slot->stream, cudaStreamNonBlocking);
  for (;;) {
    std::shared_ptr<Request> req;
    PoolMesh* pm = nullptr;
    std::vector<afd_mesh*> drop;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->queue.empty()) {
          if (S->stopping) {
            lk.unlock();
            if (slot->stream) cudaStreamDestroy(slot->stream);
            return;
          }
          S->cv_work.wait(lk);
          continue;
        }
        pm = admit(S, *S->queue.front(), drop);
        if (pm) {
          req = S->queue.front();
          S->queue.pop_front();
          break;
        }
        S->cv_work.wait(lk);
      }
    }
    for (afd_mesh* d : drop) afd_destroy(d);
    int rc = AFD_OK;
    std::string err;
    if (!pm->m) {
      afd_mesh* nm = nullptr;
      rc = afd_create_mesh(req->nx, req->ny, req->nz, &S->cfg.opt, slot->stream, &nm);
      if (rc != AFD_OK) err = afd_last_error();
      pm->m = nm;
      pm->has_solution = false;
    }
    afd_mesh* m = pm->m;
    const size_t ndof = 3 * (size_t)(req->nx + 1) * (req->ny + 1) * (req->nz + 1);
    std::vector<double> u(ndof, 0.0);
    afd_stats st{};
    double J = 0.0;
    // warm start: a session mesh whose last solve had the same loads and supports
    const bool warm = rc == AFD_OK && req->session && pm->has_solution && pm->f_last == req->f &&
                      pm->fixed_last == req->fixed;
    if (rc == AFD_OK) rc = afd_set_element_moduli(m, req->E.data(), 0);
    if (rc == AFD_OK && !warm) rc = afd_set_loads_bcs(m, 1, req->f.data(), 0, req->fixed.data(), 0);
    if (rc == AFD_OK) {
      rc = afd_solve(m, req->tol, warm ? 1 : 0, &st, u.data(), 0);
      if (rc == AFD_OK || rc == AFD_ERR_NOT_CONVERGED) {
        const int rj = afd_compliance(m, &J);
        if (rc == AFD_OK) rc = rj;
      }
    }
    if (rc != AFD_OK && err.empty()) err = afd_last_error();
    const double ms = std::chrono::duration<double, std::milli>(Clock::now() - req->submitted).count();
    afd_mesh* bad = nullptr;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if ((rc != AFD_OK && rc != AFD_ERR_NOT_CONVERGED) || !pm->m) {
        // a failed mesh is not kept
        for (size_t i = 0; i < S->pool.size(); ++i)
          if (S->pool[i].get() == pm) {
            bad = pool_remove(S, i);
            break;
          }
      } else {
        pm->busy = false;
        pm->last_used = ++S->tick;
        if (pm->session) {
          pm->has_solution = rc == AFD_OK;
          if (!warm) {
            pm->f_last = req->f;
            pm->fixed_last = req->fixed;
          }
        }
      }
      req->status = rc;
      req->stats = st;
      req->J = J;
      req->latency_ms = ms;
      req->u.swap(u);
      req->error = err;
      req->E.clear();
      req->E.shrink_to_fit();
      req->f.clear();
      req->f.shrink_to_fit();
      req->done = true;
    }
    if (bad) afd_destroy(bad);
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

}  // namespace

int afd_server_create(const afd_server_config* cfg, afd_server** out) {
  if (!cfg || !out || cfg->max_slots < 1 || cfg->max_slots > 64 || !(cfg->budget_bytes > 0)) return AFD_ERR_INVALID_ARG;
  *out = nullptr;
  afd_server* S = new afd_server();
  S->cfg = *cfg;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return AFD_ERR_CUDA;
  }
  for (int i = 0; i < cfg->max_slots; ++i) {
    S->slots.emplace_back(new Slot());
    Slot* sl = S->slots.back().get();
    sl->th = std::thread(worker, S, sl);
  }
  *out = S;
  return AFD_OK;
}

int afd_server_submit_session(afd_server* S, int64_t session, int nx, int ny, int nz, const double* E, const double* f,
                              const uint8_t* fixed_dof_mask, double rel_tol, int64_t* id_out) {
  if (!S || !E || !f || !fixed_dof_mask || !id_out || nx < 1 || ny < 1 || nz < 1 || !(rel_tol > 0) || session < 0)
    return AFD_ERR_INVALID_ARG;
  auto r = std::make_shared<Request>();
  r->session = session;
  r->nx = nx;
  r->ny = ny;
  r->nz = nz;
  const size_t ne = (size_t)nx * ny * nz, ndof = 3 * (size_t)(nx + 1) * (ny + 1) * (nz + 1);
  r->E.assign(E, E + ne);
  r->f.assign(f, f + ndof);
  r->fixed.assign(fixed_dof_mask, fixed_dof_mask + ndof);
  r->tol = rel_tol;
  r->bytes = afd_mesh_bytes(nx, ny, nz, 1, &S->cfg.opt);
  if ((double)r->bytes > S->cfg.budget_bytes) return AFD_ERR_OOM;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return AFD_ERR_STATE;
    r->id = S->next_id++;
    r->submitted = Clock::now();
    S->all[r->id] = r;
    S->queue.push_back(r);
  }
  S->cv_work.notify_all();
  *id_out = r->id;
  return AFD_OK;
}

int afd_server_submit(afd_server* S, int nx, int ny, int nz, const double* E, const double* f,
                      const uint8_t* fixed_dof_mask, double rel_tol, int64_t* id_out) {
  return afd_server_submit_session(S, 0, nx, ny, nz, E, f, fixed_dof_mask, rel_tol, id_out);
}

int afd_server_end_session(afd_server* S, int64_t session) {
  if (!S || session <= 0) return AFD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  for (auto& p : S->pool)
    if (p->session == session) {
      // the mesh stays resident as an ordinary pooled mesh of its size
      p->session = 0;
      p->has_solution = false;
      p->f_last.clear();
      p->fixed_last.clear();
    }
  S->cv_work.notify_all();
  return AFD_OK;
}

int afd_server_wait(afd_server* S, int64_t id, afd_stats* stats, double* J_out, double* latency_ms, double* u_out) {
  if (!S) return AFD_ERR_INVALID_ARG;
  std::shared_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return AFD_ERR_INVALID_ARG;
    r = it->second;
    S->cv_done.wait(lk, [&] { return r->done; });
    S->all.erase(it);
  }
  if (stats) *stats = r->stats;
  if (J_out) *J_out = r->J;
  if (latency_ms) *latency_ms = r->latency_ms;
  if (u_out && !r->u.empty()) memcpy(u_out, r->u.data(), r->u.size() * sizeof(double));
  return r->status;
}

int afd_server_resident(afd_server* S, int* meshes, double* bytes) {
  if (!S) return AFD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  if (meshes) *meshes = (int)S->pool.size();
  if (bytes) *bytes = S->in_use;
  return AFD_OK;
}

void afd_server_destroy(afd_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  for (auto& sl : S->slots)
    if (sl->th.joinable()) sl->th.join();
  for (auto& p : S->pool)
    if (p->m) afd_destroy(p->m);
  S->pool.clear();
  delete S;
}
