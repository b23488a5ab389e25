// Serving runtime: solves of different mesh sizes admitted continuously under
// a device-memory budget, each in its own slot (worker thread + CUDA stream),
// so that the kernels of the requests in flight overlap on the GPU.  Built on
// the public mesh API of afd.h only.
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

struct Slot {
  std::thread th;
  cudaStream_t stream = nullptr;
  afd_mesh* mesh = nullptr;   // kept for a request of the same size
  int nx = 0, ny = 0, nz = 0;
  size_t bytes = 0;           // budget held by the kept mesh
};

}  // namespace

struct afd_server {
  afd_server_config cfg;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<int64_t, std::shared_ptr<Request>> all;
  int64_t next_id = 1;
  double in_use = 0.0;        // bytes held by meshes in flight or kept by slots
  bool stopping = false;
  std::vector<std::unique_ptr<Slot>> slots;
};

namespace {

// One slot: take the head of the queue when the budget allows (dropping the
// slot's kept mesh if that makes room), solve it on the slot's stream, keep
// the mesh for a later request of the same size.
void worker(afd_server* S, Slot* slot) {
  cudaSetDevice(S->device);
  cudaStreamCreateWithFlags(&slot->stream, cudaStreamNonBlocking);
  for (;;) {
    std::shared_ptr<Request> req;
    bool reuse = false;
    afd_mesh* drop = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->queue.empty()) {
          if (S->stopping) {
            drop = slot->mesh;
            S->in_use -= (double)slot->bytes;
            slot->mesh = nullptr;
            slot->bytes = 0;
            lk.unlock();
            if (drop) afd_destroy(drop);
            if (slot->stream) cudaStreamDestroy(slot->stream);
            return;
          }
          S->cv_work.wait(lk);
          continue;
        }
        const std::shared_ptr<Request>& head = S->queue.front();
        const bool same = slot->mesh && slot->nx == head->nx && slot->ny == head->ny && slot->nz == head->nz;
        const double need = same ? 0.0 : (double)head->bytes;
        const double freed = same ? 0.0 : (double)slot->bytes;
        if (S->in_use - freed + need <= S->cfg.budget_bytes) {
          req = head;
          S->queue.pop_front();
          S->in_use += need - freed;
          reuse = same;
          if (!same) {
            drop = slot->mesh;
            slot->mesh = nullptr;
            slot->bytes = req->bytes;
            slot->nx = req->nx;
            slot->ny = req->ny;
            slot->nz = req->nz;
          }
          break;
        }
        // the head does not fit: give back this slot's kept mesh so that it can
        if (slot->mesh) {
          afd_mesh* m = slot->mesh;
          S->in_use -= (double)slot->bytes;
          slot->mesh = nullptr;
          slot->bytes = 0;
          lk.unlock();
          afd_destroy(m);
          lk.lock();
          S->cv_work.notify_all();
          continue;
        }
        S->cv_work.wait(lk);
      }
    }
    if (drop) afd_destroy(drop);
    int rc = AFD_OK;
    std::string err;
    if (!reuse) {
      rc = afd_create_mesh(req->nx, req->ny, req->nz, &S->cfg.opt, slot->stream, &slot->mesh);
      if (rc != AFD_OK) {
        err = afd_last_error();
        slot->mesh = nullptr;
      }
    }
    afd_mesh* m = slot->mesh;
    const size_t ndof = 3 * (size_t)(req->nx + 1) * (req->ny + 1) * (req->nz + 1);
    std::vector<double> u(ndof, 0.0);
    afd_stats st{};
    double J = 0.0;
    if (rc == AFD_OK) rc = afd_set_element_moduli(m, req->E.data(), 0);
    if (rc == AFD_OK) rc = afd_set_loads_bcs(m, 1, req->f.data(), 0, req->fixed.data(), 0);
    if (rc == AFD_OK) {
      rc = afd_solve(m, req->tol, 0, &st, u.data(), 0);
      if (rc == AFD_OK || rc == AFD_ERR_NOT_CONVERGED) {
        const int rj = afd_compliance(m, &J);
        if (rc == AFD_OK) rc = rj;
      }
    }
    if (rc != AFD_OK && err.empty()) err = afd_last_error();
    const double ms = std::chrono::duration<double, std::milli>(Clock::now() - req->submitted).count();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (rc != AFD_OK && rc != AFD_ERR_NOT_CONVERGED && slot->mesh) {
        // a failed mesh is not kept
        afd_mesh* bad = slot->mesh;
        slot->mesh = nullptr;
        S->in_use -= (double)slot->bytes;
        slot->bytes = 0;
        afd_destroy(bad);
      } else if (!slot->mesh) {
        S->in_use -= (double)slot->bytes;
        slot->bytes = 0;
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

int afd_server_submit(afd_server* S, int nx, int ny, int nz, const double* E, const double* f,
                      const uint8_t* fixed_dof_mask, double rel_tol, int64_t* id_out) {
  if (!S || !E || !f || !fixed_dof_mask || !id_out || nx < 1 || ny < 1 || nz < 1 || !(rel_tol > 0))
    return AFD_ERR_INVALID_ARG;
  auto r = std::make_shared<Request>();
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

void afd_server_destroy(afd_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  for (auto& sl : S->slots)
    if (sl->th.joinable()) sl->th.join();
  delete S;
}
