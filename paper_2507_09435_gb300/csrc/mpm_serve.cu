// Continuous-batching serving loop over implicit-MPM scenes (declared in
// include/mpm_serve.h).  Host code only: worker threads, each with its own
// CUDA stream, take requests from a FIFO queue when a slot is free and the
// request's device footprint fits in the memory budget beside the running
// ones, and drive each request's scene through its load steps with the C ABI
// of mpm.h.  Concurrent scenes overlap on the device through their streams.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "mpm.h"
#include "mpm_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

template <class T>
std::vector<T> copy_of(const T* p, size_t n) {
  return p ? std::vector<T>(p, p + n) : std::vector<T>();
}

struct Request {
  long long id = 0;
  mpm_scene_desc desc{};
  int np = 0, nmat = 0, nsteps = 0;
  std::vector<double> x, vol0, mass, E_p, phi_p, pc0_p, be0;
  std::vector<int> mat_id;
  std::vector<mpm_material> mats;
  std::vector<int> trac_p;
  std::vector<double> trac_f;
  std::vector<int> step_ndof;
  std::vector<long long> step_dof;
  std::vector<double> step_value, step_grav;
  size_t footprint = 0;
  Clock::time_point t_submit, t_start, t_end;
  bool done = false;
  mpm_request_result res{};
  std::vector<double> out_x, out_pp;
};

}  // namespace

struct mpm_server {
  int slots = 0;
  int device = 0;
  size_t budget = 0, in_use = 0, peak_in_use = 0;
  int running = 0, peak_running = 0;
  long long next_id = 1, submitted = 0, completed = 0, failed = 0;
  bool stop = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::map<long long, std::unique_ptr<Request>> reqs;
  std::vector<std::thread> workers;
};

namespace {

// Run one request on this worker's stream; fills req->res and the outputs.
void run_request(Request* r, cudaStream_t st, int slot) {
  mpm_request_result& R = r->res;
  R.slot = slot;
  R.footprint = r->footprint;
  mpm_scene* s = nullptr;
  mpm_status rc = mpm_create_scene(&r->desc, r->np, r->x.data(), r->vol0.data(), r->mass.data(),
                                   r->mat_id.data(), r->E_p.empty() ? nullptr : r->E_p.data(),
                                   r->phi_p.empty() ? nullptr : r->phi_p.data(),
                                   r->pc0_p.empty() ? nullptr : r->pc0_p.data(), r->mats.data(), r->nmat,
                                   (void*)st, &s);
  if (rc == MPM_OK && !r->be0.empty()) rc = mpm_set_particles(s, r->be0.data(), nullptr, nullptr);
  if (rc == MPM_OK && !r->trac_p.empty())
    rc = mpm_set_traction(s, (int)r->trac_p.size(), r->trac_p.data(), r->trac_f.data());
  size_t off = 0;
  for (int k = 0; rc == MPM_OK && k < r->nsteps; ++k) {
    const int n = r->step_ndof[k];
    rc = mpm_set_dirichlet(s, n, r->step_dof.data() + off, r->step_value.data() + off);
    off += (size_t)n;
    if (rc == MPM_OK) rc = mpm_set_gravity(s, r->step_grav.data() + 3 * (size_t)k);
    mpm_step_report rep{};
    if (rc == MPM_OK) rc = mpm_solve_step(s, &rep);
    R.newton_iters += rep.newton_iters;
    R.krylov_iters += rep.krylov_iters_total;
    if (rc == MPM_OK) R.steps_done += 1;
  }
  if (s && rc == MPM_OK) {
    r->out_x.assign((size_t)r->np * 3, 0.0);
    rc = mpm_get_particles(s, r->out_x.data(), nullptr, nullptr, nullptr, nullptr);
    if (rc == MPM_OK && r->desc.formulation == MPM_UP) {
      r->out_pp.assign((size_t)r->np, 0.0);
      rc = mpm_get_pressure(s, r->out_pp.data());
    }
  }
  if (s) mpm_destroy_scene(s);
  R.status = rc;
}

void worker(mpm_server* sv, int slot) {
  cudaSetDevice(sv->device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      // admission: FIFO head, when it fits in the budget beside the running
      // requests (or when nothing runs, so that an oversized request runs alone)
      sv->cv_work.wait(lk, [&] {
        if (sv->stop) return true;
        if (sv->queue.empty()) return false;
        const Request* h = sv->queue.front();
        return sv->running == 0 || sv->in_use + h->footprint <= sv->budget;
      });
      if (sv->stop) break;
      r = sv->queue.front();
      sv->queue.pop_front();
      sv->in_use += r->footprint;
      sv->running += 1;
      sv->peak_in_use = std::max(sv->peak_in_use, sv->in_use);
      sv->peak_running = std::max(sv->peak_running, sv->running);
      r->t_start = Clock::now();
    }
    // another queued request may fit as well
    sv->cv_work.notify_all();
    if (st) run_request(r, st, slot);
    else r->res.status = MPM_ERR_CUDA;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      r->t_end = Clock::now();
      r->res.t_queue_ms = ms_between(r->t_submit, r->t_start);
      r->res.t_service_ms = ms_between(r->t_start, r->t_end);
      r->res.t_latency_ms = ms_between(r->t_submit, r->t_end);
      r->done = true;
      sv->in_use -= r->footprint;
      sv->running -= 1;
      sv->completed += 1;
      if (r->res.status != MPM_OK) sv->failed += 1;
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
  }
  if (st) cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

mpm_status mpm_server_create(int slots, size_t budget_bytes, mpm_server** out) {
  if (!out || slots < 1 || slots > 64) return MPM_ERR_INVALID_ARG;
  *out = nullptr;
  auto* sv = new (std::nothrow) mpm_server();
  if (!sv) return MPM_ERR_OOM;
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    return MPM_ERR_CUDA;
  }
  if (budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      delete sv;
      return MPM_ERR_CUDA;
    }
    budget_bytes = fr / 10 * 8;
  }
  sv->slots = slots;
  sv->budget = budget_bytes;
  try {
    for (int k = 0; k < slots; ++k) sv->workers.emplace_back(worker, sv, k);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto& t : sv->workers) t.join();
    delete sv;
    return MPM_ERR_INVALID_ARG;
  }
  *out = sv;
  return MPM_OK;
}

mpm_status mpm_server_submit(mpm_server* sv, const mpm_request* q, long long* ticket) {
  if (!sv || !q || !ticket || !q->desc || q->np < 0 || q->nmat < 1 || !q->mats || q->nsteps < 0 ||
      q->ntraction < 0)
    return MPM_ERR_INVALID_ARG;
  if (q->np > 0 && (!q->x || !q->vol0 || !q->mass || !q->mat_id)) return MPM_ERR_INVALID_ARG;
  if (q->nsteps > 0 && (!q->step_ndof || !q->step_gravity)) return MPM_ERR_INVALID_ARG;
  if (q->ntraction > 0 && (!q->traction_particle || !q->traction_force)) return MPM_ERR_INVALID_ARG;
  size_t fp = 0;
  mpm_status rc = mpm_footprint_bytes(q->desc, q->np, &fp);
  if (rc != MPM_OK) return rc;
  auto r = std::make_unique<Request>();
  try {
    const size_t np = (size_t)q->np;
    r->desc = *q->desc;
    r->np = q->np;
    r->nmat = q->nmat;
    r->nsteps = q->nsteps;
    r->x = copy_of(q->x, np * 3);
    r->vol0 = copy_of(q->vol0, np);
    r->mass = copy_of(q->mass, np);
    r->mat_id = copy_of(q->mat_id, np);
    r->E_p = copy_of(q->E_p, np);
    r->phi_p = copy_of(q->phi_p, np);
    r->pc0_p = copy_of(q->pc0_p, np);
    r->be0 = copy_of(q->be0, np * 6);
    r->mats = copy_of(q->mats, (size_t)q->nmat);
    r->trac_p = copy_of(q->traction_particle, (size_t)q->ntraction);
    r->trac_f = copy_of(q->traction_force, (size_t)q->ntraction * 3);
    r->step_ndof = copy_of(q->step_ndof, (size_t)q->nsteps);
    size_t tot = 0;
    for (int k = 0; k < q->nsteps; ++k) {
      if (q->step_ndof[k] < 0) return MPM_ERR_INVALID_ARG;
      tot += (size_t)q->step_ndof[k];
    }
    if (tot > 0 && (!q->step_dof || !q->step_value)) return MPM_ERR_INVALID_ARG;
    r->step_dof = copy_of(q->step_dof, tot);
    r->step_value = copy_of(q->step_value, tot);
    r->step_grav = copy_of(q->step_gravity, (size_t)q->nsteps * 3);
  } catch (...) {
    return MPM_ERR_OOM;
  }
  r->footprint = fp;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->id = sv->next_id++;
    r->t_submit = Clock::now();
    *ticket = r->id;
    sv->queue.push_back(r.get());
    sv->reqs[r->id] = std::move(r);
    sv->submitted += 1;
  }
  sv->cv_work.notify_all();
  return MPM_OK;
}

mpm_status mpm_server_wait(mpm_server* sv, long long ticket, mpm_request_result* out) {
  if (!sv || !out) return MPM_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return MPM_ERR_INVALID_ARG;
  Request* r = it->second.get();
  sv->cv_done.wait(lk, [&] { return r->done; });
  *out = r->res;
  return MPM_OK;
}

mpm_status mpm_server_result_particles(mpm_server* sv, long long ticket, double* x, double* pp) {
  if (!sv) return MPM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end() || !it->second->done) return MPM_ERR_INVALID_ARG;
  Request* r = it->second.get();
  if (r->res.status != MPM_OK) return (mpm_status)r->res.status;
  if (x) std::copy(r->out_x.begin(), r->out_x.end(), x);
  if (pp) {
    if (r->out_pp.empty()) return MPM_ERR_INVALID_ARG;
    std::copy(r->out_pp.begin(), r->out_pp.end(), pp);
  }
  return MPM_OK;
}

mpm_status mpm_server_release(mpm_server* sv, long long ticket) {
  if (!sv) return MPM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end() || !it->second->done) return MPM_ERR_INVALID_ARG;
  sv->reqs.erase(it);
  return MPM_OK;
}

mpm_status mpm_server_get_stats(const mpm_server* csv, mpm_server_stats* out) {
  mpm_server* sv = const_cast<mpm_server*>(csv);
  if (!sv || !out) return MPM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  out->slots = sv->slots;
  out->budget = sv->budget;
  out->in_use = sv->in_use;
  out->peak_in_use = sv->peak_in_use;
  out->running = sv->running;
  out->peak_running = sv->peak_running;
  out->submitted = sv->submitted;
  out->completed = sv->completed;
  out->failed = sv->failed;
  return MPM_OK;
}

void mpm_server_destroy(mpm_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    // queued requests are dropped: mark them done with an error
    for (Request* r : sv->queue) {
      r->res.status = MPM_ERR_STATE;
      r->done = true;
    }
    sv->queue.clear();
  }
  sv->cv_work.notify_all();
  sv->cv_done.notify_all();
  for (auto& t : sv->workers) t.join();
  delete sv;
}

}  // extern "C"
