// serve.cu -- continuous-batching request loop over many independent
// radiative-transfer problems on one GPU (the serving form of the library).
//
// A request is a whole problem: configuration, particles, initial state,
// constant sources and a number of backward-Euler steps of size dt.  The
// server keeps every admitted problem RESIDENT on the device (its particles,
// neighbour lists, operator, AMG hierarchy and Krylov vectors live in its own
// sph_rt handle, on its own CUDA stream) and interleaves their time steps:
//
//   submit   copies the request into host memory and queues it (FIFO)
//   admit    the scheduler moves queued requests onto the device while the
//            estimated device footprint of all resident problems stays under
//            the HBM budget (the estimate is replaced by the measured bytes
//            once the problem is set up)
//   run      worker threads take resident problems from a ready queue, advance
//            each by `steps_per_tick` steps on the problem's own stream, and
//            put it back; work of different problems overlaps on the device
//   retire   a finished problem's state is copied out and its device memory
//            released, which lets the next queued request in
//   fuse     small requests (n_total <= fuse_max_n) that are ready at the
//            same time and share configuration, dt and step count run as one
//            sph_rt_batch: one persistent kernel launch per step for all of
//            them, all steps in one CUDA-graph launch
//
// Each problem's kernels are the library's deterministic kernels on its own
// data, so a request's result does not depend on what else is resident.
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

#include "common.cuh"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  int64_t id = 0;
  sph_rt_config cfg;
  int64_t n = 0;
  int32_t steps = 0, done_steps = 0;
  double dt = 0.0;
  std::vector<double> pos, mass, rho, h, sigma0, e0, E0, Qe, QE;
  std::vector<int32_t> kind;
  std::vector<int64_t> copy_of;
  bool has_copy = false, has_Qe = false, has_QE = false;
  // results
  std::vector<double> e, E;
  sph_rt_stats last{};
  int state = SPH_RT_SRV_QUEUED;
  sph_rt_status status = SPH_RT_OK;
  std::string err;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int64_t reserved = 0;  // bytes counted against the budget
  sph_rt *handle = nullptr;
  int64_t particle_steps = 0;
  int64_t n_int = 0;   // interior particles
  bool fused = false;  // ran in a fused batch
};

int64_t estimate_bytes(int dim, int64_t n) {
  // neighbour + operator + AMG bytes per stored pair, per-particle vectors,
  // with the mean neighbour count of a jittered lattice at h = 1.5 dx
  const double pairs = dim == 3 ? 113.0 : (dim == 2 ? 27.0 : 3.0);
  return (int64_t)(n * (pairs * 56.0 + 600.0)) + (int64_t)(8 << 20);
}

}  // namespace

struct sph_rt_srv {
  sph_rt_srv_config cfg;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Request>> queued;
  std::deque<std::shared_ptr<Request>> ready;
  std::map<int64_t, std::shared_ptr<Request>> all;
  std::vector<std::thread> workers;
  int64_t next_id = 1;
  int64_t resident_bytes = 0;
  int64_t peak_bytes = 0;
  int resident = 0, peak_resident = 0, busy = 0;
  std::vector<sph_rt *> idle;  // handles of retired requests, kept with their buffer pools
  bool stopping = false;
  std::string err;
  double t_first = 0, t_last = 0;
  int64_t total_particle_steps = 0;
  int64_t fused_requests = 0, fused_batches = 0;
  // launch shapes tuned by earlier fused batches (cfg.autotune), keyed by the
  // batch key's configuration bytes and dt: a later fused batch of the same
  // key reuses the shape instead of tuning again
  std::map<std::string, sph_rt_batch_shape> batch_shapes;
};

namespace {

int64_t handle_bytes(const sph_rt *s) {
  int64_t b = 0;
  for (auto &kv : s->alloc_size) b += (int64_t)kv.second;
  for (auto &kv : s->pool) b += (int64_t)kv.first;
  return b;
}

int64_t idle_bytes_locked(const sph_rt_srv *S) {
  int64_t b = 0;
  for (const sph_rt *h : S->idle) b += handle_bytes(h);
  return b;
}

// Admit as many queued requests as fit (called with the lock held).  Idle
// handles' pooled buffers count against the budget; they are given back to
// CUDA only when a queued request would not fit otherwise.
void admit_locked(sph_rt_srv *S) {
  while (!S->queued.empty()) {
    auto R = S->queued.front();
    int64_t est = estimate_bytes(R->cfg.dim, R->n);
    if (S->resident >= S->cfg.max_resident) break;
    bool empty = S->resident == 0;
    int64_t budget = (int64_t)S->cfg.hbm_budget_bytes;
    if (!empty && S->resident_bytes + idle_bytes_locked(S) + est > budget) {
      while (!S->idle.empty() && S->resident_bytes + idle_bytes_locked(S) + est > budget) {
        sph_rt_destroy(S->idle.back());
        S->idle.pop_back();
      }
      if (S->resident_bytes + est > budget) break;
    }
    S->queued.pop_front();
    R->reserved = est;
    S->resident_bytes += est;
    S->resident++;
    S->peak_resident = std::max(S->peak_resident, S->resident);
    R->state = SPH_RT_SRV_ADMITTED;
    R->t_admit = now_s();
    S->ready.push_back(R);
  }
}

// Set up a newly admitted request on the device (worker thread, no lock).
sph_rt_status setup_request(sph_rt_srv *S, Request *R) {
  sph_rt_config c = R->cfg;
  c.device = S->cfg.device;
  c.stream = nullptr;  // own stream per problem
  sph_rt *h = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->idle.empty()) {
      h = S->idle.back();
      S->idle.pop_back();
    }
  }
  if (h) {
    // reuse a retired handle: its stream and buffer pool stay, the problem
    // configuration is replaced (validated like sph_rt_create)
    sph_rt *probe = nullptr;
    sph_rt_status rc = sph_rt_create(&c, &probe);
    if (rc) {
      R->err = sph_rt_last_error(nullptr);
      std::lock_guard<std::mutex> lk(S->mu);
      S->idle.push_back(h);
      return rc;
    }
    sph_rt_destroy(probe);
    c.stream = h->cfg.stream;
    h->cfg = c;
    h->dim = c.dim;
    R->handle = h;
  } else {
    sph_rt_status rc = sph_rt_create(&c, &R->handle);
    if (rc) {
      R->err = sph_rt_last_error(nullptr);
      return rc;
    }
  }
  sph_rt_status rc = sph_rt_set_particles(R->handle, R->n, R->pos.data(), R->mass.data(), R->rho.data(),
                            R->h.data(), R->sigma0.data(), R->kind.data(),
                            R->has_copy ? R->copy_of.data() : nullptr, R->e0.data(),
                            R->E0.data());
  if (rc) R->err = sph_rt_last_error(R->handle);
  return rc;
}

void finish_request(sph_rt_srv *S, const std::shared_ptr<Request> &R, sph_rt_status rc) {
  if (R->handle) {
    if (rc == SPH_RT_OK) {
      R->e.resize(R->n);
      R->E.resize(R->n);
      rc = sph_rt_get_energies(R->handle, R->e.data(), R->E.data(), nullptr);
      if (rc) R->err = sph_rt_last_error(R->handle);
    } else if (R->err.empty()) {
      R->err = sph_rt_last_error(R->handle);
    }
    sphrt::free_all(R->handle);  // buffers go to the handle's pool for the next request
    R->handle->err.clear();
    std::lock_guard<std::mutex> lk(S->mu);
    S->idle.push_back(R->handle);
    R->handle = nullptr;
  }
  // host copies of the inputs are no longer needed
  R->pos.clear(); R->pos.shrink_to_fit();
  R->mass.clear(); R->mass.shrink_to_fit();
  R->rho.clear(); R->rho.shrink_to_fit();
  R->h.clear(); R->h.shrink_to_fit();
  R->sigma0.clear(); R->sigma0.shrink_to_fit();
  R->e0.clear(); R->e0.shrink_to_fit();
  R->E0.clear(); R->E0.shrink_to_fit();
  R->Qe.clear(); R->Qe.shrink_to_fit();
  R->QE.clear(); R->QE.shrink_to_fit();
  std::lock_guard<std::mutex> lk(S->mu);
  R->status = rc;
  R->state = rc == SPH_RT_OK ? SPH_RT_SRV_DONE : SPH_RT_SRV_FAILED;
  R->t_done = now_s();
  S->t_last = std::max(S->t_last, R->t_done);
  if (rc == SPH_RT_OK) S->total_particle_steps += R->particle_steps;
  S->resident_bytes -= R->reserved;
  S->resident--;
  admit_locked(S);
  S->cv.notify_all();
}

bool fusable(const sph_rt_srv *S, const Request &R) {
  return S->cfg.fuse_max_n > 0 && R.n <= S->cfg.fuse_max_n && !R.handle && R.done_steps == 0;
}

// Requests that can share one batch: same configuration (device and stream
// aside), dt and number of steps.
bool same_batch_key(const Request &a, const Request &b) {
  sph_rt_config ca, cb;
  memcpy(&ca, &a.cfg, sizeof ca);
  memcpy(&cb, &b.cfg, sizeof cb);
  ca.stream = cb.stream = nullptr;
  ca.device = cb.device = 0;
  return memcmp(&ca, &cb, sizeof ca) == 0 && a.dt == b.dt && a.steps == b.steps;
}

// Run a group of fused requests to completion as one batch (worker thread,
// no lock held).  Every member is finished here.
void run_fused(sph_rt_srv *S, std::vector<std::shared_ptr<Request>> &group) {
  sph_rt_config c = group[0]->cfg;
  c.device = S->cfg.device;
  c.stream = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto &R : group) {
      R->state = SPH_RT_SRV_RUNNING;
      R->fused = true;
    }
  }
  sph_rt_batch *B = nullptr;
  sph_rt_status rc = sph_rt_batch_create(&c, &B);
  if (rc) {
    for (auto &R : group) {
      R->err = sph_rt_last_error(nullptr);
      finish_request(S, R, rc);
    }
    return;
  }
  std::string shape_key;
  bool shape_known = false;
  if (c.autotune == 1) {
    sph_rt_config kc = c;
    kc.device = 0;
    const double dt = group[0]->dt;
    shape_key.assign(reinterpret_cast<const char *>(&kc), sizeof kc);
    shape_key.append(reinterpret_cast<const char *>(&dt), sizeof dt);
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->batch_shapes.find(shape_key);
    if (it != S->batch_shapes.end()) shape_known = sph_rt_batch_set_shape(B, &it->second) == 0;
  }
  std::vector<std::shared_ptr<Request>> members;
  std::vector<int32_t> index;
  // all members' set-ups at once (overlapping on the GPU); if that fails, one
  // by one, so that only the failing requests fail
  std::vector<sph_rt_problem> probs;
  for (auto &R : group)
    probs.push_back({R->n, R->pos.data(), R->mass.data(), R->rho.data(), R->h.data(),
                     R->sigma0.data(), R->kind.data(), R->has_copy ? R->copy_of.data() : nullptr,
                     R->e0.data(), R->E0.data()});
  int32_t first = 0;
  const bool all_in =
      sph_rt_batch_add_many(B, (int32_t)probs.size(), probs.data(), 4, &first) == SPH_RT_OK;
  for (size_t m = 0; m < group.size(); ++m) {
    auto &R = group[m];
    int32_t k = all_in ? first + (int32_t)m : -1;
    sph_rt_status r2 = SPH_RT_OK;
    if (!all_in)
      r2 = sph_rt_batch_add(B, R->n, R->pos.data(), R->mass.data(), R->rho.data(), R->h.data(),
                            R->sigma0.data(), R->kind.data(),
                            R->has_copy ? R->copy_of.data() : nullptr, R->e0.data(),
                            R->E0.data(), &k);
    if (!r2 && (R->has_Qe || R->has_QE))
      r2 = sph_rt_batch_set_sources(B, k, R->has_Qe ? R->Qe.data() : nullptr,
                                    R->has_QE ? R->QE.data() : nullptr);
    if (r2) {
      R->err = sph_rt_batch_last_error(B);
      finish_request(S, R, r2);
      continue;
    }
    members.push_back(R);
    index.push_back(k);
  }
  if (!members.empty()) {
    const size_t K = (size_t)sph_rt_batch_size(B);
    std::vector<int32_t> st(K, 0), ou(K, 0), kr(K, 0);
    rc = sph_rt_batch_run(B, members[0]->dt, members[0]->steps, st.data(), ou.data(), kr.data());
    const bool hard = rc != SPH_RT_OK && rc != SPH_RT_ENOTCONV;
    if (c.autotune == 1 && !shape_known && !hard) {
      sph_rt_batch_shape sh;
      if (sph_rt_batch_get_shape(B, &sh) == 0) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->batch_shapes.emplace(shape_key, sh);
      }
    }
    const std::string msg = rc ? sph_rt_batch_last_error(B) : "";
    for (size_t m = 0; m < members.size(); ++m) {
      auto &R = members[m];
      const int32_t k = index[m];
      sph_rt_status r2 = hard ? rc : (st[k] == 0 ? SPH_RT_OK : SPH_RT_ENOTCONV);
      if (r2 == SPH_RT_OK) {
        R->e.resize(R->n);
        R->E.resize(R->n);
        r2 = sph_rt_batch_get_energies(B, k, R->e.data(), R->E.data());
        R->last.outer_iters = ou[k];  // totals over the run for a fused request
        R->last.krylov_iters_total = kr[k];
        R->done_steps = R->steps;
        R->particle_steps = R->n_int * R->steps;
      }
      if (r2) R->err = hard ? msg : (r2 == SPH_RT_ENOTCONV ? "step did not converge" : sph_rt_batch_last_error(B));
      finish_request(S, R, r2);
    }
  }
  sph_rt_batch_destroy(B);
}

void worker_main(sph_rt_srv *S) {
  cudaSetDevice(S->cfg.device);
  for (;;) {
    std::shared_ptr<Request> R;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] { return S->stopping || !S->ready.empty(); });
      if (S->stopping) return;  // resident handles are released by destroy
      R = S->ready.front();
      S->ready.pop_front();
      S->busy++;
    }
    if (fusable(S, *R)) {
      std::vector<std::shared_ptr<Request>> group{R};
      {
        std::lock_guard<std::mutex> lk(S->mu);
        for (auto it = S->ready.begin();
             it != S->ready.end() && (int)group.size() < S->cfg.fuse_max_k;) {
          if (fusable(S, **it) && same_batch_key(*R, **it)) {
            group.push_back(*it);
            it = S->ready.erase(it);
          } else {
            ++it;
          }
        }
        S->fused_batches++;
        S->fused_requests += (int64_t)group.size();
      }
      run_fused(S, group);
      std::lock_guard<std::mutex> lk(S->mu);
      S->busy--;
      continue;
    }
    sph_rt_status rc = SPH_RT_OK;
    if (!R->handle) {
      rc = setup_request(S, R.get());
      if (rc == SPH_RT_OK) {
        std::lock_guard<std::mutex> lk(S->mu);
        int64_t actual = handle_bytes(R->handle);
        S->resident_bytes += actual - R->reserved;
        R->reserved = actual;
        S->peak_bytes = std::max(S->peak_bytes, S->resident_bytes);
        R->state = SPH_RT_SRV_RUNNING;
      }
    }
    int k = 0;
    while (rc == SPH_RT_OK && R->done_steps < R->steps && k < S->cfg.steps_per_tick) {
      rc = sph_rt_step(R->handle, R->dt, R->has_Qe ? R->Qe.data() : nullptr,
                       R->has_QE ? R->QE.data() : nullptr, nullptr, nullptr, &R->last);
      if (rc) R->err = sph_rt_last_error(R->handle);
      R->done_steps++;
      R->particle_steps += R->handle ? R->handle->n_int : 0;
      ++k;
    }
    bool finished = rc != SPH_RT_OK || R->done_steps >= R->steps;
    if (finished) {
      finish_request(S, R, rc);
      std::lock_guard<std::mutex> lk(S->mu);
      S->busy--;
    } else {
      std::lock_guard<std::mutex> lk(S->mu);
      S->ready.push_back(R);
      S->busy--;
      S->cv.notify_all();
    }
  }
}

}  // namespace

using namespace sphrt;

extern "C" void sph_rt_srv_default_config(sph_rt_srv_config *c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->workers = 8;
  c->max_resident = 64;
  c->steps_per_tick = 1;
  c->hbm_budget_bytes = 120e9;
  c->device = 0;
  c->fuse_max_n = 20000;
  c->fuse_max_k = 64;
}

extern "C" sph_rt_status sph_rt_srv_create(const sph_rt_srv_config *cfg, sph_rt_srv **out) {
  if (!out || !cfg) return SPH_RT_EINVAL;
  *out = nullptr;
  if (cfg->workers < 1 || cfg->workers > 256 || cfg->max_resident < 1 ||
      cfg->steps_per_tick < 1 || !(cfg->hbm_budget_bytes > 0) || cfg->device < 0 ||
      cfg->fuse_max_n < 0 || cfg->fuse_max_k < 1)
    return SPH_RT_EINVAL;
  sph_rt_srv *S = new (std::nothrow) sph_rt_srv();
  if (!S) return SPH_RT_ENOMEM;
  S->cfg = *cfg;
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return SPH_RT_EDEVICE;
  }
  for (int w = 0; w < cfg->workers; ++w) S->workers.emplace_back(worker_main, S);
  *out = S;
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_srv_submit(sph_rt_srv *S, const sph_rt_config *cfg,
                                           int64_t n_total, const double *pos,
                                           const double *mass, const double *rho,
                                           const double *h, const double *sigma0,
                                           const int32_t *kind, const int64_t *copy_of,
                                           const double *e0, const double *E0, const double *Qe,
                                           const double *QE, int32_t steps, double dt,
                                           int64_t *request_id) {
  if (!S || !cfg || !request_id) return SPH_RT_EINVAL;
  if (n_total < 1 || steps < 1 || !(dt > 0) || !pos || !mass || !rho || !h || !sigma0 || !kind ||
      !e0 || !E0)
    return SPH_RT_EINVAL;
  auto R = std::make_shared<Request>();
  R->cfg = *cfg;
  R->n = n_total;
  R->steps = steps;
  R->dt = dt;
  const int dim = cfg->dim;
  R->pos.assign(pos, pos + n_total * dim);
  R->mass.assign(mass, mass + n_total);
  R->rho.assign(rho, rho + n_total);
  R->h.assign(h, h + n_total);
  R->sigma0.assign(sigma0, sigma0 + n_total);
  R->kind.assign(kind, kind + n_total);
  for (int64_t i = 0; i < n_total; ++i) R->n_int += kind[i] == SPH_RT_INTERIOR;
  R->e0.assign(e0, e0 + n_total);
  R->E0.assign(E0, E0 + n_total);
  if (copy_of) {
    R->copy_of.assign(copy_of, copy_of + n_total);
    R->has_copy = true;
  }
  if (Qe) {
    R->Qe.assign(Qe, Qe + n_total);
    R->has_Qe = true;
  }
  if (QE) {
    R->QE.assign(QE, QE + n_total);
    R->has_QE = true;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  R->id = S->next_id++;
  R->t_submit = now_s();
  if (S->t_first == 0) S->t_first = R->t_submit;
  S->all[R->id] = R;
  S->queued.push_back(R);
  admit_locked(S);
  S->cv.notify_all();
  *request_id = R->id;
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_srv_poll(sph_rt_srv *S, int64_t id, int32_t *state,
                                         double times[3]) {
  if (!S) return SPH_RT_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return SPH_RT_EINVAL;
  if (state) *state = it->second->state;
  if (times) {
    times[0] = it->second->t_submit;
    times[1] = it->second->t_admit;
    times[2] = it->second->t_done;
  }
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_srv_wait(sph_rt_srv *S, int64_t id) {
  if (!S) return SPH_RT_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return SPH_RT_EINVAL;
  auto R = it->second;
  S->cv.wait(lk, [&] { return R->state == SPH_RT_SRV_DONE || R->state == SPH_RT_SRV_FAILED; });
  return R->status;
}

extern "C" sph_rt_status sph_rt_srv_result(sph_rt_srv *S, int64_t id, double *e, double *E,
                                           sph_rt_stats *last_stats, char *msg, int64_t msg_len) {
  if (!S) return SPH_RT_EINVAL;
  std::shared_ptr<Request> R;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return SPH_RT_EINVAL;
    R = it->second;
    if (R->state != SPH_RT_SRV_DONE && R->state != SPH_RT_SRV_FAILED) return SPH_RT_ESTATE;
  }
  if (msg && msg_len > 0) {
    strncpy(msg, R->err.c_str(), (size_t)msg_len - 1);
    msg[msg_len - 1] = 0;
  }
  if (R->state == SPH_RT_SRV_FAILED) return R->status;
  if (e) memcpy(e, R->e.data(), sizeof(double) * R->n);
  if (E) memcpy(E, R->E.data(), sizeof(double) * R->n);
  if (last_stats) *last_stats = R->last;
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_srv_info(sph_rt_srv *S, sph_rt_srv_info_t *info) {
  if (!S || !info) return SPH_RT_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  info->queued = (int32_t)S->queued.size();
  info->resident = S->resident;
  info->peak_resident = S->peak_resident;
  info->resident_bytes = S->resident_bytes;
  info->peak_bytes = S->peak_bytes;
  info->particle_steps = S->total_particle_steps;
  info->t_first_submit = S->t_first;
  info->t_last_done = S->t_last;
  info->fused_requests = S->fused_requests;
  info->fused_batches = S->fused_batches;
  return SPH_RT_OK;
}

extern "C" void sph_rt_srv_destroy(sph_rt_srv *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
    S->queued.clear();
    S->cv.notify_all();
  }
  for (auto &t : S->workers) t.join();
  for (auto &kv : S->all)
    if (kv.second->handle) sph_rt_destroy(kv.second->handle);
  for (sph_rt *h : S->idle) sph_rt_destroy(h);
  delete S;
}
