// sph_rt.cu -- the C ABI of include/sph_rt.h: handle lifecycle, host-side
// validation, and the step driver that follows Alg. 1 of the paper
// (initial material solve, then outer iterations of diffusion solve and
// material solve until Eq. mat-rad-convergence holds).
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace sphrt {

// defined in the other translation units
sph_rt_status build_particles(sph_rt *s, int64_t n, const double *pos_c, const double *mass_c,
                              const double *rho_c, const double *h_c, const double *sig0_c,
                              const int32_t *kind_c, const int64_t *copy_of_c, const double *e0_c,
                              const double *E0_c, int64_t n_int);
sph_rt_status launch_properties(sph_rt *s, double dt);
sph_rt_status launch_assembly(sph_rt *s, double dt, double *gersh_out);
sph_rt_status launch_rhs(sph_rt *s, double dt);
sph_rt_status launch_set_guess(sph_rt *s, int order, const double *w);
sph_rt_status launch_newton(sph_rt *s, double dt, const double *E_new, const double *E_prev,
                            const double *e_start, double *e_out);
sph_rt_status launch_totals(sph_rt *s, const double *e, const double *E);
sph_rt_status launch_check_inputs(sph_rt *s, const double *Qe, const double *QE,
                                  const double *ge, const double *gE);
sph_rt_status launch_balance(sph_rt *s, double dt, const double *E);
sph_rt_status launch_ghost_install(sph_rt *s, const double *ge_c, const double *gE_c);
sph_rt_status launch_copy_sync(sph_rt *s);
sph_rt_status launch_gather_interior(sph_rt *s, const double *in_c, double *out);
sph_rt_status launch_scatter_caller(sph_rt *s, const double *in_s, int64_t count, double *out_c);
sph_rt_status launch_finish(sph_rt *s, const double *e_new, const double *E_new);
sph_rt_status launch_save_before(sph_rt *s);
sph_rt_status launch_dt_control(sph_rt *s, double dt);
sph_rt_status pcg_solve(sph_rt *s, int *iters, bool *converged);
sph_rt_status autotune_fine_shape(sph_rt *s);
sph_rt_status outer_loop(sph_rt *s, double dt);
void outer_loop_account(sph_rt *s, const Scalars &h);
void loop_graph_release(sph_rt *s);
sph_rt_status launch_cheb_slots(sph_rt *s, int first, const double *gersh_dev,
                                const std::vector<int> &mode, const std::vector<int> &degree);
sph_rt_status amg_setup(sph_rt *s);
void amg_release(sph_rt *s);
sph_rt_status validate_device_particles(sph_rt *s, int64_t n, const double *pos,
                                        const double *mass, const double *rho, const double *h,
                                        const double *sigma0, const int32_t *kind,
                                        const int64_t *copy_of, const double *e0,
                                        const double *E0, int64_t *n_int_out);

bool trace_enabled() {
  static const bool on = [] {
    const char *v = getenv("SPH_RT_TRACE");
    return v && v[0] == '1';
  }();
  return on;
}

sph_rt_status set_error(sph_rt *s, sph_rt_status st, const std::string &msg) {
  if (s) s->err = msg;
  return st;
}

bool cuda_ok(sph_rt *s, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return true;
  if (s) s->err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  return false;
}

// Device memory of a particle set comes from a per-handle caching allocator:
// buffers released by free_all() go to a size-keyed free list and are handed
// out again (best fit, at most twice the request) by the next particle set, so
// re-setting particles of similar size does no cudaFree/cudaMalloc (both of
// which synchronise the device).  A destroyed handle gives its buffers to a
// library-wide cache per device (up to kCacheBytes; beyond that they go back
// to CUDA), from which new handles take before calling cudaMalloc: a batch's
// staging handles and the serving loop's fused batches, created and destroyed
// again and again, then neither allocate nor synchronise the device.  A
// handle hands buffers on only after its stream has finished with them.  When
// an allocation fails, the handle's free list and the cache go back to CUDA
// and the request is retried once.
constexpr size_t kCacheBytes = size_t(8) << 30;
constexpr int kCacheDevices = 64;
struct DeviceCache {
  std::mutex mu;
  std::multimap<size_t, void *> free[kCacheDevices];
  size_t bytes[kCacheDevices] = {};
};
static DeviceCache &device_cache() {
  static DeviceCache *c = new DeviceCache();  // lives as long as the process
  return *c;
}
static bool cache_take(int dev, size_t bytes, void **p, size_t *got) {
  if (dev < 0 || dev >= kCacheDevices) return false;
  DeviceCache &c = device_cache();
  std::lock_guard<std::mutex> lk(c.mu);
  auto it = c.free[dev].lower_bound(bytes);
  if (it == c.free[dev].end() || it->first > 2 * bytes) return false;
  *p = it->second;
  *got = it->first;
  c.bytes[dev] -= it->first;
  c.free[dev].erase(it);
  return true;
}
static void cache_give(int dev, void *p, size_t bytes) {
  if (dev >= 0 && dev < kCacheDevices) {
    DeviceCache &c = device_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.bytes[dev] + bytes <= kCacheBytes) {
      c.free[dev].emplace(bytes, p);
      c.bytes[dev] += bytes;
      return;
    }
  }
  cudaFree(p);
}
static void cache_trim(int dev) {
  if (dev < 0 || dev >= kCacheDevices) return;
  DeviceCache &c = device_cache();
  std::lock_guard<std::mutex> lk(c.mu);
  for (auto &kv : c.free[dev]) cudaFree(kv.second);
  c.free[dev].clear();
  c.bytes[dev] = 0;
}

// the handle's free list to the library cache (its stream is idle)
static void pool_release(sph_rt *s) {
  for (auto &kv : s->pool) cache_give(s->cfg.device, kv.second, kv.first);
  s->pool.clear();
}

void *dalloc_bytes(sph_rt *s, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  auto it = s->pool.lower_bound(bytes);
  if (it != s->pool.end() && it->first <= 2 * bytes) {
    void *p = it->second;
    s->alloc_size[p] = it->first;
    s->pool.erase(it);
    s->allocs.push_back(p);
    return p;
  }
  void *p = nullptr;
  size_t got = 0;
  if (cache_take(s->cfg.device, bytes, &p, &got)) {
    s->alloc_size[p] = got;
    s->allocs.push_back(p);
    return p;
  }
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (s->cuda_ready) cudaStreamSynchronize(s->stream);
    pool_release(s);
    cache_trim(s->cfg.device);
    e = cudaMalloc(&p, bytes);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    s->err = "device allocation of " + std::to_string(bytes) + " bytes failed: " +
             cudaGetErrorString(e);
    return nullptr;
  }
  s->alloc_size[p] = bytes;
  s->allocs.push_back(p);
  return p;
}

void free_all(sph_rt *s) {
  if (s->gate_host) *s->gate_host = s->gate_epoch;  // release a held timing gate
  if (s->cuda_ready) cudaStreamSynchronize(s->stream);
  loop_graph_release(s);  // its launches refer to the buffers released below
  amg_release(s);
  for (void *p : s->allocs) s->pool.emplace(s->alloc_size[p], p);
  s->allocs.clear();
  s->alloc_size.clear();
  s->have_particles = false;
  s->have_operator = false;
  s->amg_ready = false;
  s->gcol = nullptr;
  s->gvx = s->gvy = s->gvz = nullptr;
  s->mat_val32 = nullptr;
  s->diag32 = s->invdiag32 = nullptr;
  s->amg_gersh = nullptr;
  s->cheb_slots = nullptr;
  s->ev_flags = nullptr;
  s->ev_used = 0;
}

// Return one buffer of the current particle set to the free list.
void dfree(sph_rt *s, void *p) {
  if (!p) return;
  auto it = std::find(s->allocs.begin(), s->allocs.end(), p);
  if (it == s->allocs.end()) return;
  s->allocs.erase(it);
  s->pool.emplace(s->alloc_size[p], p);
  s->alloc_size.erase(p);
}

void free_everything(sph_rt *s) {
  free_all(s);
  pool_release(s);
}

}  // namespace sphrt

using namespace sphrt;

// ---------------------------------------------------------------------------
// configuration
// ---------------------------------------------------------------------------
extern "C" void sph_rt_default_config(sph_rt_config *c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->dim = 3;
  c->kernel = SPH_RT_M4_SPLINE;
  c->a = 1.0;
  c->c = 1.0;
  c->cv = 1.0;
  c->limiter = SPH_RT_LIMITER_NONE;
  c->larsen_k = 2.0;
  c->opacity_exp = 0.0;
  c->T_floor = 0.0;
  c->tol_outer_e = 1e-8;
  c->tol_outer_E = 1e-8;
  c->tol_inner_e = 1e-13;
  c->tol_krylov = 1e-12;
  c->max_outer = 50;
  c->max_inner_e = 50;
  c->max_krylov = 2000;
  c->precond = SPH_RT_PRECOND_AMG;
  c->precision = SPH_RT_FP64;
  c->cheb_degree = 1;
  c->amg_rebuild = 0;
  c->amg_theta = 0.02;
  c->check_every = 8;
  c->kernel_timing = 0;
  c->autotune = 0;
  c->amg_tail = 0;
  c->coarse_fp32 = 1;
  c->graphs = 1;
  c->pdl = 1;
  c->fine_post_smooth = 1;
  c->reliable_drop = 1e-4;
  c->dt_target = 0.0;
  c->dt_growth = 10.0;
  c->dt_min = 0.0;
  c->dt_max = 1e300;
  c->dt_eta_floor = 1e-15;
  c->cell_list = SPH_RT_CELLS_AUTO;
  c->index64 = 0;
  c->krylov_start = 3;
  c->device = 0;
  c->stream = nullptr;
}

static bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

static sph_rt_status check_config(const sph_rt_config *c, std::string &why) {
  if (c->dim < 1 || c->dim > 3) return why = "dim must be 1, 2 or 3", SPH_RT_EINVAL;
  if (c->kernel != SPH_RT_M4_SPLINE && c->kernel != SPH_RT_WENDLAND_C4)
    return why = "kernel must be SPH_RT_M4_SPLINE or SPH_RT_WENDLAND_C4", SPH_RT_EINVAL;
  if (!(isfinite(c->a) && c->a >= 0.0) || !finite_pos(c->c) || !finite_pos(c->cv))
    return why = "a must be finite and >= 0 (0: no emission); c and cv finite and positive",
           SPH_RT_EINVAL;
  if (c->limiter < 0 || c->limiter > 2) return why = "limiter out of range", SPH_RT_EINVAL;
  if (c->limiter == SPH_RT_LIMITER_LARSEN && !finite_pos(c->larsen_k))
    return why = "larsen_k must be positive", SPH_RT_EINVAL;
  if (!isfinite(c->opacity_exp)) return why = "opacity_exp must be finite", SPH_RT_EINVAL;
  if (!isfinite(c->T_floor) || c->T_floor < 0) return why = "T_floor must be >= 0", SPH_RT_EINVAL;
  if (!(isfinite(c->sigma_s) && c->sigma_s >= 0.0))
    return why = "sigma_s must be finite and >= 0", SPH_RT_EINVAL;
  if (!finite_pos(c->tol_outer_e) || !finite_pos(c->tol_outer_E) || !finite_pos(c->tol_inner_e) ||
      !finite_pos(c->tol_krylov))
    return why = "tolerances must be finite and positive", SPH_RT_EINVAL;
  if (c->max_outer < 1 || c->max_outer > 100000 || c->max_inner_e < 1 || c->max_krylov < 1)
    return why = "iteration limits must be >= 1 (max_outer <= 100000)", SPH_RT_EINVAL;
  if (c->precond < 0 || c->precond > 2) return why = "precond out of range", SPH_RT_EINVAL;
  if (c->precision < 0 || c->precision > 1) return why = "precision out of range", SPH_RT_EINVAL;
  if (c->cheb_degree < 1 || c->cheb_degree > 16)
    return why = "cheb_degree must be in [1, 16]", SPH_RT_EINVAL;
  if (!(c->amg_theta >= 0.0 && c->amg_theta < 1.0))
    return why = "amg_theta must be in [0, 1)", SPH_RT_EINVAL;
  if (c->check_every < 1) return why = "check_every must be >= 1", SPH_RT_EINVAL;
  if (c->graphs < 0 || c->graphs > 1) return why = "graphs must be 0 or 1", SPH_RT_EINVAL;
  if (c->pdl < 0 || c->pdl > 1) return why = "pdl must be 0 or 1", SPH_RT_EINVAL;
  if (c->amg_tail < 0 || c->amg_tail > 1) return why = "amg_tail must be 0 or 1", SPH_RT_EINVAL;
  if (c->coarse_fp32 < 0 || c->coarse_fp32 > 1)
    return why = "coarse_fp32 must be 0 or 1", SPH_RT_EINVAL;
  if (c->fine_post_smooth < 0 || c->fine_post_smooth > 1)
    return why = "fine_post_smooth must be 0 or 1", SPH_RT_EINVAL;
  if (c->fine_post_smooth == 0 && c->cheb_degree != 1)
    return why = "fine_post_smooth = 0 needs cheb_degree = 1", SPH_RT_EINVAL;
  if (!(c->reliable_drop > 0.0 && c->reliable_drop < 1.0))
    return why = "reliable_drop must be in (0, 1)", SPH_RT_EINVAL;
  if (!(c->dt_target >= 0.0 && c->dt_target < 1e300))
    return why = "dt_target must be >= 0 (0 = no time step choice)", SPH_RT_EINVAL;
  if (!(c->dt_growth >= 1.0 && c->dt_growth < 1e300) || !(c->dt_min >= 0.0) ||
      !(c->dt_max > 0.0) || !(c->dt_min <= c->dt_max) || !(c->dt_eta_floor >= 0.0 &&
      c->dt_eta_floor < 1e300))
    return why = "time step limits: dt_growth >= 1, 0 <= dt_min <= dt_max, dt_eta_floor >= 0",
           SPH_RT_EINVAL;
  if (c->cell_list < SPH_RT_CELLS_AUTO || c->cell_list > SPH_RT_CELLS_SORTED)
    return why = "cell_list must be SPH_RT_CELLS_AUTO, _DENSE or _SORTED", SPH_RT_EINVAL;
  if (c->index64 < 0 || c->index64 > 1) return why = "index64 must be 0 or 1", SPH_RT_EINVAL;
  if (c->krylov_start < 0 || c->krylov_start > 3)
    return why = "krylov_start must be 0 .. 3", SPH_RT_EINVAL;
  if (c->autotune < 0 || c->autotune > 2) return why = "autotune must be 0, 1 or 2", SPH_RT_EINVAL;
  if (c->device < 0) return why = "device must be >= 0", SPH_RT_EINVAL;
  return SPH_RT_OK;
}

static thread_local std::string g_create_error;  // why the last handle-less call failed

namespace sphrt {
void set_thread_error(const std::string &msg) { g_create_error = msg; }
}  // namespace sphrt

extern "C" sph_rt_status sph_rt_create(const sph_rt_config *cfg, sph_rt **out) {
  if (!out) return SPH_RT_EINVAL;
  *out = nullptr;
  if (!cfg) {
    g_create_error = "cfg is NULL";
    return SPH_RT_EINVAL;
  }
  std::string why;
  if (check_config(cfg, why) != SPH_RT_OK) {
    g_create_error = why;
    return SPH_RT_EINVAL;
  }
  sph_rt *s = new (std::nothrow) sph_rt();
  if (!s) {
    g_create_error = "out of host memory";
    return SPH_RT_ENOMEM;
  }
  s->cfg = *cfg;
  s->dim = cfg->dim;
  *out = s;
  return SPH_RT_OK;
}

sph_rt_status ensure_cuda(sph_rt *s) {
  if (s->cuda_ready) return SPH_RT_OK;
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  int sms = 0;
  SPH_CUDA(s, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->cfg.device));
  s->num_sms = sms > 0 ? sms : 152;
  if (s->cfg.stream) {
    s->stream = (cudaStream_t)s->cfg.stream;
    s->own_stream = false;
  } else {
    SPH_CUDA(s, cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
  }
  SPH_CUDA(s, cudaMallocHost(&s->sc_host, sizeof(Scalars)));
  s->cuda_ready = true;
  return SPH_RT_OK;
}

extern "C" void sph_rt_destroy(sph_rt *s) {
  if (!s) return;
  if (s->cuda_ready) {
    cudaSetDevice(s->cfg.device);
    free_everything(s);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->gate_host) cudaFreeHost((void *)s->gate_host);
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    if (s->sc_host) cudaFreeHost(s->sc_host);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  }
  delete s;
}

extern "C" sph_rt_status sph_rt_release_cached_memory(int32_t device) {
  if (device < 0) return SPH_RT_EINVAL;
  cache_trim(device);
  return SPH_RT_OK;
}

extern "C" const char *sph_rt_last_error(const sph_rt *s) {
  return s ? s->err.c_str() : g_create_error.c_str();
}

extern "C" int64_t sph_rt_launch_count(const sph_rt *s) { return s ? s->launches : 0; }

extern "C" sph_rt_status sph_rt_get_config(const sph_rt *s, sph_rt_config *cfg) {
  if (!s || !cfg) return SPH_RT_EINVAL;
  *cfg = s->cfg;
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_get_solver_tuning(const sph_rt *s, sph_rt_tune_trial *trials,
                                                  int32_t cap, int32_t *count) {
  if (!s || !count || cap < 0) return SPH_RT_EINVAL;
  *count = (int32_t)s->tune_trials.size();
  for (int32_t k = 0; trials && k < cap && k < *count; ++k) trials[k] = s->tune_trials[k];
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_loop_graph_info(const sph_rt *s, int64_t *captures,
                                                int64_t *launches) {
  if (!s) return SPH_RT_EINVAL;
  if (captures) *captures = s->graph_builds;
  if (launches) *launches = s->graph_launches;
  return SPH_RT_OK;
}

// ---------------------------------------------------------------------------
// particles
// ---------------------------------------------------------------------------
static sph_rt_status validate_host_particles(sph_rt *s, int64_t n, const double *pos,
                                             const double *mass, const double *rho,
                                             const double *h, const double *sigma0,
                                             const int32_t *kind, const int64_t *copy_of,
                                             const double *e0, const double *E0,
                                             int64_t *n_int) {
  if (n < 1) return set_error(s, SPH_RT_EINVAL, "n_total must be >= 1");
  if (n >= ((int64_t)1 << 31) - 1) return set_error(s, SPH_RT_EINVAL, "n_total must be < 2^31");
  if (!pos || !mass || !rho || !h || !sigma0 || !kind || !e0 || !E0)
    return set_error(s, SPH_RT_EINVAL, "a required particle array is NULL");
  int64_t ni = 0;
  for (int64_t i = 0; i < n; ++i) {
    for (int d = 0; d < s->dim; ++d)
      if (!isfinite(pos[i * s->dim + d]))
        return set_error(s, SPH_RT_EINVAL, "non-finite position at particle " + std::to_string(i));
    if (!finite_pos(mass[i]) || !finite_pos(rho[i]) || !finite_pos(h[i]))
      return set_error(s, SPH_RT_EINVAL,
                       "mass, rho and h must be finite and positive (particle " +
                           std::to_string(i) + ")");
    if (!isfinite(sigma0[i]) || sigma0[i] < 0)
      return set_error(s, SPH_RT_EINVAL, "sigma0 must be finite and >= 0 (particle " +
                                             std::to_string(i) + ")");
    if (!isfinite(e0[i]) || !isfinite(E0[i]))
      return set_error(s, SPH_RT_EINVAL, "non-finite initial energy at particle " +
                                             std::to_string(i));
    if (kind[i] < 0 || kind[i] > 2)
      return set_error(s, SPH_RT_EINVAL, "kind out of range at particle " + std::to_string(i));
    if (kind[i] == SPH_RT_INTERIOR) ++ni;
    if (kind[i] == SPH_RT_COPY) {
      if (!copy_of) return set_error(s, SPH_RT_EINVAL, "copy ghosts need copy_of");
      int64_t c = copy_of[i];
      if (c < 0 || c >= n || kind[c] != SPH_RT_INTERIOR)
        return set_error(s, SPH_RT_EINVAL,
                         "copy_of must name an interior particle (particle " + std::to_string(i) +
                             ")");
    }
  }
  if (ni == 0) return set_error(s, SPH_RT_EINVAL, "no interior particle");
  *n_int = ni;
  return SPH_RT_OK;
}

static sph_rt_status alloc_step_vectors(sph_rt *s) {
  int64_t n = s->n, ni = s->n_int;
  double **full[] = {&s->T, &s->sigma, &s->f, &s->R, &s->lambda, &s->D, &s->tmp_n, &s->tmp_n2,
                     &s->tmp_n3, &s->e_bak, &s->E_bak, &s->stage_ge, &s->stage_gE};
  for (double **p : full)
    if (!(*p = dalloc<double>(s, n))) return SPH_RT_ENOMEM;
  double **inner[] = {&s->e_old, &s->E_old, &s->e_l, &s->E_l, &s->e_new, &s->Qe, &s->QE, &s->b,
                      &s->x, &s->r, &s->z, &s->p, &s->q, &s->w, &s->diag, &s->invdiag, &s->gb,
                      &s->z_old, &s->E_hist[0], &s->E_hist[1], &s->E_hist[2]};
  for (double **p : inner)
    if (!(*p = dalloc<double>(s, ni))) return SPH_RT_ENOMEM;
  if (!(s->gersh = dalloc<double>(s, 1))) return SPH_RT_ENOMEM;
  if (s->cfg.precision == SPH_RT_MIXED) {
    s->mat_val32 = dalloc<float>(s, s->nnz_mat);
    s->diag32 = dalloc<float>(s, ni);
    s->invdiag32 = dalloc<float>(s, ni);
    if (!s->mat_val32 || !s->diag32 || !s->invdiag32) return SPH_RT_ENOMEM;
  }
  if (!(s->cheb_slots = dalloc<ChebCoef>(s, kChebSlots))) return SPH_RT_ENOMEM;
  SPH_CUDA(s, cudaMemsetAsync(s->Qe, 0, sizeof(double) * ni, s->stream));
  SPH_CUDA(s, cudaMemsetAsync(s->QE, 0, sizeof(double) * ni, s->stream));
  return SPH_RT_OK;
}

static sph_rt_status set_particles_common(sph_rt *s, int64_t n, const double *pos,
                                          const double *mass, const double *rho, const double *h,
                                          const double *sigma0, const int32_t *kind,
                                          const int64_t *copy_of, const double *e0,
                                          const double *E0, bool device) {
  if (!s) return SPH_RT_EINVAL;
  int64_t n_int = 0;
  sph_rt_status rc;
  if (!device) {
    rc = validate_host_particles(s, n, pos, mass, rho, h, sigma0, kind, copy_of, e0, E0, &n_int);
    if (rc) return rc;
  }
  if ((rc = ensure_cuda(s))) return rc;
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  if (device) {
    if (n < 1 || n >= ((int64_t)1 << 31) - 1)
      return set_error(s, SPH_RT_EINVAL, "n_total must be in [1, 2^31)");
    if (!pos || !mass || !rho || !h || !sigma0 || !kind || !e0 || !E0)
      return set_error(s, SPH_RT_EINVAL, "a required particle array is NULL");
    rc = validate_device_particles(s, n, pos, mass, rho, h, sigma0, kind, copy_of, e0, E0, &n_int);
    if (rc) return rc;
  }
  free_all(s);
  s->err.clear();
  const double *dpos = pos, *dm = mass, *dr = rho, *dh = h, *ds = sigma0, *de = e0, *dE = E0;
  const int32_t *dk = kind;
  const int64_t *dc = copy_of;
  if (!device) {
    // upload caller-order arrays into temporaries
    double *b_pos = dalloc<double>(s, (size_t)n * s->dim);
    double *b7 = dalloc<double>(s, (size_t)n * 6);
    int32_t *b_kind = dalloc<int32_t>(s, n);
    int64_t *b_copy = copy_of ? dalloc<int64_t>(s, n) : nullptr;
    if (!b_pos || !b7 || !b_kind || (copy_of && !b_copy)) return SPH_RT_ENOMEM;
    SPH_CUDA(s, cudaMemcpyAsync(b_pos, pos, sizeof(double) * n * s->dim, cudaMemcpyHostToDevice, s->stream));
    const double *src[6] = {mass, rho, h, sigma0, e0, E0};
    for (int k = 0; k < 6; ++k)
      SPH_CUDA(s, cudaMemcpyAsync(b7 + (size_t)k * n, src[k], sizeof(double) * n,
                                  cudaMemcpyHostToDevice, s->stream));
    SPH_CUDA(s, cudaMemcpyAsync(b_kind, kind, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s->stream));
    if (copy_of)
      SPH_CUDA(s, cudaMemcpyAsync(b_copy, copy_of, sizeof(int64_t) * n, cudaMemcpyHostToDevice, s->stream));
    dpos = b_pos;
    dm = b7;
    dr = b7 + n;
    dh = b7 + 2 * n;
    ds = b7 + 3 * n;
    de = b7 + 4 * n;
    dE = b7 + 5 * n;
    dk = b_kind;
    dc = b_copy;
  }
  SPH_TRACE("set_particles: n=%lld n_int=%lld", (long long)n, (long long)n_int);
  rc = build_particles(s, n, dpos, dm, dr, dh, ds, dk, dc, de, dE, n_int);
  SPH_TRACE("set_particles: built, nnz_nbr=%lld nnz_mat=%lld rc=%d", (long long)s->nnz_nbr,
            (long long)s->nnz_mat, (int)rc);
  if (rc) {
    free_all(s);
    return rc;
  }
  if ((rc = alloc_step_vectors(s))) {
    free_all(s);
    return rc;
  }
  SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  s->have_particles = true;
  s->have_operator = false;
  s->amg_ready = false;
  s->hist = 0;  // no previous step of this particle set (slot order) yet
  // the tuned loads in flight (they never change a result bit) carry over to
  // a particle set within 25 % of the tuned one's rows and entries and with the
  // same lanes per row; otherwise the first step tunes them again
  if (s->fine_shape_set) {
    auto near = [](int64_t a, int64_t b) { return 4 * (a > b ? a - b : b - a) <= (a > b ? a : b); };
    const int W = lanes_for_mean(s->n_int ? (double)s->nnz_mat / (double)s->n_int : 0.0);
    if (!near(s->n_int, s->fine_shape_n) || !near(s->nnz_mat, s->fine_shape_nnz) ||
        W != s->fine_shape.W)
      s->fine_shape_set = false;
  }
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_set_particles(sph_rt *s, int64_t n_total, const double *pos,
                                              const double *mass, const double *rho,
                                              const double *h, const double *sigma0,
                                              const int32_t *kind, const int64_t *copy_of,
                                              const double *e0, const double *E0) {
  return set_particles_common(s, n_total, pos, mass, rho, h, sigma0, kind, copy_of, e0, E0, false);
}

extern "C" sph_rt_status sph_rt_set_particles_device(sph_rt *s, int64_t n_total,
                                                     const double *pos, const double *mass,
                                                     const double *rho, const double *h,
                                                     const double *sigma0, const int32_t *kind,
                                                     const int64_t *copy_of, const double *e0,
                                                     const double *E0) {
  return set_particles_common(s, n_total, pos, mass, rho, h, sigma0, kind, copy_of, e0, E0, true);
}

// ---------------------------------------------------------------------------
// smoothing lengths (Sec. 3.1) and moving particles
// ---------------------------------------------------------------------------
namespace sphrt {
sph_rt_status smoothing_iterate(sph_rt *s, double eta, double tol, int max_iter, int *iters);
}

// caller-order device copies of the current particle set: positions (unless
// the caller gives new ones), kinds and copy sources
__global__ void caller_layout_kernel(int64_t n, int dim, const int64_t *slot2caller,
                                     const double *px, const double *py, const double *pz,
                                     const int32_t *kind, const int32_t *copysrc,
                                     double *pos_c, int32_t *kind_c, int64_t *copy_c) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = slot2caller[t];
    if (pos_c) {
      pos_c[c * dim] = px[t];
      if (dim > 1) pos_c[c * dim + 1] = py[t];
      if (dim > 2) pos_c[c * dim + 2] = pz[t];
    }
    kind_c[c] = kind[t];
    copy_c[c] = copysrc[t] >= 0 ? slot2caller[copysrc[t]] : -1;
  }
}

// Rebuild the particle set (Morton order, neighbour lists, operator sparsity;
// the AMG hierarchy follows on the next step) from its own device data in
// caller order, with new positions (device, caller order) or the current ones,
// keeping masses, densities, smoothing lengths (s->h), opacities, kinds and
// the state e, E.
static sph_rt_status rebuild_particles(sph_rt *s, const double *new_pos) {
  const int64_t n = s->n;
  const int dim = s->dim;
  double *pos_c = nullptr, *arr = nullptr;
  int32_t *kind_c = nullptr;
  int64_t *copy_c = nullptr;
  sph_rt_status rc = SPH_RT_OK;
  if (cudaMalloc(&pos_c, sizeof(double) * n * dim) != cudaSuccess ||
      cudaMalloc(&arr, sizeof(double) * n * 6) != cudaSuccess ||
      cudaMalloc(&kind_c, sizeof(int32_t) * n) != cudaSuccess ||
      cudaMalloc(&copy_c, sizeof(int64_t) * n) != cudaSuccess) {
    cudaGetLastError();
    rc = set_error(s, SPH_RT_ENOMEM, "no device memory for the particle rebuild");
  }
  if (!rc) {
    const int g = (int)((n + kBlock - 1) / kBlock < (int64_t)s->num_sms * 8
                            ? (n + kBlock - 1) / kBlock
                            : (int64_t)s->num_sms * 8);
    caller_layout_kernel<<<g, kBlock, 0, s->stream>>>(n, dim, s->slot2caller, s->px, s->py, s->pz,
                                                      s->kind, s->copysrc,
                                                      new_pos ? nullptr : pos_c, kind_c, copy_c);
    s->launches++;
    const double *src[6] = {s->mass, s->rho, s->h, s->sigma0, s->e, s->E};
    for (int k = 0; k < 6 && !rc; ++k) rc = launch_scatter_caller(s, src[k], n, arr + (size_t)k * n);
    if (!rc && new_pos &&
        cudaMemcpyAsync(pos_c, new_pos, sizeof(double) * n * dim, cudaMemcpyDeviceToDevice,
                        s->stream) != cudaSuccess)
      rc = set_error(s, SPH_RT_EDEVICE, "copying the new positions failed");
    if (!rc && (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s->stream) != cudaSuccess))
      rc = set_error(s, SPH_RT_EDEVICE, "gathering the particle set failed");
  }
  if (!rc)
    rc = set_particles_common(s, n, pos_c, arr, arr + n, arr + 2 * n, arr + 3 * n, kind_c, copy_c,
                              arr + 4 * n, arr + 5 * n, true);
  cudaFree(pos_c);
  cudaFree(arr);
  cudaFree(kind_c);
  cudaFree(copy_c);
  return rc;
}

extern "C" sph_rt_status sph_rt_adapt_smoothing_lengths(sph_rt *s, double eta, double tol,
                                                        int32_t max_iter, int32_t *iters) {
  if (!s) return SPH_RT_EINVAL;
  if (!s->have_particles) return set_error(s, SPH_RT_ESTATE, "no particles");
  if (!(isfinite(eta) && eta > 0.0) || !(isfinite(tol) && tol > 0.0) || max_iter < 1)
    return set_error(s, SPH_RT_EINVAL, "eta and tol must be positive, max_iter >= 1");
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  int it = 0;
  sph_rt_status rc = smoothing_iterate(s, eta, tol, max_iter, &it);
  if (rc) return rc;
  if (iters) *iters = it;
  return rebuild_particles(s, nullptr);
}

extern "C" sph_rt_status sph_rt_get_smoothing_lengths(sph_rt *s, double *h) {
  if (!s || !h) return SPH_RT_EINVAL;
  if (!s->have_particles) return set_error(s, SPH_RT_ESTATE, "no particles");
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  sph_rt_status rc = launch_scatter_caller(s, s->h, s->n, s->tmp_n);
  if (rc) return rc;
  SPH_CUDA(s, cudaMemcpyAsync(h, s->tmp_n, sizeof(double) * s->n, cudaMemcpyDeviceToHost, s->stream));
  SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_move_particles_device(sph_rt *s, const double *pos) {
  if (!s || !pos) return SPH_RT_EINVAL;
  if (!s->have_particles) return set_error(s, SPH_RT_ESTATE, "no particles");
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  return rebuild_particles(s, pos);
}

extern "C" sph_rt_status sph_rt_move_particles(sph_rt *s, const double *pos) {
  if (!s || !pos) return SPH_RT_EINVAL;
  if (!s->have_particles) return set_error(s, SPH_RT_ESTATE, "no particles");
  const int64_t count = s->n * s->dim;
  for (int64_t k = 0; k < count; ++k)
    if (!isfinite(pos[k]))
      return set_error(s, SPH_RT_EINVAL, "non-finite position at particle " +
                                             std::to_string(k / s->dim));
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  double *d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * count) != cudaSuccess) {
    cudaGetLastError();
    return set_error(s, SPH_RT_ENOMEM, "no device memory for the new positions");
  }
  sph_rt_status rc = SPH_RT_OK;
  if (cudaMemcpyAsync(d, pos, sizeof(double) * count, cudaMemcpyHostToDevice, s->stream) !=
      cudaSuccess)
    rc = set_error(s, SPH_RT_EDEVICE, "copying the new positions failed");
  if (!rc) rc = rebuild_particles(s, d);
  cudaStreamSynchronize(s->stream);
  cudaFree(d);
  return rc;
}

extern "C" sph_rt_status sph_rt_get_sizes(const sph_rt *s, int64_t *n_interior,
                                          int64_t *nnz_neighbors, int64_t *nnz_operator) {
  if (!s) return SPH_RT_EINVAL;
  if (!s->have_particles) return SPH_RT_ESTATE;
  if (n_interior) *n_interior = s->n_int;
  if (nnz_neighbors) *nnz_neighbors = s->nnz_nbr;
  if (nnz_operator) *nnz_operator = s->nnz_mat;
  return SPH_RT_OK;
}

// ---------------------------------------------------------------------------
// step
// ---------------------------------------------------------------------------
struct PhaseTimer {
  sph_rt *s;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
  void begin(int phase) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s->stream);
    ev.push_back({phase, {a, b}});
  }
  void end() { cudaEventRecord(ev.back().second.second, s->stream); }
  void collect(double *ms5) {
    for (auto &p : ev) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p.second.first, p.second.second) == cudaSuccess)
        ms5[p.first] += t;
      cudaEventDestroy(p.second.first);
      cudaEventDestroy(p.second.second);
    }
    ev.clear();
  }
  ~PhaseTimer() {
    for (auto &p : ev) {
      cudaEventDestroy(p.second.first);
      cudaEventDestroy(p.second.second);
    }
  }
};

static sph_rt_status read_scalars(sph_rt *s) {
  SPH_CUDA(s, cudaMemcpyAsync(s->sc_host, s->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s->stream));
  SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  return SPH_RT_OK;
}

static sph_rt_status tune_then_step(sph_rt *s, double dt, const double *Qe_c,
                                    const double *QE_c, const double *ge_c, const double *gE_c,
                                    sph_rt_stats *stats);

static sph_rt_status step_common(sph_rt *s, double dt, const double *Qe_c, const double *QE_c,
                                 const double *ge_c, const double *gE_c, sph_rt_stats *stats) {
  sph_rt_status rc;
  if (s->cfg.autotune == 1 && !s->solver_tuned)
    return tune_then_step(s, dt, Qe_c, QE_c, ge_c, gE_c, stats);
  PhaseTimer tm{s, {}};
  double ms[5] = {0, 0, 0, 0, 0};  // setup, assembly, amg, krylov, newton
  sph_rt_stats st;
  memset(&st, 0, sizeof st);
  const int64_t ni = s->n_int;
  const size_t nb = sizeof(double) * ni;

  SPH_TRACE("step: begin n=%lld n_int=%lld nnz=%lld dt=%g", (long long)s->n, (long long)s->n_int,
            (long long)s->nnz_mat, dt);
  // input check and energy before the step.  They are read with the step's
  // results at the end (one host round trip per step); a step that will build
  // the AMG structure reads them first, so that the kept hierarchy never comes
  // from a rejected input.
  if ((rc = launch_check_inputs(s, Qe_c, QE_c, ge_c, gE_c))) return rc;
  if ((rc = launch_totals(s, s->e, s->E))) return rc;
  if ((rc = launch_save_before(s))) return rc;
  if (s->cfg.precond == SPH_RT_PRECOND_AMG && (!s->amg_ready || s->cfg.amg_rebuild)) {
    if ((rc = read_scalars(s))) return rc;
    if (s->sc_host->bad_input)
      return set_error(s, SPH_RT_EINVAL, "non-finite source or ghost value");
  }

  tm.begin(0);
  // snapshot of the state (restored if the step does not converge)
  SPH_CUDA(s, cudaMemcpyAsync(s->e_bak, s->e, sizeof(double) * s->n, cudaMemcpyDeviceToDevice, s->stream));
  SPH_CUDA(s, cudaMemcpyAsync(s->E_bak, s->E, sizeof(double) * s->n, cudaMemcpyDeviceToDevice, s->stream));
  // sources (interior, slot order)
  if ((rc = launch_gather_interior(s, Qe_c, s->Qe))) return rc;
  if ((rc = launch_gather_interior(s, QE_c, s->QE))) return rc;
  // material data from the state at the start of the step (a3)
  if ((rc = launch_properties(s, dt))) return rc;
  // Dirichlet ghost values at t^n
  if ((rc = launch_ghost_install(s, ge_c, gE_c))) return rc;
  tm.end();

  SPH_TRACE("step: properties and ghosts queued");
  tm.begin(1);
  if ((rc = launch_assembly(s, dt, s->gersh))) return rc;  // a4
  tm.end();
  s->have_operator = true;
  if (s->cfg.precond == SPH_RT_PRECOND_CHEBYSHEV) {
    // coefficients on [1 - g, 1 + g] straight from the device Gershgorin bound
    if ((rc = launch_cheb_slots(s, 0, s->gersh, {0}, {s->cfg.cheb_degree}))) return rc;
  }
  if (s->cfg.autotune && !s->fine_shape_set) {
    if ((rc = autotune_fine_shape(s))) return rc;
  }

  if (s->cfg.precond == SPH_RT_PRECOND_AMG) {  // a5
    tm.begin(2);
    if ((rc = amg_setup(s))) return rc;
    tm.end();
  }

  SPH_TRACE("step: preconditioner ready (levels %d)", (int)s->levels.size());
  // Alg. 1: e^{n,0} = e^{n-1}, E^{n,0} = E^{n-1}; material solve with E^{n,0}
  // krylov_start = p: the first solve starts from the extrapolation in time of
  // order min(p, converged steps behind) through E^{n-1}, ..., E^{n-1-p}.  The
  // history moves down one place: E_hist[j] <- E_hist[j-1], E_hist[0] <- E_old
  // (E^{n-2}, the last step's start, before E_old is overwritten).
  const int K = s->cfg.krylov_start;
  const int order = std::min(K, s->hist);
  if (K >= 1) {
    for (int j = K - 1; j >= 1; --j)
      SPH_CUDA(s, cudaMemcpyAsync(s->E_hist[j], s->E_hist[j - 1], nb, cudaMemcpyDeviceToDevice,
                                  s->stream));
    SPH_CUDA(s, cudaMemcpyAsync(s->E_hist[0], s->E_old, nb, cudaMemcpyDeviceToDevice, s->stream));
  }
  double gw[4] = {1.0, 0.0, 0.0, 0.0};
  if (order >= 1) extrap_weights(order, dt, s->dt_hist, gw);
  if ((rc = launch_set_guess(s, order, gw))) return rc;
  const int hist0 = s->hist;
  s->hist = 0;  // until this step has converged
  SPH_CUDA(s, cudaMemcpyAsync(s->e_old, s->e, nb, cudaMemcpyDeviceToDevice, s->stream));
  SPH_CUDA(s, cudaMemcpyAsync(s->E_old, s->E, nb, cudaMemcpyDeviceToDevice, s->stream));
  SPH_CUDA(s, cudaMemcpyAsync(s->E_l, s->E, nb, cudaMemcpyDeviceToDevice, s->stream));
  tm.begin(4);
  if ((rc = launch_newton(s, dt, s->E_l, s->E_l, s->e_old, s->e_l))) return rc;  // a8
  tm.end();

  // Alg. 1 outer loop: rhs (a7), Krylov solve (a6), material solve (a8) and the
  // convergence test (a9), as one device-driven CUDA graph or host-driven
  tm.begin(3);
  if ((rc = outer_loop(s, dt))) return rc;
  tm.end();
  // commit (converged, valid input) or restore the snapshot, ghost copies,
  // energy balance and totals; then the one host read of the step
  if ((rc = launch_finish(s, s->e_l, s->E_l))) return rc;
  if ((rc = launch_copy_sync(s))) return rc;
  if ((rc = launch_balance(s, dt, s->E))) return rc;
  if ((rc = launch_totals(s, s->e, s->E))) return rc;
  // time step choice (Sec. 3.3) from the committed state; a step that did not
  // converge restored the snapshot, so its proposal is not reported
  if (s->cfg.dt_target > 0.0 && (rc = launch_dt_control(s, dt))) return rc;
  if ((rc = read_scalars(s))) return rc;
  if (s->sc_host->bad_input) {
    tm.collect(ms);
    return set_error(s, SPH_RT_EINVAL, "non-finite source or ghost value");
  }
  {
    const Scalars &h = *s->sc_host;
    outer_loop_account(s, h);
    st.outer_iters = h.outer_iters;
    st.krylov_iters_total = h.krylov_total;
    for (int k = 0; k < 64 && k < h.outer_iters; ++k)
      st.krylov_iters_per_outer[k] = h.krylov_per_outer[k];
    st.newton_iters_max = h.newton_max;
    st.last_change_e = h.last_change_e;
    st.last_change_E = h.last_change_E;
    SPH_TRACE("step: outer loop status %d, %d outer, %d krylov", h.outer_status, h.outer_iters,
              h.krylov_total);
  }
  const bool converged = s->sc_host->outer_status == 1;
  const bool krylov_fail = s->sc_host->outer_status == 2;
  s->hist = converged ? std::min(hist0 + 1, 3) : 0;  // this step's start is the next E^{n-2}
  s->dt_hist[2] = s->dt_hist[1];
  s->dt_hist[1] = s->dt_hist[0];
  s->dt_hist[0] = dt;
  st.energy_before = s->sc_host->energy_before_e + s->sc_host->energy_before_E;

  if (!converged) {
    // the snapshot was restored on the device (ghost values included)
    tm.collect(ms);
    if (stats) *stats = st;
    return set_error(s, SPH_RT_ENOTCONV,
                     krylov_fail ? "Krylov solve did not converge (max_krylov or breakdown)"
                                 : "outer iteration did not converge within max_outer");
  }
  st.source_energy = s->sc_host->red[6];
  st.boundary_energy = s->sc_host->red[7];
  st.energy_after = s->sc_host->red[4] + s->sc_host->red[5];
  if (s->cfg.dt_target > 0.0) {
    st.eta_e = s->sc_host->dtc_eta_e;
    st.eta_E = s->sc_host->dtc_eta_E;
    st.dt_next = s->sc_host->dtc_next;
  }
  tm.collect(ms);
  st.t_setup_ms = ms[0];
  st.t_assembly_ms = ms[1];
  st.t_amg_ms = ms[2];
  st.t_krylov_ms = ms[3];
  st.t_newton_ms = ms[4];
  if (stats) *stats = st;
  return SPH_RT_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the solver (config.autotune), run once per handle on its first
// step.  The balance between a stronger smoother (fewer Krylov iterations)
// and its sweeps, and whether the finest level's post-smoothing pays (the
// V-cycle-product CG drops it and takes the CG product from the V-cycle's
// A P sweep), depends on the operator and the size: measured at 64^3 the
// symmetric V-cycle wins, at 128^3 the V-cycle-product CG.  Each candidate
// runs the step twice from the same state -- the first run captures its step
// graph (and on the first candidate builds the AMG structure), the second is
// timed with CUDA events on the handle's stream -- and the state is restored
// from the step's own snapshot after each run.  A candidate whose step does
// not converge is skipped; the fastest of the others is kept in s->cfg.
// ---------------------------------------------------------------------------
static sph_rt_status tune_then_step(sph_rt *s, double dt, const double *Qe_c,
                                    const double *QE_c, const double *ge_c, const double *gE_c,
                                    sph_rt_stats *stats) {
  s->solver_tuned = true;  // the trials below are steps too
  s->hist = 0;              // every trial starts its solves from the state
  s->tune_trials.clear();
  const sph_rt_config c0 = s->cfg;
  std::vector<sph_rt_tune_trial> cand;
  if (c0.precond == SPH_RT_PRECOND_JACOBI)  // nothing to tune
    return step_common(s, dt, Qe_c, QE_c, ge_c, gE_c, stats);
  if (c0.precond == SPH_RT_PRECOND_AMG) {
    cand.push_back({0, 1, c0.reliable_drop, -1.0});
    if (c0.precision == SPH_RT_MIXED)
      for (double drop : {1e-4, 1e-6})
        if (drop != c0.reliable_drop) cand.push_back({0, 1, drop, -1.0});
    for (int deg : {1, 2, 3}) cand.push_back({1, deg, c0.reliable_drop, -1.0});
  } else {
    for (int deg : {1, 2, 3, 4, 6}) cand.push_back({c0.fine_post_smooth, deg, c0.reliable_drop, -1.0});
  }
  const size_t nb = sizeof(double) * (size_t)s->n;
  // the step inputs, kept for every trial (a staged host input sits in a
  // buffer that a step may also use as scratch)
  const double *in[4] = {Qe_c, QE_c, ge_c, gE_c};
  double *keep[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int a = 0; a < 4; ++a) {
    if (!in[a]) continue;
    if (!(keep[a] = dalloc<double>(s, s->n))) return SPH_RT_ENOMEM;
    SPH_CUDA(s, cudaMemcpyAsync(keep[a], in[a], nb, cudaMemcpyDeviceToDevice, s->stream));
  }
  cudaEvent_t ev[2] = {nullptr, nullptr};
  SPH_CUDA(s, cudaEventCreate(&ev[0]));
  if (cudaEventCreate(&ev[1]) != cudaSuccess) {
    cudaEventDestroy(ev[0]);
    return set_error(s, SPH_RT_EDEVICE, "autotune: cudaEventCreate failed");
  }
  sph_rt_status rc = SPH_RT_OK;
  int best = -1;
  for (size_t k = 0; k < cand.size() && !rc; ++k) {
    s->cfg.fine_post_smooth = cand[k].fine_post_smooth;
    s->cfg.cheb_degree = cand[k].cheb_degree;
    s->cfg.reliable_drop = cand[k].reliable_drop;
    for (int rep = 0; rep < 2; ++rep) {
      if (cudaEventRecord(ev[0], s->stream) != cudaSuccess) {
        rc = set_error(s, SPH_RT_EDEVICE, "autotune: cudaEventRecord failed");
        break;
      }
      s->hist = 0;
      sph_rt_status r2 = step_common(s, dt, keep[0], keep[1], keep[2], keep[3], nullptr);
      if (r2 == SPH_RT_ENOTCONV) break;  // the step restored its snapshot itself
      if (r2) {
        rc = r2;
        break;
      }
      float ms = -1.0f;
      if (cudaEventRecord(ev[1], s->stream) != cudaSuccess ||
          cudaMemcpyAsync(s->e, s->e_bak, nb, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess ||
          cudaMemcpyAsync(s->E, s->E_bak, nb, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess ||
          cudaStreamSynchronize(s->stream) != cudaSuccess ||
          cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) {
        rc = set_error(s, SPH_RT_EDEVICE, "autotune: CUDA error in a trial");
        break;
      }
      if (rep == 1) cand[k].ms = ms;
    }
    if (!rc && cand[k].ms >= 0.0 && (best < 0 || cand[k].ms < cand[best].ms)) best = (int)k;
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  s->tune_trials = cand;
  s->cfg = c0;
  if (best >= 0) {
    s->cfg.fine_post_smooth = cand[best].fine_post_smooth;
    s->cfg.cheb_degree = cand[best].cheb_degree;
    s->cfg.reliable_drop = cand[best].reliable_drop;
  }
  if (!rc) {
    // the step itself, from the kept inputs (the staged ones may be overwritten)
    s->err.clear();
    s->hist = 0;
    rc = step_common(s, dt, keep[0], keep[1], keep[2], keep[3], stats);
  }
  cudaStreamSynchronize(s->stream);
  for (double *p : keep) dfree(s, p);
  return rc;
}

static sph_rt_status step_entry(sph_rt *s, double dt, const double *Qe, const double *QE,
                                const double *ge, const double *gE, sph_rt_stats *stats,
                                bool device) {
  if (!s) return SPH_RT_EINVAL;
  if (!s->have_particles) return set_error(s, SPH_RT_ESTATE, "step before set_particles");
  if (!isfinite(dt) || dt <= 0.0) return set_error(s, SPH_RT_EINVAL, "dt must be finite and > 0");
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  const int64_t n = s->n;
  if (!device) {
    const double *arrs[4] = {Qe, QE, ge, gE};
    // stage host arrays on the device (caller order); they are checked there
    double *stage[4] = {s->tmp_n, s->tmp_n2, s->stage_ge, s->stage_gE};
    const double *dptr[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < 4; ++k) {
      if (!arrs[k]) continue;
      SPH_CUDA(s, cudaMemcpyAsync(stage[k], arrs[k], sizeof(double) * n, cudaMemcpyHostToDevice,
                                  s->stream));
      dptr[k] = stage[k];
    }
    sph_rt_status rc = step_common(s, dt, dptr[0], dptr[1], dptr[2], dptr[3], stats);
    return rc;
  }
  return step_common(s, dt, Qe, QE, ge, gE, stats);
}

extern "C" sph_rt_status sph_rt_step(sph_rt *s, double dt, const double *Qe, const double *QE,
                                     const double *ghost_e, const double *ghost_E,
                                     sph_rt_stats *stats) {
  return step_entry(s, dt, Qe, QE, ghost_e, ghost_E, stats, false);
}

extern "C" sph_rt_status sph_rt_step_device(sph_rt *s, double dt, const double *Qe,
                                            const double *QE, const double *ghost_e,
                                            const double *ghost_E, sph_rt_stats *stats) {
  return step_entry(s, dt, Qe, QE, ghost_e, ghost_E, stats, true);
}

// ---------------------------------------------------------------------------
// read-out
// ---------------------------------------------------------------------------
extern "C" sph_rt_status sph_rt_get_energies_device(sph_rt *s, double *e, double *E) {
  if (!s) return SPH_RT_EINVAL;
  if (!s->have_particles) return set_error(s, SPH_RT_ESTATE, "no particles");
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  sph_rt_status rc;
  if (e && (rc = launch_scatter_caller(s, s->e, s->n, e))) return rc;
  if (E && (rc = launch_scatter_caller(s, s->E, s->n, E))) return rc;
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_get_energies(sph_rt *s, double *e, double *E, double totals[2]) {
  if (!s) return SPH_RT_EINVAL;
  if (!s->have_particles) return set_error(s, SPH_RT_ESTATE, "no particles");
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  sph_rt_status rc;
  if ((rc = sph_rt_get_energies_device(s, e ? s->tmp_n : nullptr, E ? s->tmp_n2 : nullptr)))
    return rc;
  if (e) SPH_CUDA(s, cudaMemcpyAsync(e, s->tmp_n, sizeof(double) * s->n, cudaMemcpyDeviceToHost, s->stream));
  if (E) SPH_CUDA(s, cudaMemcpyAsync(E, s->tmp_n2, sizeof(double) * s->n, cudaMemcpyDeviceToHost, s->stream));
  if (totals) {
    if ((rc = launch_totals(s, s->e, s->E))) return rc;
    if ((rc = read_scalars(s))) return rc;
    totals[0] = s->sc_host->red[4];
    totals[1] = s->sc_host->red[5];
  }
  SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_extrapolation_weights(int32_t order, double dt,
                                                      const double *dt_hist, double *w) {
  if (!w || order < 0 || order > 3 || (order > 0 && !dt_hist)) return SPH_RT_EINVAL;
  if (!(isfinite(dt) && dt > 0.0)) return SPH_RT_EINVAL;
  for (int j = 0; j < order; ++j)
    if (!(isfinite(dt_hist[j]) && dt_hist[j] > 0.0)) return SPH_RT_EINVAL;
  double g[4] = {1.0, 0.0, 0.0, 0.0};
  if (order > 0) extrap_weights(order, dt, dt_hist, g);
  for (int j = 0; j <= order; ++j) w[j] = g[j];
  return SPH_RT_OK;
}

// The extrapolated Krylov start's history between steps: row 0 is E_old (E^{n-2},
// the last step's start), row j E_hist[j-1] (E^{n-2-j}); depth min(hist, p) rows
// are valid, the ones the next step's extrapolation of order p reads.
static double *history_row(sph_rt *s, int j) { return j == 0 ? s->E_old : s->E_hist[j - 1]; }

extern "C" sph_rt_status sph_rt_get_history(sph_rt *s, int32_t *depth, double *E_hist,
                                            double *dt_hist) {
  if (!s || !depth) return SPH_RT_EINVAL;
  if (!s->have_particles) return set_error(s, SPH_RT_ESTATE, "no particles");
  const int d = std::min(s->hist, s->cfg.krylov_start);
  *depth = d;
  if (dt_hist)
    for (int j = 0; j < 3; ++j) dt_hist[j] = j < d ? s->dt_hist[j] : 0.0;
  if (!E_hist) return SPH_RT_OK;
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  const size_t nb = sizeof(double) * (size_t)s->n;
  sph_rt_status rc;
  for (int j = 0; j < 3; ++j) {
    SPH_CUDA(s, cudaMemsetAsync(s->tmp_n, 0, nb, s->stream));
    if (j < d && (rc = launch_scatter_caller(s, history_row(s, j), s->n_int, s->tmp_n))) return rc;
    SPH_CUDA(s, cudaMemcpyAsync(E_hist + (size_t)j * s->n, s->tmp_n, nb, cudaMemcpyDeviceToHost,
                                s->stream));
    SPH_CUDA(s, cudaStreamSynchronize(s->stream));  // tmp_n is reused by the next row
  }
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_set_history(sph_rt *s, int32_t depth, const double *E_hist,
                                            const double *dt_hist) {
  if (!s || !E_hist || !dt_hist) return SPH_RT_EINVAL;
  if (!s->have_particles) return set_error(s, SPH_RT_ESTATE, "no particles");
  if (depth < 1 || depth > s->cfg.krylov_start)
    return set_error(s, SPH_RT_EINVAL, "depth must be 1 .. krylov_start");
  for (int j = 0; j < depth; ++j)
    if (!(isfinite(dt_hist[j]) && dt_hist[j] > 0.0))
      return set_error(s, SPH_RT_EINVAL, "dt_hist entries must be finite and > 0");
  const int64_t count = (int64_t)depth * s->n;
  for (int64_t i = 0; i < count; ++i)
    if (!isfinite(E_hist[i]))
      return set_error(s, SPH_RT_EINVAL, "non-finite E_hist entry at row " +
                                             std::to_string(i / s->n) + ", particle " +
                                             std::to_string(i % s->n));
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  const size_t nb = sizeof(double) * (size_t)s->n;
  sph_rt_status rc;
  for (int j = 0; j < depth; ++j) {
    SPH_CUDA(s, cudaMemcpyAsync(s->tmp_n, E_hist + (size_t)j * s->n, nb, cudaMemcpyHostToDevice,
                                s->stream));
    if ((rc = launch_gather_interior(s, s->tmp_n, history_row(s, j)))) return rc;
    SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  }
  s->hist = depth;
  for (int j = 0; j < 3; ++j) s->dt_hist[j] = j < depth ? dt_hist[j] : 0.0;
  return SPH_RT_OK;
}

template <typename T>
static sph_rt_status d2h(sph_rt *s, std::vector<T> &out, const T *src, int64_t count) {
  out.resize((size_t)count);
  if (count > 0)
    SPH_CUDA(s, cudaMemcpyAsync(out.data(), src, sizeof(T) * count, cudaMemcpyDeviceToHost, s->stream));
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_get_neighbors(sph_rt *s, int64_t *rowptr, int64_t *cols) {
  if (!s || !rowptr) return SPH_RT_EINVAL;
  if (!s->have_particles) return set_error(s, SPH_RT_ESTATE, "no particles");
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  std::vector<int64_t> s2c, ptr;
  std::vector<int32_t> col;
  sph_rt_status rc;
  if ((rc = d2h(s, s2c, s->slot2caller, s->n))) return rc;
  if ((rc = d2h(s, ptr, s->nbr_ptr, s->n_int + 1))) return rc;
  if (cols && (rc = d2h(s, col, s->nbr_col, s->nnz_nbr))) return rc;
  SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  const int64_t n = s->n;
  std::vector<int64_t> cnt((size_t)n, 0);
  for (int64_t slot = 0; slot < s->n_int; ++slot) cnt[s2c[slot]] = ptr[slot + 1] - ptr[slot];
  rowptr[0] = 0;
  for (int64_t i = 0; i < n; ++i) rowptr[i + 1] = rowptr[i] + cnt[i];
  if (cols) {
    for (int64_t slot = 0; slot < s->n_int; ++slot) {
      int64_t c = s2c[slot];
      int64_t *o = cols + rowptr[c];
      for (int64_t k = ptr[slot]; k < ptr[slot + 1]; ++k) *o++ = s2c[col[k]];
      std::sort(cols + rowptr[c], cols + rowptr[c + 1]);
    }
  }
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_get_operator(sph_rt *s, int64_t *rowptr, int64_t *cols,
                                             double *vals, double *diag, double *gb) {
  if (!s) return SPH_RT_EINVAL;
  if (!s->have_particles || !s->have_operator)
    return set_error(s, SPH_RT_ESTATE, "no operator assembled yet (call sph_rt_step first)");
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  std::vector<int64_t> s2c, ptr;
  std::vector<int32_t> col;
  std::vector<double> val, dg, g, V;
  sph_rt_status rc;
  if ((rc = d2h(s, s2c, s->slot2caller, s->n))) return rc;
  if ((rc = d2h(s, ptr, s->mat_ptr, s->n_int + 1))) return rc;
  if ((rc = d2h(s, col, s->mat_col, s->nnz_mat))) return rc;
  if ((rc = d2h(s, val, s->mat_val, s->nnz_mat))) return rc;
  if ((rc = d2h(s, dg, s->diag, s->n_int))) return rc;
  if ((rc = d2h(s, g, s->gb, s->n_int))) return rc;
  if ((rc = d2h(s, V, s->V, s->n_int))) return rc;
  SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  const int64_t n = s->n;
  std::vector<int64_t> cnt((size_t)n, 0);
  for (int64_t slot = 0; slot < s->n_int; ++slot) cnt[s2c[slot]] = ptr[slot + 1] - ptr[slot];
  std::vector<int64_t> rp((size_t)n + 1, 0);
  for (int64_t i = 0; i < n; ++i) rp[i + 1] = rp[i] + cnt[i];
  if (rowptr) memcpy(rowptr, rp.data(), sizeof(int64_t) * (n + 1));
  if (diag)
    for (int64_t i = 0; i < n; ++i) diag[i] = 0.0;
  if (gb)
    for (int64_t i = 0; i < n; ++i) gb[i] = 0.0;
  for (int64_t slot = 0; slot < s->n_int; ++slot) {
    int64_t c = s2c[slot];
    double invVi = 1.0 / V[slot];
    for (int64_t k = ptr[slot]; k < ptr[slot + 1]; ++k) {
      int64_t at = rp[c] + (k - ptr[slot]);
      if (cols) cols[at] = s2c[col[k]];
      if (vals) vals[at] = val[k] * invVi;
    }
    if (diag) diag[c] = dg[slot] * invVi;
    if (gb) gb[c] = g[slot];
  }
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_get_properties(sph_rt *s, double *T, double *sigma, double *f,
                                               double *R, double *lambda, double *D) {
  if (!s) return SPH_RT_EINVAL;
  if (!s->have_particles || !s->have_operator)
    return set_error(s, SPH_RT_ESTATE, "no step taken yet");
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  double *outs[6] = {T, sigma, f, R, lambda, D};
  const double *srcs[6] = {s->T, s->sigma, s->f, s->R, s->lambda, s->D};
  for (int k = 0; k < 6; ++k) {
    if (!outs[k]) continue;
    sph_rt_status rc = launch_scatter_caller(s, srcs[k], s->n, s->tmp_n);
    if (rc) return rc;
    SPH_CUDA(s, cudaMemcpyAsync(outs[k], s->tmp_n, sizeof(double) * s->n, cudaMemcpyDeviceToHost, s->stream));
    SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  }
  return SPH_RT_OK;
}

namespace sphrt {
int amg_levels(const sph_rt *s, int64_t *rows, int64_t *nnz, int maxl);
}

extern "C" sph_rt_status sph_rt_get_amg_info(sph_rt *s, int32_t *nlevels, int64_t *rows,
                                             int64_t *nnz, int32_t max_levels) {
  if (!s || !nlevels) return SPH_RT_EINVAL;
  if (!s->amg_ready) return set_error(s, SPH_RT_ESTATE, "no AMG hierarchy (step with precond AMG first)");
  int64_t r[64], z[64];
  int k = amg_levels(s, r, z, 64);
  *nlevels = k;
  for (int l = 0; l < k && l < max_levels; ++l) {
    if (rows) rows[l] = r[l];
    if (nnz) nnz[l] = z[l];
  }
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_kernel_stats(sph_rt *s, int64_t *launches, double *total_ms,
                                             double *bytes, int reset) {
  if (!s) return SPH_RT_EINVAL;
  if (launches) *launches = s->spmv_launches;
  if (total_ms) *total_ms = s->spmv_ms;
  if (bytes) *bytes = s->spmv_bytes;
  if (reset) {
    s->spmv_launches = 0;
    s->spmv_ms = 0.0;
    s->spmv_bytes = 0.0;
    for (int k = 0; k < kTimedKinds; ++k) {
      s->kind_launches[k] = 0;
      s->kind_ms[k] = 0.0;
      s->kind_bytes[k] = 0.0;
    }
  }
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_kernel_stats_kind(sph_rt *s, int32_t kind, int64_t *launches,
                                                  double *total_ms, double *bytes) {
  if (!s) return SPH_RT_EINVAL;
  if (kind < 0 || kind >= kTimedKinds)
    return set_error(s, SPH_RT_EINVAL, "kernel kind out of range");
  if (launches) *launches = s->kind_launches[kind];
  if (total_ms) *total_ms = s->kind_ms[kind];
  if (bytes) *bytes = s->kind_bytes[kind];
  return SPH_RT_OK;
}
