// graph.cu -- the outer loop of Alg. 1 (rows a6-a9 of the hot path):
//
//   while e^n, E^n not converged (Eq. mat-rad-convergence):
//     right-hand side of r-dagger (Eq. ne-equations), Krylov solve for E^{l+1},
//     per-particle material solve m(e, E^{l+1}) = 0 (Eq. full-material-solve)
//
// Two drivers run the same kernels in the same order (results are bitwise
// the same):
//   * graph: the whole loop is one CUDA graph.  An outer conditional WHILE
//     node repeats {rhs, CG prologue, inner WHILE node {one CG iteration},
//     material solve, convergence test}; the loop conditions are set on the
//     device (cudaGraphSetConditional), so a step needs no host round trip
//     between its first and its last kernel and no launch is issued after
//     convergence.  The graph is captured once per particle set / hierarchy
//     and replayed every step while the launch parameters stay the same.
//   * host: the loop runs on the host, reading the device state after every
//     outer iteration (used with per-launch kernel timing).
// Every device-side loop is bounded: the Krylov loop by max_krylov + 1 trips,
// the outer loop by max_outer + 1 trips, whatever the arithmetic does.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "common.cuh"

namespace sphrt {

sph_rt_status launch_rhs(sph_rt *s, double dt);
sph_rt_status launch_newton(sph_rt *s, double dt, const double *E_new, const double *E_prev,
                            const double *e_start, double *e_out);
sph_rt_status pcg_prologue(sph_rt *s);
sph_rt_status pcg_iteration(sph_rt *s);
sph_rt_status pcg_solve(sph_rt *s, int *iters, bool *converged);
void amg_signature(const sph_rt *s, std::vector<uint64_t> &sig);
CsrView<double> fine_view(const sph_rt *s);

// outer-loop state at the start of a step; newton_max starts from the initial
// material solve of Alg. 1 (its iteration count is in red[2])
__global__ void outer_init_kernel(Scalars *sc) {
  sc->outer_iters = 0;
  sc->outer_status = 0;
  sc->outer_trips = 0;
  sc->krylov_total = 0;
  sc->krylov_trips = 0;
  sc->krylov_solve_trips = 0;
  sc->newton_max = (int)sc->red[2];
  sc->yvalid = 0;  // a new step has a new operator
  sc->last_change_e = 0.0;
  sc->last_change_E = 0.0;
  for (int k = 0; k < 64; ++k) sc->krylov_per_outer[k] = 0;
}

// Before the Krylov WHILE node: enter unless the prologue already converged.
__global__ void krylov_enter_kernel(Scalars *sc, cudaGraphConditionalHandle h) {
  sc->krylov_solve_trips = 0;
  cudaGraphSetConditional(h, sc->done ? 0u : 1u);
}

// End of a Krylov trip: go on while not converged, at most max_trips trips.
__global__ void krylov_cond_kernel(Scalars *sc, int max_trips, cudaGraphConditionalHandle h) {
  sc->krylov_trips += 1;
  const int t = ++sc->krylov_solve_trips;
  cudaGraphSetConditional(h, (sc->done || t >= max_trips) ? 0u : 1u);
}

// After the material solve of an outer iteration: the Krylov check, the
// bookkeeping of the step statistics and the outer convergence test
// max_i |x^{l+1} - x^l| / |x^{l+1}| < tol for e and E (changes in red[0..1],
// Newton iterations in red[2]).  In the graph it also sets the loop condition.
__global__ void outer_check_kernel(Scalars *sc, double tol_e, double tol_E, int max_outer,
                                   cudaGraphConditionalHandle h, int in_graph) {
  int status = 0;
  sc->outer_trips += 1;
  const bool kconv = !sc->breakdown && !(sc->rnorm2 > sc->thresh2);
  if (!kconv) {
    status = 2;
  } else {
    const int o = sc->outer_iters;
    if (o < 64) sc->krylov_per_outer[o] = sc->iters;
    sc->krylov_total += sc->iters;
    sc->outer_iters = o + 1;
    const double ce = sc->red[0], cE = sc->red[1];
    sc->newton_max = max(sc->newton_max, (int)sc->red[2]);
    sc->last_change_e = ce;
    sc->last_change_E = cE;
    if (ce < tol_e && cE < tol_E)
      status = 1;
    else if (sc->outer_iters >= max_outer)
      status = 3;
  }
  if (status == 0 && sc->outer_trips > max_outer) status = 3;
  sc->outer_status = status;
  if (in_graph) cudaGraphSetConditional(h, status == 0 ? 1u : 0u);
}

// The new iterate becomes the current one: e^l <- e^{l+1}, E^l <- E^{l+1} (= x).
__global__ void iterate_copy_kernel(int64_t n, const double *e_new, double *e_l,
                                    const double *x, double *E_l) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    e_l[i] = e_new[i];
    E_l[i] = x[i];
  }
}

static int copy_grid(const sph_rt *s, int64_t n) {
  int64_t g = ceil_div(n > 0 ? n : 1, kBlock), cap = (int64_t)s->num_sms * 8;
  return (int)(g < cap ? g : cap);
}

static sph_rt_status launch_outer_tail(sph_rt *s, double dt, cudaGraphConditionalHandle h,
                                       int in_graph) {
  sph_rt_status rc;
  // a8: material solve with E^{l+1} = x, from e^l
  if ((rc = launch_newton(s, dt, s->x, s->E_l, s->e_l, s->e_new))) return rc;
  // a9: convergence test and statistics
  outer_check_kernel<<<1, 1, 0, s->stream>>>(s->sc, s->cfg.tol_outer_e, s->cfg.tol_outer_E,
                                              s->cfg.max_outer, h, in_graph);
  SPH_LAUNCHED(s);
  iterate_copy_kernel<<<copy_grid(s, s->n_int), kBlock, 0, s->stream>>>(
      s->n_int, s->e_new, s->e_l, s->x, s->E_l);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

// ---------------------------------------------------------------------------
// host-driven loop
// ---------------------------------------------------------------------------
static sph_rt_status outer_loop_host(sph_rt *s, double dt) {
  sph_rt_status rc;
  outer_init_kernel<<<1, 1, 0, s->stream>>>(s->sc);
  SPH_LAUNCHED(s);
  for (;;) {
    if ((rc = launch_rhs(s, dt))) return rc;  // a7 (also x = E^l)
    int kit = 0;
    bool kconv = false;
    if ((rc = pcg_solve(s, &kit, &kconv))) return rc;  // a6
    if ((rc = launch_outer_tail(s, dt, 0, 0))) return rc;
    SPH_CUDA(s, cudaMemcpyAsync(s->sc_host, s->sc, sizeof(Scalars), cudaMemcpyDeviceToHost,
                                s->stream));
    SPH_CUDA(s, cudaStreamSynchronize(s->stream));
    SPH_TRACE("outer %d: krylov %d, changes %g %g, status %d", s->sc_host->outer_iters, kit,
              s->sc_host->last_change_e, s->sc_host->last_change_E, s->sc_host->outer_status);
    if (s->sc_host->outer_status != 0) return SPH_RT_OK;
  }
}

// ---------------------------------------------------------------------------
// graph-driven loop
// ---------------------------------------------------------------------------
static void sig_u64(std::vector<uint64_t> &v, const void *p, size_t bytes) {
  const unsigned char *c = static_cast<const unsigned char *>(p);
  for (size_t o = 0; o < bytes; o += 8) {
    uint64_t w = 0;
    memcpy(&w, c + o, bytes - o < 8 ? bytes - o : 8);
    v.push_back(w);
  }
}

// Everything the captured launches depend on: configuration, dt, sizes, the
// buffers they touch and the fine / AMG operator layout.
static std::vector<uint64_t> loop_signature(const sph_rt *s, double dt) {
  std::vector<uint64_t> v;
  sph_rt_config c;
  memcpy(&c, &s->cfg, sizeof c);  // bytewise (padding included): stable across calls
  c.stream = nullptr;  // the graph is launched on the current stream, whatever it is
  sig_u64(v, &c, sizeof c);
  sig_u64(v, &dt, sizeof dt);
  const int64_t sizes[4] = {s->n, s->n_int, s->nnz_mat, (int64_t)s->num_sms};
  sig_u64(v, sizes, sizeof sizes);
  const void *bufs[] = {s->b,     s->x,     s->r,    s->z,     s->z_old, s->p,      s->q,
                        s->w,     s->tmp_n2, s->invV, s->sc,   s->partials, s->e_l, s->e_new,
                        s->E_l,   s->E_old, s->e_old, s->rho, s->sigma, s->f,       s->Qe,
                        s->QE,    s->gb,    s->V,     s->cheb_slots};
  sig_u64(v, bufs, sizeof bufs);
  CsrView<double> A = fine_view(s);
  sig_u64(v, &A, sizeof A);
  if (s->cfg.precond == SPH_RT_PRECOND_AMG) amg_signature(s, v);
  return v;
}

void loop_graph_release(sph_rt *s) {
  if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
  if (s->graph) cudaGraphDestroy(s->graph);
  s->graph_exec = nullptr;
  s->graph = nullptr;
  s->graph_sig.clear();
}

// Capture the loop.  Launch helpers write to s->stream, which points at the
// private capture stream meanwhile; the launch counter is restored afterwards
// (captured kernels are counted when the graph runs).
static sph_rt_status build_loop_graph(sph_rt *s, double dt) {
  loop_graph_release(s);
  if (!s->cap_stream) SPH_CUDA(s, cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  SPH_CUDA(s, cudaGraphCreate(&g, 0));
  s->graph = g;
  cudaGraphConditionalHandle h_out, h_in;
  SPH_CUDA(s, cudaGraphConditionalHandleCreate(&h_out, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams op = {cudaGraphNodeTypeConditional};
  op.conditional.handle = h_out;
  op.conditional.type = cudaGraphCondTypeWhile;
  op.conditional.size = 1;
  cudaGraphNode_t n_out;
  SPH_CUDA(s, cudaGraphAddNode(&n_out, g, nullptr, nullptr, 0, &op));
  cudaGraph_t body_out = op.conditional.phGraph_out[0];
  SPH_CUDA(s, cudaGraphConditionalHandleCreate(&h_in, body_out, 0, 0));

  cudaStream_t user = s->stream;
  const int64_t launches0 = s->launches;
  s->stream = s->cap_stream;
  cudaGraph_t body_in = nullptr;
  auto capture_outer = [&]() -> sph_rt_status {
    sph_rt_status rc;
    if ((rc = launch_rhs(s, dt))) return rc;  // a7
    if ((rc = pcg_prologue(s))) return rc;     // a6, first part
    krylov_enter_kernel<<<1, 1, 0, s->stream>>>(s->sc, h_in);
    SPH_LAUNCHED(s);
    // the Krylov WHILE node goes after everything captured so far
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaGraph_t cg = nullptr;
    SPH_CUDA(s, cudaStreamGetCaptureInfo(s->stream, &cst, nullptr, &cg, &deps, nullptr, &ndeps));
    cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
    ip.conditional.handle = h_in;
    ip.conditional.type = cudaGraphCondTypeWhile;
    ip.conditional.size = 1;
    cudaGraphNode_t n_in;
    SPH_CUDA(s, cudaGraphAddNode(&n_in, cg, deps, nullptr, ndeps, &ip));
    body_in = ip.conditional.phGraph_out[0];
    SPH_CUDA(s, cudaStreamUpdateCaptureDependencies(s->stream, &n_in, nullptr, 1,
                                                    cudaStreamSetCaptureDependencies));
    return launch_outer_tail(s, dt, h_out, 1);  // a8, a9
  };
  auto capture_inner = [&]() -> sph_rt_status {
    sph_rt_status rc;
    if ((rc = pcg_iteration(s))) return rc;  // a6, one iteration
    krylov_cond_kernel<<<1, 1, 0, s->stream>>>(s->sc, s->cfg.max_krylov + 1, h_in);
    SPH_LAUNCHED(s);
    return SPH_RT_OK;
  };
  auto capture_into = [&](cudaGraph_t into, auto &&body, int64_t *count) -> sph_rt_status {
    const int64_t l0 = s->launches;
    SPH_CUDA(s, cudaStreamBeginCaptureToGraph(s->stream, into, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed));
    sph_rt_status rc = body();
    cudaGraph_t out = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->stream, &out);
    if (rc) return rc;
    if (e != cudaSuccess) {
      cuda_ok(s, e, "cudaStreamEndCapture");
      return SPH_RT_EDEVICE;
    }
    *count = s->launches - l0;
    return SPH_RT_OK;
  };
  sph_rt_status rc = capture_into(body_out, capture_outer, &s->graph_l_outer);
  if (!rc) rc = capture_into(body_in, capture_inner, &s->graph_l_inner);
  s->stream = user;
  s->launches = launches0;
  if (rc) {
    loop_graph_release(s);
    return rc;
  }
  SPH_CUDA(s, cudaGraphInstantiate(&s->graph_exec, g, 0));
  s->graph_sig = loop_signature(s, dt);
  s->graph_builds++;
  SPH_TRACE("loop graph captured: %lld kernels per outer trip, %lld per Krylov trip",
            (long long)s->graph_l_outer, (long long)s->graph_l_inner);
  return SPH_RT_OK;
}

static sph_rt_status outer_loop_graph(sph_rt *s, double dt) {
  sph_rt_status rc;
  if (!s->graph_exec || s->graph_sig != loop_signature(s, dt)) {
    if ((rc = build_loop_graph(s, dt))) return rc;
  }
  outer_init_kernel<<<1, 1, 0, s->stream>>>(s->sc);
  SPH_LAUNCHED(s);
  SPH_CUDA(s, cudaGraphLaunch(s->graph_exec, s->stream));
  s->graph_launches++;
  return SPH_RT_OK;
}

// Runs the loop; the results are in the device Scalars (outer_status and the
// statistics), read by the caller.
sph_rt_status outer_loop(sph_rt *s, double dt) {
  if (s->cfg.graphs && !s->cfg.kernel_timing) return outer_loop_graph(s, dt);
  return outer_loop_host(s, dt);
}

// Kernels the graph ran, from the trip counters (after the Scalars were read).
void outer_loop_account(sph_rt *s, const Scalars &h) {
  if (!(s->cfg.graphs && !s->cfg.kernel_timing)) return;
  s->launches += (int64_t)h.outer_trips * s->graph_l_outer +
                 (int64_t)h.krylov_trips * s->graph_l_inner;
}

}  // namespace sphrt
