// krylov.cu -- preconditioned conjugate gradients for the radiation diffusion
// solve (row a6 of the hot path), plus the SpMV-shaped kernels it is built
// from (Jacobi and Chebyshev preconditioners; the Chebyshev kernels are also
// the AMG smoother).
//
// The paper solves Eq. diffusion-solve with GMRES and a BoomerAMG
// preconditioner, set up once per step and warm-started from E^l (Sec. 3.2).
// Here the operator is stored as B = V A, which is symmetric positive
// definite (an M-matrix with strict diagonal dominance), so CG is the Krylov
// method.  Per iteration: the x / r update fused with ||r|| and the
// convergence test, the preconditioner, the inner product (r, z), and the
// SpMV fused with the direction update and (p, q).  With the AMG
// preconditioner the update also writes the V-cycle's first smoother step and
// (r, z) rides in the V-cycle's last sweep.  The stopping test is the paper's
// unscaled residual ||b - A E||_2 <= tol ||b||_2, with A E - b = V^{-1}(B E - V b).
//
// All scalars of the iteration (rho, alpha, beta, norms, convergence flag)
// live on the device.  Every kernel of an iteration starts by reading the
// `done` flag.  The iteration is driven either from the host (several
// iterations queued per read of the flag; iterations queued after
// convergence are empty launches) or, inside the step's CUDA graph, by a
// conditional WHILE node that stops exactly at convergence (graph.cu).
#include <cuda_runtime.h>

#include <cstring>
#include <utility>
#include <vector>

#include "common.cuh"

namespace sphrt {

template <typename T>
__device__ __forceinline__ T ld(const T *p) {
  return __ldg(p);
}

// ---------------------------------------------------------------------------
// r = b - B x;  rnorm2 = ||r / V||^2;  done = rnorm2 <= thresh2.
// ---------------------------------------------------------------------------
template <int W, int U>
__global__ void __launch_bounds__(kBlock, sweep_min_blocks(U)) resid_kernel(CsrView<double> A, const double *b, const double *x, double *r,
                             const double *invV, Scalars *sc, double *partials, int *wflag) {
  pdl_wait();
  mark_work(wflag, 1);
  const int own = tile_own_row<W>(threadIdx.x & 31);
  int64_t r0, r1;
  warp_rows<W>(A.n, r0, r1);
  double acc = 0.0;
  for (int64_t base = r0; base < r1; base += 32) {
    const int rows = (int)(r1 - base < 32 ? r1 - base : 32);
    const int64_t i = base + own;
    const bool active = own < rows;
    const double s = tile_row_sums<W, U, double, double>(base, rows, A.ptr, A.col, A.val, x);
    if (active) {
      const double bi = b[i], dg = A.diag[i], xi = x[i], iv = invV[i];
      double ri = bi - fmadd(dg, xi, s);
      r[i] = ri;
      double ru = ri * iv;
      acc += ru * ru;
    }
  }
  __shared__ double sh[32];
  acc = block_sum(acc, sh);
  double part[1] = {acc}, out[1];
  const bool mx[1] = {false};
  if (last_block_combine<1>(part, partials, &sc->counter, out, mx) && threadIdx.x == 0) {
    sc->rnorm2 = out[0];
    sc->iters = 0;
    sc->done = !(out[0] > sc->thresh2);  // also stops on NaN
    if (!(out[0] == out[0])) sc->breakdown = 1;
  }
}

// ---------------------------------------------------------------------------
// w = B z;  q = w + beta q;  p = z + beta p;  pq = (p, q);  alpha = rho / pq.
// (q = B p without a second SpMV: B p = B z + beta B p_old.)
// ---------------------------------------------------------------------------
template <int W, int U>
__global__ void __launch_bounds__(kBlock, sweep_min_blocks(U)) spmv_pq_kernel(CsrView<double> A, const double *z, double *q, double *p, int first,
                               Scalars *sc, double *partials, int *wflag) {
  pdl_wait();
  if (sc->done) {
    mark_work(wflag, 0);
    return;
  }
  mark_work(wflag, 1);
  const double beta = first ? 0.0 : sc->beta;
  const int own = tile_own_row<W>(threadIdx.x & 31);
  int64_t r0, r1;
  warp_rows<W>(A.n, r0, r1);
  double acc = 0.0;
  for (int64_t base = r0; base < r1; base += 32) {
    const int rows = (int)(r1 - base < 32 ? r1 - base : 32);
    const int64_t i = base + own;
    const bool active = own < rows;
    const double s = tile_row_sums<W, U, double, double>(base, rows, A.ptr, A.col, A.val, z);
    if (active) {
      const double zi = z[i], dg = A.diag[i];
      const double qo = first ? 0.0 : q[i], po = first ? 0.0 : p[i];
      double wi = fmadd(dg, zi, s);
      double qi = first ? wi : fmadd(beta, qo, wi);
      double pi = first ? zi : fmadd(beta, po, zi);
      q[i] = qi;
      p[i] = pi;
      acc += pi * qi;
    }
  }
  __shared__ double sh[32];
  acc = block_sum(acc, sh);
  double part[1] = {acc}, out[1];
  const bool mx[1] = {false};
  if (last_block_combine<1>(part, partials, &sc->counter, out, mx) && threadIdx.x == 0) {
    double pq = out[0];
    sc->pq = pq;
    if (!(pq > 0.0) || !(pq < 1e308)) {  // loss of positive definiteness or NaN
      sc->breakdown = 1;
      sc->done = 1;
    } else {
      sc->alpha = sc->rho / pq;
    }
  }
}

// x += alpha p;  r -= alpha q;  rnorm2 = ||r / V||^2;  convergence test; and,
// with fi.d set, the finest level's zero-guess smoother start on the new r
// (FineInit).  The start is also written when this iteration converges; the
// V-cycle's launches then return at once and nothing reads it.
template <typename IT>
__global__ void update_kernel(int64_t n, double *x, double *r, const double *p, const double *q,
                              const double *invV, int maxit, Scalars *sc, double *partials,
                              FineInit<IT> fi) {
  pdl_wait();
  if (sc->done) return;
  const double alpha = sc->alpha;
  const double inv_theta = fi.d ? fi.cf->inv_theta : 0.0;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    double ri = r[i] - alpha * q[i];
    r[i] = ri;
    double ru = ri * invV[i];
    acc += ru * ru;
    if (fi.d) {
      const IT rv = (IT)ri;
      if (fi.r_lo) fi.r_lo[i] = rv;
      const IT di = (IT)(inv_theta * (double)fi.invdiag[i] * (double)rv);
      fi.d[i] = di;
      fi.z[i] = di;
    }
  }
  __shared__ double sh[32];
  acc = block_sum(acc, sh);
  double part[1] = {acc}, out[1];
  const bool mx[1] = {false};
  if (last_block_combine<1>(part, partials, &sc->counter, out, mx) && threadIdx.x == 0) {
    sc->rnorm2 = out[0];
    sc->iters += 1;
    if (!(out[0] > sc->thresh2) || sc->iters >= maxit) sc->done = 1;
    if (!(out[0] == out[0])) sc->breakdown = 1;
  }
}

// Jacobi: z = D^{-1} r, fused with rho = (r, z) and beta.
__global__ void jacobi_dot_kernel(int64_t n, const double *r, const double *invdiag, double *z,
                                  int first, Scalars *sc, double *partials) {
  pdl_wait();
  if (sc->done) return;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double zi = r[i] * invdiag[i];
    z[i] = zi;
    acc += r[i] * zi;
  }
  __shared__ double sh[32];
  acc = block_sum(acc, sh);
  double part[1] = {acc}, out[1];
  const bool mx[1] = {false};
  if (last_block_combine<1>(part, partials, &sc->counter, out, mx) && threadIdx.x == 0) {
    if (!first) sc->beta = out[0] / sc->rho;
    sc->rho = out[0];
  }
}

// rho = (r, z) and beta, for preconditioners that write z themselves.
template <typename VT>
__global__ void dot_rz_kernel(int64_t n, const double *r, const VT *z, int first, Scalars *sc,
                              double *partials) {
  pdl_wait();
  if (sc->done) return;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += r[i] * (double)z[i];
  __shared__ double sh[32];
  acc = block_sum(acc, sh);
  double part[1] = {acc}, out[1];
  const bool mx[1] = {false};
  if (last_block_combine<1>(part, partials, &sc->counter, out, mx) && threadIdx.x == 0) {
    if (!first) sc->beta = out[0] / sc->rho;
    sc->rho = out[0];
  }
}

// Flexible variant (Polak-Ribiere): beta = ((r, z) - (r, z_old)) / rho_old.
// Used when the preconditioner is only approximately symmetric (an FP32
// V-cycle): it keeps CG's short recurrence without assuming exact symmetry.
__global__ void dot_rz_flex_kernel(int64_t n, const double *r, const double *z,
                                   const double *z_old, int first, Scalars *sc,
                                   double *partials) {
  pdl_wait();
  if (sc->done) return;
  double a = 0.0, b = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double ri = r[i];
    a += ri * z[i];
    if (!first) b += ri * z_old[i];
  }
  __shared__ double sh[32];
  a = block_sum(a, sh);
  __syncthreads();
  b = block_sum(b, sh);
  double part[2] = {a, b}, out[2];
  const bool mx[2] = {false, false};
  if (last_block_combine<2>(part, partials, &sc->counter, out, mx) && threadIdx.x == 0) {
    if (!first) sc->beta = (out[0] - out[1]) / sc->rho;
    sc->rho = out[0];
  }
}

// The same for the FP32 V-cycle of the mixed form, fused with widening its
// result: z32 is the new preconditioned residual, z still holds the previous
// one (the FP32 V-cycle never writes z), so (r, z_old) is read from z before
// z = (double) z32 overwrites it.  Same sums in the same order as widening,
// copying z to z_old and dot_rz_flex_kernel, in one pass instead of three.
__global__ void dot_rz_flex32_kernel(int64_t n, const double *r, const float *z32, double *z,
                                     int first, Scalars *sc, double *partials) {
  pdl_wait();
  if (sc->done) return;
  double a = 0.0, b = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = r[i];
    const double zn = (double)z32[i];
    if (!first) b += ri * z[i];
    a += ri * zn;
    z[i] = zn;
  }
  __shared__ double sh[32];
  a = block_sum(a, sh);
  __syncthreads();
  b = block_sum(b, sh);
  double part[2] = {a, b}, out[2];
  const bool mx[2] = {false, false};
  if (last_block_combine<2>(part, partials, &sc->counter, out, mx) && threadIdx.x == 0) {
    if (!first) sc->beta = (out[0] - out[1]) / sc->rho;
    sc->rho = out[0];
  }
}

// ---------------------------------------------------------------------------
// Chebyshev iteration for A z = r (A = level operator, D = its diagonal) on
// the interval [lmin, lmax] of D^{-1} A (Saad, Iterative Methods, Alg. 12.1).
// init:  zero guess:  d = D^{-1} r / theta,              z = d
//        otherwise:   d = D^{-1} (r - A z_in) / theta,   z_out = z_in + d
// step:  d = c1 d + c2 D^{-1} (r - A z_in),              z_out = z_in + d
// ---------------------------------------------------------------------------
template <typename MT, typename VT>
__global__ void cheb_init_zero_kernel(int64_t n, const VT *r, const MT *invdiag,
                                      const ChebCoef *cf, VT *d, VT *z, const Scalars *sc) {
  pdl_wait();
  if (sc && sc->done) return;
  const double inv_theta = cf->inv_theta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    VT di = (VT)(inv_theta * (double)invdiag[i] * (double)r[i]);
    d[i] = di;
    z[i] = di;
  }
}


// PRE: load the row operands before the row sums (coarse levels: shorter
// dependent chain) or after them (finest level: fewer registers, more warps).
template <int W, int U, typename MT, typename VT, bool PRE>
__device__ __forceinline__ void cheb_step_body(const CsrView<MT> &A, const VT *r, const VT *z_in,
                                               VT *z_out, VT *d, const ChebCoef *cf, int k,
                                               const Scalars *sc, int *wflag) {
  pdl_wait();
  if (sc && sc->done) {
    mark_work(wflag, 0);
    return;
  }
  mark_work(wflag, 1);
  // step k of the recurrence; k = 0 is the first step from a nonzero guess
  const double c1 = k > 0 ? cf->c1[k] : 0.0, c2 = k > 0 ? cf->c2[k] : cf->inv_theta;
  const VT vc1 = (VT)c1, vc2 = (VT)c2;
  const int own = tile_own_row<W>(threadIdx.x & 31);
  int64_t r0, r1;
  warp_rows<W>(A.n, r0, r1);
  for (int64_t base = r0; base < r1; base += 32) {
    const int rows = (int)(r1 - base < 32 ? r1 - base : 32);
    const int64_t i = base + own;
    const bool active = own < rows;
    VT ri = VT(0), zi = VT(0), dg = VT(0), idg = VT(0), dold = VT(0);
    auto operands = [&]() {
      ri = r[i];
      zi = z_in[i];
      dg = (VT)A.diag[i];
      idg = (VT)A.invdiag[i];
      if (k > 0) dold = d[i];  // the first step must not read d
    };
    if (PRE && active) operands();
    const VT s = tile_row_sums<W, U, MT, VT>(base, rows, A.ptr, A.col, A.val, z_in);
    if (active) {
      if (!PRE) operands();
      VT res = ri - fmadd(dg, zi, s);
      VT di = (vc2 * idg) * res;
      if (k > 0) di = fmadd(vc1, dold, di);
      d[i] = di;
      z_out[i] = zi + di;
    }
  }
}
// The same sweep under two names, so that profiles separate the finest
// level (HBM-streamed operator) from the coarse levels (L2-resident).
template <int W, int U, typename MT, typename VT>
__global__ void __launch_bounds__(kBlock, kCoarseMinBlocks) cheb_step_kernel(CsrView<MT> A, const VT *r, const VT *z_in, VT *z_out, VT *d,
                                 const ChebCoef *cf, int k, const Scalars *sc, int *wflag) {
  cheb_step_body<W, U, MT, VT, true>(A, r, z_in, z_out, d, cf, k, sc, wflag);
}
template <int W, int U, typename MT, typename VT>
__global__ void __launch_bounds__(kBlock, sweep_min_blocks(U)) fine_cheb_step_kernel(CsrView<MT> A, const VT *r, const VT *z_in, VT *z_out,
                                      VT *d, const ChebCoef *cf, int k, const Scalars *sc,
                                      int *wflag) {
  cheb_step_body<W, U, MT, VT, false>(A, r, z_in, z_out, d, cf, k, sc, wflag);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int grid_cap(const sph_rt *s, int64_t n, int per_block) {
  int64_t g = ceil_div(n > 0 ? n : 1, per_block);
  int64_t cap = (int64_t)s->num_sms * 8;
  if (cap > kMaxRedBlocks) cap = kMaxRedBlocks;
  return (int)(g < cap ? g : cap);
}


CsrView<double> fine_view(const sph_rt *s) {
  CsrView<double> A;
  memset(&A, 0, sizeof A);  // no indeterminate padding (the view is part of a graph signature)
  A.n = s->n_int;
  A.ptr = s->mat_ptr;
  A.col = s->mat_col;
  A.val = s->mat_val;
  A.diag = s->diag;
  A.invdiag = s->invdiag;
  A.nnz = s->nnz_mat;
  RowShape sh = s->fine_shape_set ? s->fine_shape
                                  : shape_for_mean(s->n_int ? (double)s->nnz_mat / s->n_int : 0.0);
  A.W = sh.W;
  A.U = sh.U;
  return A;
}

// Kernel-time bracketing of fine SpMV-class launches (config.kernel_timing).
constexpr int kEventPairs = 2048;
void timing_flush(sph_rt *s) {
  if (s->gate_host) *s->gate_host = s->gate_epoch;  // never wait on a held stream
  if (!s->cfg.kernel_timing || s->ev_used == 0) return;
  const int pairs = s->ev_used / 2;
  std::vector<int> flags(pairs, 1);
  cudaEventSynchronize(s->ev_pool[s->ev_used - 1]);
  if (s->ev_flags)
    cudaMemcpy(flags.data(), s->ev_flags, sizeof(int) * pairs, cudaMemcpyDeviceToHost);
  for (int k = 0; k < pairs; ++k) {
    if (!flags[k]) continue;  // returned at once: the solve had converged
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s->ev_pool[2 * k], s->ev_pool[2 * k + 1]);
    s->spmv_ms += ms;
    s->spmv_launches++;
    s->spmv_bytes += s->ev_bytes[k];
    const int kd = s->ev_kind[k];
    s->kind_ms[kd] += ms;
    s->kind_launches[kd]++;
    s->kind_bytes[kd] += s->ev_bytes[k];
  }
  s->ev_used = 0;
}
int *timing_begin(sph_rt *s) {
  if (!s->cfg.kernel_timing) return nullptr;
  if (s->ev_pool.empty()) {
    for (int k = 0; k < 2 * kEventPairs; ++k) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) break;
      s->ev_pool.push_back(e);
    }
    s->ev_bytes.assign(kEventPairs, 0.0);
    s->ev_kind.assign(kEventPairs, 0);
  }
  if (!s->ev_flags) s->ev_flags = dalloc<int>(s, kEventPairs);
  if (s->ev_used + 2 > (int)s->ev_pool.size()) timing_flush(s);
  const int pair = s->ev_used / 2;
  cudaEventRecord(s->ev_pool[s->ev_used++], s->stream);
  return s->ev_flags ? s->ev_flags + pair : nullptr;
}
void timing_end(sph_rt *s, double bytes, int kind) {
  if (!s->cfg.kernel_timing) return;
  s->ev_bytes[(s->ev_used - 1) / 2] = bytes;
  s->ev_kind[(s->ev_used - 1) / 2] = kind;
  cudaEventRecord(s->ev_pool[s->ev_used++], s->stream);
}

// Algorithmic bytes of the SpMV-class kernels: column index and value per
// stored nonzero (the gathered vector entry counted once, per row) plus the
// per-row vectors each kernel reads and writes.
template <typename MT>
double spmv_class_bytes(const CsrView<MT> &A, int row_bytes) {
  return (4.0 + sizeof(MT)) * (double)A.nnz + (double)row_bytes * (double)A.n;
}
// resid: rowptr, diag, b, x, r, 1/V        spmv_pq: rowptr, diag, z, q r/w, p r/w
constexpr int kRowBytesResid = 48, kRowBytesSpmvPQ = 56;

// Chebyshev polynomial preconditioner/smoother: `degree` steps from z
// (zero_guess: z = 0 on entry), coefficients from the device slot `cf`
// (filled on the device from the Gershgorin bounds of the step, so no host
// read of the bounds is needed).  d and tmp are scratch vectors of length n.
template <typename MT, typename VT>
sph_rt_status cheb_apply(sph_rt *s, const CsrView<MT> &A, const VT *r, VT *z, VT *d, VT *tmp,
                         int degree, const ChebCoef *cf, bool zero_guess, const Scalars *sc,
                         bool first_step_done) {
  if (degree < 1) degree = 1;
  if (degree > kChebMaxDeg) degree = kChebMaxDeg;
  int g = grid_cap(s, A.n, kBlock);
  // fine-level sweeps are timed with the other fine SpMV-class kernels; per row:
  // rowptr, diag, 1/diag, r, z_in, z_out, d r/w (vectors of type VT)
  const bool fine = A.ptr == s->mat_ptr;
  const int gw = fine ? row_grid(s->num_sms, A.n, A.W, A.U)
                      : row_grid_blocks(s->num_sms, A.n, A.W, kCoarseMinBlocks);
  const double bytes = spmv_class_bytes(A, 8 + 2 * (int)sizeof(MT) + 5 * (int)sizeof(VT));
  auto step = [&](const VT *zin, VT *zout, int k) -> sph_rt_status {
    int *wf = fine ? timing_begin(s) : nullptr;
    if (fine)
      SPH_DISPATCH_SHAPE(A.W, A.U,
                         (pdl_launch(s, fine_cheb_step_kernel<W, U, MT, VT>, gw, kBlock, 0,
                             A, r, zin, zout, d, cf, k, sc, wf)));
    else
      SPH_DISPATCH_SHAPE(A.W, A.U,
                         (pdl_launch(s, cheb_step_kernel<W, U, MT, VT>, gw, kBlock, 0,
                             A, r, zin, zout, d, cf, k, sc, wf)));
    SPH_LAUNCHED(s);
    if (fine) timing_end(s, bytes, kTimedCheb);
    return SPH_RT_OK;
  };
  // ping-pong between z and tmp so that the last write lands in z
  VT *bufs[2] = {z, tmp};
  // `degree` writes in all (the init or first step, then degree-1 steps); the
  // first goes to bufs[w0], each later one flips buffers, the last hits bufs[0].
  int w0 = (degree - 1) % 2;
  sph_rt_status rc;
  if (first_step_done) {
    // the caller has made step 0 from a nonzero guess, result in bufs[w0]
  } else if (zero_guess) {
    pdl_launch(s, cheb_init_zero_kernel<MT, VT>, g, kBlock, 0, A.n, r, A.invdiag, cf, d,
                                                                 bufs[w0], sc);
    SPH_LAUNCHED(s);
  } else {
    // the guess is read from bufs[w0 ^ 1]
    if (w0 == 0) {
      SPH_CUDA(s, cudaMemcpyAsync(tmp, z, sizeof(VT) * A.n, cudaMemcpyDeviceToDevice, s->stream));
    }
    if ((rc = step(bufs[w0 ^ 1], bufs[w0], 0))) return rc;
  }
  int at = w0;
  for (int k = 1; k < degree; ++k) {
    if ((rc = step(bufs[at], bufs[at ^ 1], k))) return rc;
    at ^= 1;
  }
  return SPH_RT_OK;
}

template sph_rt_status cheb_apply<double, double>(sph_rt *, const CsrView<double> &, const double *,
                                                  double *, double *, double *, int,
                                                  const ChebCoef *, bool, const Scalars *, bool);
template sph_rt_status cheb_apply<float, float>(sph_rt *, const CsrView<float> &, const float *,
                                                float *, float *, float *, int, const ChebCoef *,
                                                bool, const Scalars *, bool);

// Preconditioner hooks implemented by the AMG translation unit.  init_done:
// the finest level's smoother start was written by the CG update (amg_fine_init);
// df: fuse the inner product into the last sweep where the V-cycle allows it
// (*dot_done tells whether it did).
sph_rt_status amg_apply(sph_rt *s, const double *r, double *z, const Scalars *sc, bool init_done,
                        const DotFuse *df, bool *dot_done);
sph_rt_status amg_apply_to32(sph_rt *s, const double *r, const Scalars *sc, bool init_done,
                             const DotFuse *df, bool *dot_done);
const float *amg_z32(const sph_rt *s);
bool amg_fine_init(sph_rt *s, FineInit<double> *f64, FineInit<float> *f32);

// The mixed form with the AMG preconditioner widens the V-cycle's FP32 result
// inside the flexible inner product (no z_old copy).
static bool fused_flex(const sph_rt *s) {
  return s->cfg.precision == SPH_RT_MIXED && s->cfg.precond == SPH_RT_PRECOND_AMG;
}

// z = M^{-1} r followed by rho = (r, z) (and beta unless first).  init_done:
// the update kernel has made the AMG finest level's smoother start.
static sph_rt_status precondition(sph_rt *s, const CsrView<double> &A, int first,
                                  bool init_done = false) {
  int g = grid_cap(s, A.n, kBlock);
  sph_rt_status rc;
  switch (s->cfg.precond) {
    case SPH_RT_PRECOND_JACOBI:
      pdl_launch(s, jacobi_dot_kernel, g, kBlock, 0, A.n, s->r, A.invdiag, s->z, first, s->sc,
                                                      s->partials);
      SPH_LAUNCHED(s);
      return SPH_RT_OK;
    case SPH_RT_PRECOND_CHEBYSHEV:
      rc = cheb_apply<double, double>(s, A, s->r, s->z, s->w, s->tmp_n2, s->cfg.cheb_degree,
                                      s->cheb_slots, true, s->sc, false);
      if (rc) return rc;
      break;
    default: {
      const DotFuse df = {first, fused_flex(s) ? 1 : 0, s->r, s->z, s->sc, s->partials};
      bool dot_done = false;
      if (fused_flex(s)) {
        if ((rc = amg_apply_to32(s, s->r, s->sc, init_done, &df, &dot_done))) return rc;
        if (!dot_done) {
          pdl_launch(s, dot_rz_flex32_kernel, g, kBlock, 0, A.n, s->r, amg_z32(s), s->z, first,
                                                             s->sc, s->partials);
          SPH_LAUNCHED(s);
        }
        return SPH_RT_OK;
      }
      if ((rc = amg_apply(s, s->r, s->z, s->sc, init_done, &df, &dot_done))) return rc;
      if (dot_done) return SPH_RT_OK;
      break;
    }
  }
  if (s->cfg.precision == SPH_RT_MIXED) {
    pdl_launch(s, dot_rz_flex_kernel, g, kBlock, 0, A.n, s->r, s->z, s->z_old, first, s->sc,
                                                     s->partials);
    SPH_LAUNCHED(s);
    return SPH_RT_OK;
  }
  pdl_launch(s, dot_rz_kernel<double>, g, kBlock, 0, A.n, s->r, s->z, first, s->sc, s->partials);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

// Plain SpMV y = B x (off-diagonal part plus diagonal), for the autotuner.
template <int W, int U>
__global__ void __launch_bounds__(kBlock, sweep_min_blocks(U))
    spmv_plain_kernel(CsrView<double> A, const double *x, double *y) {
  const int own = tile_own_row<W>(threadIdx.x & 31);
  int64_t r0, r1;
  warp_rows<W>(A.n, r0, r1);
  for (int64_t base = r0; base < r1; base += 32) {
    const int rows = (int)(r1 - base < 32 ? r1 - base : 32);
    const int64_t i = base + own;
    const double s = tile_row_sums<W, U, double, double>(base, rows, A.ptr, A.col, A.val, x);
    if (own < rows) y[i] = A.diag[i] * x[i] + s;
  }
}

// Autotuner: time every supported row-group shape on the fine operator
// (3 launches each after one warm-up, CUDA events on the library stream) and
// keep the fastest for all fine-level SpMV-class kernels of this particle set.
sph_rt_status autotune_fine_shape(sph_rt *s) {
  if (s->fine_shape_set) return SPH_RT_OK;
  CsrView<double> A = fine_view(s);
  // candidates share W (so the choice cannot change any result bit) and differ in U
  const int W0 = lanes_for_mean(A.n ? (double)A.nnz / A.n : 0.0);
  std::vector<RowShape> cands = {{W0, 4}, {W0, 8}};
  cudaEvent_t e0, e1;
  SPH_CUDA(s, cudaEventCreate(&e0));
  SPH_CUDA(s, cudaEventCreate(&e1));
  RowShape pick = shape_for_mean(A.n ? (double)A.nnz / A.n : 0.0);
  // candidates alternate over 3 rounds of 6 back-to-back launches (the way the
  // solver issues them), on the current E; the smallest round total wins
  std::vector<float> best(cands.size(), 1e30f);
  for (int round = 0; round < 3; ++round) {
    for (size_t ci = 0; ci < cands.size(); ++ci) {
      const RowShape &c = cands[ci];
      const int gw = row_grid(s->num_sms, A.n, c.W, c.U);
      float ms = 0.f;
      for (int rep = 0; rep < 7; ++rep) {
        if (rep == 1) cudaEventRecord(e0, s->stream);
        SPH_DISPATCH_SHAPE(c.W, c.U, (spmv_plain_kernel<W, U><<<gw, kBlock, 0, s->stream>>>(
                                         A, s->E, s->w)));
        SPH_LAUNCHED(s);
      }
      cudaEventRecord(e1, s->stream);
      SPH_CUDA(s, cudaEventSynchronize(e1));
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best[ci]) best[ci] = ms;
    }
  }
  float bm = 1e30f;
  for (size_t ci = 0; ci < cands.size(); ++ci)
    if (best[ci] < bm) {
      bm = best[ci];
      pick = cands[ci];
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s->fine_shape = pick;
  s->fine_shape_set = true;
  s->fine_shape_n = s->n_int;
  s->fine_shape_nnz = s->nnz_mat;
  return SPH_RT_OK;
}

// ---------------------------------------------------------------------------
// CG with the V-cycle's product (config.fine_post_smooth = 0; the V-cycle and
// the last sweep that yields z, B z and the CG scalars are in amg.cu,
// fcg_cycle).  The iterate x and the right-hand side b are FP64; the other
// vectors are in the hierarchy's precision T (FP64, or FP32 in the mixed form).
// Per iteration: fcg_update_kernel (directions, x, r, ||r||, the smoother start
// of the next V-cycle), [mixed: fcg_resid_kernel when a residual replacement
// is due], then the V-cycle.
//
// Mixed form.  The FP32 operator and vectors make the recursive residual r
// drift from the true one b - B x, by about the FP32 rounding of the residual
// sizes since it was last exact.  So the FP64 residual replaces r (a reliable
// update, Sleijpen & van der Vorst 1996) whenever ||r|| has dropped by the
// factor reliable_drop since the last replacement, and before convergence is
// accepted: the solve stops only on the FP64 residual, ||b - A x||_2 <= tol ||b||_2,
// the same test as the FP64 form.  The search direction is kept.
// ---------------------------------------------------------------------------
bool fcg_active(const sph_rt *s);
sph_rt_status fcg_vectors(sph_rt *s, FcgVecs *v);
sph_rt_status fcg_cycle(sph_rt *s, const FcgVecs &v, int first);

// r = b - B x in FP64 (stored in T), the smoother start zpre = c0 D^{-1} r,
// ||r / V||^2 and the convergence test.  gated: a reliable update, run only
// when the last update asked for one (sc->ru); it also keeps B x in y (mixed
// form), valid for the next solve's start if this replacement ends the solve.
// Else the start of a solve, skipped when that B x is valid (fcg_start_y_kernel
// starts from it instead).
template <int W, int U, typename T>
__global__ void __launch_bounds__(kBlock, sweep_min_blocks(U))
    fcg_resid_kernel(CsrView<double> A, const double *b, const double *x, T *r, T *zpre,
                     const T *invdiag, const ChebCoef *cf, const double *invV, int gated,
                     double *y, Scalars *sc, double *partials, int *wflag) {
  pdl_wait();
  if (gated ? (sc->done || !sc->ru) : sc->yvalid) {
    mark_work(wflag, 0);
    return;
  }
  mark_work(wflag, 1);
  const double c0 = cf->inv_theta;
  const int own = tile_own_row<W>(threadIdx.x & 31);
  int64_t r0, r1;
  warp_rows<W>(A.n, r0, r1);
  double acc = 0.0;
  for (int64_t base = r0; base < r1; base += 32) {
    const int rows = (int)(r1 - base < 32 ? r1 - base : 32);
    const int64_t i = base + own;
    const double s = tile_row_sums<W, U, double, double>(base, rows, A.ptr, A.col, A.val, x);
    if (own < rows) {
      const double bx = fmadd(A.diag[i], x[i], s);
      const double ri = b[i] - bx;
      const T rt = (T)ri;
      r[i] = rt;
      zpre[i] = (T)(c0 * (double)invdiag[i] * (double)rt);
      if (y) y[i] = bx;
      const double ru = ri * invV[i];
      acc += ru * ru;
    }
  }
  __shared__ double sh[32];
  acc = block_sum(acc, sh);
  double part[1] = {acc}, out[1];
  const bool mx[1] = {false};
  if (last_block_combine<1>(part, partials, &sc->counter, out, mx) && threadIdx.x == 0) {
    sc->rnorm2 = out[0];
    sc->rmax2 = out[0];
    sc->ru = 0;
    if (!gated) sc->iters = 0;
    sc->done = !(out[0] > sc->thresh2);  // also stops on NaN
    if (!(out[0] == out[0])) sc->breakdown = 1;
    sc->yvalid = gated && y && sc->done && !sc->breakdown;
  }
}

// Start of a solve from the kept B x (mixed form, after a solve that ended on a
// verified residual at the same x and operator): r = b - y, with the same
// smoother start, norm and test as fcg_resid_kernel.  Skipped otherwise.
template <typename T>
__global__ void fcg_start_y_kernel(int64_t n, const double *b, const double *y, T *r, T *zpre,
                                   const T *invdiag, const ChebCoef *cf, const double *invV,
                                   Scalars *sc, double *partials) {
  pdl_wait();
  if (!sc->yvalid) return;
  const double c0 = cf->inv_theta;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = b[i] - y[i];
    const T rt = (T)ri;
    r[i] = rt;
    zpre[i] = (T)(c0 * (double)invdiag[i] * (double)rt);
    const double ru = ri * invV[i];
    acc += ru * ru;
  }
  __shared__ double sh[32];
  acc = block_sum(acc, sh);
  double part[1] = {acc}, out[1];
  const bool mx[1] = {false};
  if (last_block_combine<1>(part, partials, &sc->counter, out, mx) && threadIdx.x == 0) {
    sc->rnorm2 = out[0];
    sc->rmax2 = out[0];
    sc->ru = 0;
    sc->iters = 0;
    sc->done = !(out[0] > sc->thresh2);
    if (!(out[0] == out[0])) sc->breakdown = 1;
    sc->yvalid = 0;
  }
}

// p = z + beta p, q = B z + beta q (p = z, q = B z when starting), x += alpha p,
// r -= alpha q, ||r / V||^2, the next smoother start zpre = c0 D^{-1} r, and the
// convergence test (FP64 form) or the reliable-update request (mixed form:
// drop2 = reliable_drop^2 > 0).
template <typename T>
__global__ void fcg_update_kernel(int64_t n, double *x, T *r, T *p, T *q, const T *z, const T *w,
                                  T *zpre, const T *invdiag, const ChebCoef *cf,
                                  const double *invV, int maxit, double drop2, Scalars *sc,
                                  double *partials) {
  pdl_wait();
  if (sc->done) return;
  const double alpha = sc->alpha;
  const T beta = (T)sc->beta, ta = (T)alpha;
  const bool first = sc->pfirst != 0;
  const double c0 = cf->inv_theta;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T zi = z[i], wi = w[i];
    const T pi = first ? zi : fmadd(beta, p[i], zi);
    const T qi = first ? wi : fmadd(beta, q[i], wi);
    p[i] = pi;
    q[i] = qi;
    x[i] += alpha * (double)pi;
    const T ri = r[i] - ta * qi;
    r[i] = ri;
    zpre[i] = (T)(c0 * (double)invdiag[i] * (double)ri);
    const double ru = (double)ri * invV[i];
    acc += ru * ru;
  }
  __shared__ double sh[32];
  acc = block_sum(acc, sh);
  double part[1] = {acc}, out[1];
  const bool mx[1] = {false};
  if (last_block_combine<1>(part, partials, &sc->counter, out, mx) && threadIdx.x == 0) {
    const double rn = out[0];
    sc->rnorm2 = rn;
    sc->iters += 1;
    sc->pfirst = 0;
    if (!(rn == rn)) {
      sc->breakdown = 1;
      sc->done = 1;
    } else if (drop2 <= 0.0) {  // FP64: the recursive residual is the residual
      if (!(rn > sc->thresh2) || sc->iters >= maxit) sc->done = 1;
    } else {
      if (rn > sc->rmax2) sc->rmax2 = rn;
      if (!(rn > sc->thresh2) || rn < drop2 * sc->rmax2) sc->ru = 1;
      if (sc->iters >= maxit) {
        // stop unverified: report at least the threshold so the solve is not
        // taken as converged
        sc->done = 1;
        if (!(sc->rnorm2 > sc->thresh2)) sc->rnorm2 = 4.0 * sc->thresh2 + 1e-300;
      }
    }
  }
}

static sph_rt_status fcg_resid_launch(sph_rt *s, const FcgVecs &v, int gated) {
  CsrView<double> A = fine_view(s);
  const int gw = row_grid(s->num_sms, A.n, A.W, A.U);
  const bool mixed = s->cfg.precision == SPH_RT_MIXED;
  // the mixed form keeps B x of its replacements in w (its CG vectors are FP32)
  double *y = mixed && gated ? s->w : nullptr;
  int *wf = timing_begin(s);
  if (mixed)
    SPH_DISPATCH_SHAPE(A.W, A.U,
                       (pdl_launch(s, fcg_resid_kernel<W, U, float>, gw, kBlock, 0, A, s->b,
                                   s->x, v.f32.r, v.f32.zpre, v.f32.invdiag, v.cf, s->invV, gated,
                                   y, s->sc, s->partials, wf)));
  else
    SPH_DISPATCH_SHAPE(A.W, A.U,
                       (pdl_launch(s, fcg_resid_kernel<W, U, double>, gw, kBlock, 0, A, s->b,
                                   s->x, v.f64.r, v.f64.zpre, v.f64.invdiag, v.cf, s->invV, gated,
                                   y, s->sc, s->partials, wf)));
  SPH_LAUNCHED(s);
  // rowptr, diag, b, x, 1/V, r, zpre, 1/diag (+ y)
  const double tb = mixed ? 4.0 : 8.0;
  timing_end(s, spmv_class_bytes(A, 40 + (int)(3 * tb) + (y ? 8 : 0)), kTimedTrueResid);
  if (mixed && !gated) {
    pdl_launch(s, fcg_start_y_kernel<float>, grid_cap(s, A.n, kBlock), kBlock, 0, A.n, s->b,
               (const double *)s->w, v.f32.r, v.f32.zpre, v.f32.invdiag, v.cf, s->invV, s->sc,
               s->partials);
    SPH_LAUNCHED(s);
  }
  return SPH_RT_OK;
}

static sph_rt_status fcg_prologue(sph_rt *s) {
  FcgVecs v;
  sph_rt_status rc;
  if ((rc = fcg_vectors(s, &v))) return rc;
  if ((rc = fcg_resid_launch(s, v, 0))) return rc;
  return fcg_cycle(s, v, 1);
}

static sph_rt_status fcg_iteration(sph_rt *s) {
  FcgVecs v;
  sph_rt_status rc;
  if ((rc = fcg_vectors(s, &v))) return rc;
  const int64_t n = s->n_int;
  const int g = grid_cap(s, n, kBlock);
  if (s->cfg.precision == SPH_RT_MIXED) {
    const double drop2 = s->cfg.reliable_drop * s->cfg.reliable_drop;
    const FcgSet<float> &f = v.f32;
    pdl_launch(s, fcg_update_kernel<float>, g, kBlock, 0, n, s->x, f.r, f.p, f.q,
               (const float *)f.z, (const float *)f.w, f.zpre, f.invdiag, v.cf,
               (const double *)s->invV, s->cfg.max_krylov, drop2, s->sc, s->partials);
    SPH_LAUNCHED(s);
    if ((rc = fcg_resid_launch(s, v, 1))) return rc;
  } else {
    const FcgSet<double> &f = v.f64;
    pdl_launch(s, fcg_update_kernel<double>, g, kBlock, 0, n, s->x, f.r, f.p, f.q,
               (const double *)f.z, (const double *)f.w, f.zpre, f.invdiag, v.cf,
               (const double *)s->invV, s->cfg.max_krylov, 0.0, s->sc, s->partials);
    SPH_LAUNCHED(s);
  }
  return fcg_cycle(s, v, 0);
}

// Solve B x = b from the warm start in x (row a6).  On return the host mirror
// s->sc_host holds the final scalars.
// First part of a solve: r = b - B x, z = M^{-1} r, q = B p with p = z.
sph_rt_status pcg_prologue(sph_rt *s) {
  if (fcg_active(s)) return fcg_prologue(s);
  CsrView<double> A = fine_view(s);
  const int gw = row_grid(s->num_sms, A.n, A.W, A.U);
  sph_rt_status rc;
  int *wf = timing_begin(s);
  SPH_DISPATCH_SHAPE(A.W, A.U,
                     (pdl_launch(s, resid_kernel<W, U>, gw, kBlock, 0, A, s->b, s->x, s->r,
                                                                       s->invV, s->sc,
                                                                       s->partials, wf)));
  SPH_LAUNCHED(s);
  timing_end(s, spmv_class_bytes(A, kRowBytesResid), kTimedResid);
  if ((rc = precondition(s, A, 1))) return rc;
  wf = timing_begin(s);
  SPH_DISPATCH_SHAPE(A.W, A.U,
                     (pdl_launch(s, spmv_pq_kernel<W, U>, gw, kBlock, 0, A, s->z, s->q, s->p, 1,
                                                                         s->sc, s->partials, wf)));
  SPH_LAUNCHED(s);
  timing_end(s, spmv_class_bytes(A, kRowBytesSpmvPQ), kTimedSpmvPQ);
  return SPH_RT_OK;
}

__global__ void copy_vec_kernel(int64_t n, const double *src, double *dst, const Scalars *sc) {
  pdl_wait();
  if (sc && sc->done) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// One CG iteration: x, r update and the convergence test, z = M^{-1} r, the
// new direction and q = B p.  The flexible (mixed-precision) variant keeps the
// previous z in z_old (with the AMG preconditioner: in z itself until the fused
// inner product widens the new one).  All launches are empty once `done` is set.
sph_rt_status pcg_iteration(sph_rt *s) {
  if (fcg_active(s)) return fcg_iteration(s);
  CsrView<double> A = fine_view(s);
  const int gw = row_grid(s->num_sms, A.n, A.W, A.U);
  const int g = grid_cap(s, A.n, kBlock);
  sph_rt_status rc;
  FineInit<double> f64 = {};
  FineInit<float> f32 = {};
  const bool init = s->cfg.precond == SPH_RT_PRECOND_AMG && amg_fine_init(s, &f64, &f32);
  if (f32.d)
    pdl_launch(s, update_kernel<float>, g, kBlock, 0, A.n, s->x, s->r, s->p, s->q, s->invV,
                                                      s->cfg.max_krylov, s->sc, s->partials, f32);
  else
    pdl_launch(s, update_kernel<double>, g, kBlock, 0, A.n, s->x, s->r, s->p, s->q, s->invV,
                                                       s->cfg.max_krylov, s->sc, s->partials, f64);
  SPH_LAUNCHED(s);
  if (s->cfg.precision == SPH_RT_MIXED && !fused_flex(s)) {
    pdl_launch(s, copy_vec_kernel, g, kBlock, 0, A.n, s->z, s->z_old, s->sc);
    SPH_LAUNCHED(s);
  }
  if ((rc = precondition(s, A, 0, init))) return rc;
  int *wf = timing_begin(s);
  SPH_DISPATCH_SHAPE(A.W, A.U,
                     (pdl_launch(s, spmv_pq_kernel<W, U>, gw, kBlock, 0, A, s->z, s->q, s->p, 0,
                                                                         s->sc, s->partials, wf)));
  SPH_LAUNCHED(s);
  timing_end(s, spmv_class_bytes(A, kRowBytesSpmvPQ), kTimedSpmvPQ);
  return SPH_RT_OK;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Holds the stream until the host has written `epoch` (or 2 s have passed,
// which only marks the timing as suspect).
__global__ void gate_kernel(const volatile int *flag, int epoch, Scalars *sc) {
  const unsigned long long t0 = global_ns();
  while (*flag < epoch) {
    if (global_ns() - t0 > 2000000000ull) {
      sc->gate_timeout = 1;
      return;
    }
    __nanosleep(2000);
  }
}

// With kernel timing: hold the stream (gate_begin) while a chunk is queued,
// release it (gate_end) once the chunk is complete.
static sph_rt_status gate_begin(sph_rt *s) {
  if (!s->cfg.kernel_timing) return SPH_RT_OK;
  if (!s->gate_host) {
    int *h = nullptr;
    SPH_CUDA(s, cudaHostAlloc(&h, sizeof(int), cudaHostAllocMapped));
    *h = 0;
    SPH_CUDA(s, cudaHostGetDevicePointer(&s->gate_dev, h, 0));
    s->gate_host = h;
    s->gate_epoch = 0;
  }
  ++s->gate_epoch;
  gate_kernel<<<1, 1, 0, s->stream>>>(s->gate_dev, s->gate_epoch, s->sc);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}
static void gate_end(sph_rt *s) {
  if (s->gate_host) *s->gate_host = s->gate_epoch;
}

// Host-driven solve: iterations are queued in chunks of check_every and the
// device flag is read after each chunk.
sph_rt_status pcg_solve(sph_rt *s, int *iters, bool *converged) {
  sph_rt_status rc;
  if ((rc = gate_begin(s))) return rc;
  if ((rc = pcg_prologue(s))) return rc;
  const int chunk = s->cfg.check_every > 0 ? s->cfg.check_every : 1;
  int queued = 0;
  for (;;) {
    if (queued > 0 && (rc = gate_begin(s))) return rc;
    for (int c = 0; c < chunk; ++c) {
      if ((rc = pcg_iteration(s))) return rc;
      ++queued;
    }
    gate_end(s);
    SPH_CUDA(s, cudaMemcpyAsync(s->sc_host, s->sc, sizeof(Scalars), cudaMemcpyDeviceToHost,
                                s->stream));
    SPH_CUDA(s, cudaStreamSynchronize(s->stream));
    SPH_TRACE("pcg: queued=%d iters=%d done=%d breakdown=%d rnorm2=%g", queued,
              s->sc_host->iters, s->sc_host->done, s->sc_host->breakdown, s->sc_host->rnorm2);
    if (s->sc_host->done || queued > s->cfg.max_krylov + chunk) break;
  }
  timing_flush(s);
  *iters = s->sc_host->iters;
  *converged = !s->sc_host->breakdown && !(s->sc_host->rnorm2 > s->sc_host->thresh2);
  return SPH_RT_OK;
}

// Chebyshev coefficient slots from device Gershgorin bounds g (no host read):
// mode 0: [1 - g, 1 + g] (fine-level Chebyshev preconditioner);
// mode 1: [(1 + g) / 8, 1 + g] (AMG smoother);
// mode 2: [max(1 - g, 1e-3 (1 + g)), 1 + g] (coarsest-level solve).
struct SlotSpec {
  int count;
  int mode[kChebSlots], degree[kChebSlots];
};
__global__ void cheb_slots_kernel(ChebCoef *slots, const double *gersh, const SlotSpec spec) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= spec.count) return;
  const double g = gersh[t], hi = 1.0 + g;
  double lo = 1.0 - g;
  if (spec.mode[t] == 1) lo = hi / 8.0;
  if (spec.mode[t] == 2 && lo < 1e-3 * hi) lo = 1e-3 * hi;
  cheb_coefficients(spec.degree[t], lo, hi, slots + t);
}

// Fill slots first .. first + mode.size() - 1 from the device bounds
// gersh_dev[0 ..]; mode[k] and degree[k] describe slot first + k.
sph_rt_status launch_cheb_slots(sph_rt *s, int first, const double *gersh_dev,
                                const std::vector<int> &mode, const std::vector<int> &degree) {
  SlotSpec spec;
  spec.count = (int)mode.size();
  if (spec.count == 0) return SPH_RT_OK;
  if (first + spec.count > kChebSlots)
    return set_error(s, SPH_RT_EINVAL, "too many Chebyshev slots");
  for (int k = 0; k < spec.count; ++k) {
    spec.mode[k] = mode[k];
    spec.degree[k] = degree[k];
  }
  cheb_slots_kernel<<<1, 64, 0, s->stream>>>(s->cheb_slots + first, gersh_dev, spec);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

}  // namespace sphrt
