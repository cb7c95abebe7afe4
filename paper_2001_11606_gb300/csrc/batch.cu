// batch.cu -- many small problems advanced by ONE kernel launch per time step.
//
// The serving stream is dominated in count by small problems (a few thousand
// particles), for which the per-kernel launch and host-synchronisation costs
// of the single-problem path exceed the work.  Here K problems are packed into
// one block-diagonal data set and a persistent kernel gives each problem one
// thread block, which runs the whole time step of Alg. 1 for its problem:
// material data, assembly, the initial material solve, and the outer loop of
// {right-hand side, preconditioned CG, material solve, convergence test}.
// Every reduction is a block reduction in shared memory (fixed order), every
// phase ends at a __syncthreads(), and every loop is bounded by the
// configured iteration limits, so a launch always ends.  A problem that
// converges stops (its block exits its loop) while the others go on: the
// per-problem convergence masks of the batched form.
//
// Preconditioner: Chebyshev polynomial of degree cheb_degree on D^{-1} B over
// the Gershgorin interval of each problem's operator (no coarse levels inside
// a block).  Problems keep the single-problem layout (interior slots first,
// then ghosts) inside their own slot range of the packed arrays.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"

namespace sphrt {

struct BatchView {
  int K;
  const int64_t *slot_off;  // [K+1]
  const int64_t *n_int;     // [K]
  const double *px, *py, *pz, *V, *invV, *rho, *sigma0;
  const int32_t *kind, *copysrc;  // copysrc holds packed slots
  double *e, *E;
  const double *Qe, *QE;  // packed slot order (interior entries used)
  const int64_t *nbr_ptr;  // [n_all + 1], ghost rows empty
  const int32_t *nbr_col;
  const double *nbr_F;
  const int64_t *mat_ptr;
  const int32_t *mat_col;
  const double *mat_G;
  double *mat_val;
  const int64_t *gh_ptr;
  const int32_t *gh_slot;
  const double *gh_W;
  double *T, *sigma, *f, *R, *lam, *D, *diag, *invdiag, *gb, *b, *x, *r, *z, *p, *q, *d, *t;
  double *e_old, *E_old, *e_l, *E_l, *e_new;
  int32_t *status;   // [K] 0 ok, -3 not converged
  int32_t *outer;    // [K]
  int32_t *krylov;   // [K] total Krylov iterations of the step
  double *energy;    // [K*4] before, after, source, boundary
  const int32_t *run_status;  // [K] multi-step run: nonzero = failed earlier, skip (or NULL)
};

struct BatchPhys {
  double a, c, cv, p, T_floor, larsen_k, dt, tol_inner, tol_outer_e, tol_outer_E, tol_krylov;
  int limiter, max_inner, max_outer, max_krylov, cheb_degree;
};

__device__ __forceinline__ double b_opacity(double sigma0, double Ts, double p) {
  if (p == 0.0) return sigma0;
  if (p == -3.0) return sigma0 / (Ts * Ts * Ts);
  return sigma0 * pow(Ts, p);
}
__device__ __forceinline__ double b_lambda(int limiter, double k, double R) {
  if (limiter == SPH_RT_LIMITER_LEVERMORE) return (2.0 + R) / (6.0 + 3.0 * R + R * R);
  if (limiter == SPH_RT_LIMITER_LARSEN) {
    if (k == 2.0) return 1.0 / sqrt(9.0 + R * R);
    return 1.0 / pow(pow(3.0, k) + pow(R, k), 1.0 / k);
  }
  return 1.0 / 3.0;
}

// block-wide sum / max, result broadcast to every thread
__device__ __forceinline__ double bsum(double v, double *sh, double *bc) {
  double s = block_sum(v, sh);
  if (threadIdx.x == 0) *bc = s;
  __syncthreads();
  double out = *bc;
  __syncthreads();
  return out;
}
__device__ __forceinline__ double bmax(double v, double *sh, double *bc) {
  double s = block_max(v, sh);
  if (threadIdx.x == 0) *bc = s;
  __syncthreads();
  double out = *bc;
  __syncthreads();
  return out;
}

// y = B xin over the block's rows (W lanes per row); mode 0: y = B xin,
// mode 1: y = rhs - B xin.  Ends with __syncthreads.
template <int W, int U>
__device__ void b_spmv(const BatchView &v, int64_t r0, int64_t r1, const double *xin,
                       const double *rhs, double *y, int mode) {
  const int sub = threadIdx.x % W;
  const int grp = threadIdx.x / W, ngrp = blockDim.x / W;
  for (int64_t wb = r0 + warp_first_group<W>(grp); wb < r1; wb += ngrp) {
    const int64_t i = wb + group_in_warp<W>(grp);
    const bool active = i < r1;
    double s = active ? row_dot<W, U>(v.mat_ptr[i], v.mat_ptr[i + 1], v.mat_col, v.mat_val, xin, sub)
                      : 0.0;
    s = row_reduce<W>(s);
    if (active && sub == 0) {
      double bx = v.diag[i] * xin[i] + s;
      y[i] = mode ? rhs[i] - bx : bx;
    }
  }
  __syncthreads();
}

// Chebyshev preconditioner z = p(D^{-1}B) D^{-1} r on [lo, hi], zero guess;
// ping-pong between z and v.t, result in z.  Ends with __syncthreads.
template <int W, int U>
__device__ void b_cheb(const BatchView &v, int64_t r0, int64_t r1, const double *r, double *z,
                       const ChebCoef &cf) {
  const int degree = cf.degree;
  double *buf[2] = {z, v.t};
  int at = (degree - 1) % 2;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    double di = cf.inv_theta * v.invdiag[i] * r[i];
    v.d[i] = di;
    buf[at][i] = di;
  }
  __syncthreads();
  const int sub = threadIdx.x % W;
  const int grp = threadIdx.x / W, ngrp = blockDim.x / W;
  for (int k = 1; k < degree; ++k) {
    const double c1 = cf.c1[k], c2 = cf.c2[k];
    const double *zin = buf[at];
    double *zout = buf[at ^ 1];
    for (int64_t wb = r0 + warp_first_group<W>(grp); wb < r1; wb += ngrp) {
      const int64_t i = wb + group_in_warp<W>(grp);
      const bool active = i < r1;
      double s = active ? row_dot<W, U>(v.mat_ptr[i], v.mat_ptr[i + 1], v.mat_col, v.mat_val, zin,
                                        sub)
                        : 0.0;
      s = row_reduce<W>(s);
      if (active && sub == 0) {
        double res = r[i] - (v.diag[i] * zin[i] + s);
        double di = c1 * v.d[i] + c2 * v.invdiag[i] * res;
        v.d[i] = di;
        zout[i] = zin[i] + di;
      }
    }
    __syncthreads();
    at ^= 1;
  }
}

// num / den computed once and broadcast (one FP64 division per block, not per thread)
__device__ __forceinline__ double bdiv(double num, double den, double *bc) {
  if (threadIdx.x == 0) *bc = num / den;
  __syncthreads();
  double out = *bc;
  __syncthreads();
  return out;
}

template <int W, int U>
__global__ void __launch_bounds__(512) batch_step_kernel(BatchView v, BatchPhys ph) {
  __shared__ double sh[32];
  __shared__ double bc;
  const int k = blockIdx.x;
  if (k >= v.K) return;
  if (v.run_status && v.run_status[k] != 0) return;  // failed in an earlier step of the run
  const int64_t s0 = v.slot_off[k], s1 = v.slot_off[k + 1];
  const int64_t r0 = s0, r1 = s0 + v.n_int[k];
  const int sub = threadIdx.x % W;
  const int grp = threadIdx.x / W, ngrp = blockDim.x / W;

  // energy before
  double ea = 0.0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x)
    ea += v.rho[i] * v.V[i] * v.e[i] + v.V[i] * v.E[i];
  const double energy_before = bsum(ea, sh, &bc);

  // a3: material data from the state at the start of the step
  for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
    if (v.kind[i] == SPH_RT_COPY) continue;
    double Ti = v.e[i] / ph.cv;
    double Ts = Ti > ph.T_floor ? Ti : ph.T_floor;
    double sig = b_opacity(v.sigma0[i], Ts, ph.p);
    v.T[i] = Ti;
    v.sigma[i] = sig;
    v.f[i] = 1.0 / (1.0 + ph.c * sig * ph.dt * 4.0 * ph.a * Ti * Ti * Ti / (v.rho[i] * ph.cv));
    double l0 = b_lambda(ph.limiter, ph.larsen_k, 0.0);
    v.R[i] = 0.0;
    v.lam[i] = l0;
    v.D[i] = ph.c * l0 / sig;
  }
  __syncthreads();
  if (ph.limiter != SPH_RT_LIMITER_NONE) {
    for (int64_t wb = r0 + warp_first_group<W>(grp); wb < r1; wb += ngrp) {
      const int64_t i = wb + group_in_warp<W>(grp);
      const bool active = i < r1;
      const int64_t ia = active ? i : r0;
      double xi = v.px[ia], yi = v.py[ia], zi = v.pz[ia], Ei = v.E[ia];
      double gx = 0.0, gy = 0.0, gz = 0.0;
      const int64_t kb = active ? v.nbr_ptr[i] : 0, ke = active ? v.nbr_ptr[i + 1] : 0;
      for (int64_t kk = kb + sub; kk < ke; kk += W) {
        int32_t j = v.nbr_col[kk];
        int32_t js = v.kind[j] == SPH_RT_COPY ? v.copysrc[j] : j;
        double s = v.V[j] * (v.E[js] - Ei) * v.nbr_F[kk];
        gx += s * (xi - v.px[j]);
        gy += s * (yi - v.py[j]);
        gz += s * (zi - v.pz[j]);
      }
      gx = row_reduce<W>(gx);
      gy = row_reduce<W>(gy);
      gz = row_reduce<W>(gz);
      if (active && sub == 0) {
        double gn = sqrt(gx * gx + gy * gy + gz * gz);
        double Es = Ei > 1e-300 ? Ei : 1e-300;
        double Ri = gn / (v.sigma[i] * Es);
        double l = b_lambda(ph.limiter, ph.larsen_k, Ri);
        v.R[i] = Ri;
        v.lam[i] = l;
        v.D[i] = ph.c * l / v.sigma[i];
      }
    }
    __syncthreads();
  }
  for (int64_t i = r1 + threadIdx.x; i < s1; i += blockDim.x) {
    int32_t c = v.copysrc[i];
    if (c < 0) continue;
    v.T[i] = v.T[c];
    v.sigma[i] = v.sigma[c];
    v.f[i] = v.f[c];
    v.R[i] = v.R[c];
    v.lam[i] = v.lam[c];
    v.D[i] = v.D[c];
  }
  __syncthreads();

  // a4: operator values, diagonal, Dirichlet coupling, Gershgorin bound
  double gmax = 0.0;
  for (int64_t wb = r0 + warp_first_group<W>(grp); wb < r1; wb += ngrp) {
    const int64_t i = wb + group_in_warp<W>(grp);
    const bool active = i < r1;
    double Di = active ? v.D[i] : 0.0, off = 0.0;
    const int64_t mb = active ? v.mat_ptr[i] : 0, me = active ? v.mat_ptr[i + 1] : 0;
    for (int64_t kk = mb + sub; kk < me; kk += W) {
      double val = v.mat_G[kk] * (Di + v.D[v.mat_col[kk]]);
      v.mat_val[kk] = val;
      off += val;
    }
    double wsum = 0.0, gbs = 0.0;
    const int64_t hb = active ? v.gh_ptr[i] : 0, he = active ? v.gh_ptr[i + 1] : 0;
    for (int64_t kk = hb + sub; kk < he; kk += W) {
      int32_t j = v.gh_slot[kk];
      double wk = -v.gh_W[kk] * (Di + v.D[j]);
      wsum += wk;
      gbs += wk * v.E[j];
    }
    off = row_reduce<W>(off);
    wsum = row_reduce<W>(wsum);
    gbs = row_reduce<W>(gbs);
    if (active && sub == 0) {
      double dd = v.V[i] * (1.0 / ph.dt + ph.c * v.sigma[i] * v.f[i] + wsum) - off;
      v.diag[i] = dd;
      v.invdiag[i] = 1.0 / dd;
      v.gb[i] = gbs;
      gmax = fmax(gmax, -off / dd);
    }
  }
  const double gersh = bmax(gmax, sh, &bc);
  __shared__ ChebCoef cf;
  if (threadIdx.x == 0) cheb_coefficients(ph.cheb_degree, 1.0 - gersh, 1.0 + gersh, &cf);
  __syncthreads();

  // Alg. 1: e^{n,0} = e^{n-1}, E^{n,0} = E^{n-1}, material solve with E^{n,0}
  auto newton = [&](const double *E_new, const double *E_prev, const double *e_start,
                    double *e_out, double &ce, double &cE) {
    double mce = 0.0, mcE = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      double cs = ph.c * v.sigma[i];
      double P = cs * E_new[i] + v.Qe[i];
      double rdt = v.rho[i] / ph.dt, eo = v.e_old[i], e0 = e_start[i], ei = e0;
      for (int it = 0; it < ph.max_inner; ++it) {
        double T = ei / ph.cv, T3 = T * T * T;
        double u = rdt * (ei - eo) + cs * ph.a * T3 * T - P;
        double J = rdt + 4.0 * cs * ph.a * T3 / ph.cv;
        double de = u / J;
        ei -= de;
        if (fabs(de) <= ph.tol_inner * fabs(ei)) break;
      }
      e_out[i] = ei;
      mce = fmax(mce, fabs(ei - e0) / fmax(fabs(ei), 1e-300));
      mcE = fmax(mcE, fabs(E_new[i] - E_prev[i]) / fmax(fabs(E_new[i]), 1e-300));
    }
    ce = bmax(mce, sh, &bc);
    cE = bmax(mcE, sh, &bc);
  };
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    v.e_old[i] = v.e[i];
    v.E_old[i] = v.E[i];
    v.E_l[i] = v.E[i];
  }
  __syncthreads();
  double ce = 0.0, cE = 0.0;
  newton(v.E_l, v.E_l, v.e_old, v.e_l, ce, cE);

  int outer = 0, kry_total = 0, status = -3;
  while (outer < ph.max_outer) {
    // a7: right-hand side (B-scaled), warm start, ||b||
    double bb = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      double Tl = v.e_l[i] / ph.cv;
      double cs = ph.c * v.sigma[i];
      double bi = v.E_old[i] / ph.dt + cs * ph.a * Tl * Tl * Tl * Tl - (1.0 - v.f[i]) * cs * v.E_l[i] +
                  v.QE[i] + v.gb[i];
      v.b[i] = v.V[i] * bi;
      v.x[i] = v.E_l[i];
      bb += bi * bi;
    }
    const double thresh2 = ph.tol_krylov * ph.tol_krylov * bsum(bb, sh, &bc);
    // a6: Chebyshev-preconditioned CG on B
    b_spmv<W, U>(v, r0, r1, v.x, v.b, v.r, 1);
    double rr = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      double ru = v.r[i] * v.invV[i];
      rr += ru * ru;
    }
    rr = bsum(rr, sh, &bc);
    int it = 0;
    bool kconv = rr <= thresh2;
    if (!kconv) {
      b_cheb<W, U>(v, r0, r1, v.r, v.z, cf);
      double rz = 0.0;
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        v.p[i] = v.z[i];
        rz += v.r[i] * v.z[i];
      }
      double rho_k = bsum(rz, sh, &bc);
      b_spmv<W, U>(v, r0, r1, v.p, nullptr, v.q, 0);
      while (it < ph.max_krylov) {
        double pq = 0.0;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) pq += v.p[i] * v.q[i];
        pq = bsum(pq, sh, &bc);
        if (!(pq > 0.0) || !(pq < 1e308)) break;  // breakdown
        double alpha = bdiv(rho_k, pq, &bc);
        rr = 0.0;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
          v.x[i] += alpha * v.p[i];
          double ri = v.r[i] - alpha * v.q[i];
          v.r[i] = ri;
          double ru = ri * v.invV[i];
          rr += ru * ru;
        }
        rr = bsum(rr, sh, &bc);
        ++it;
        if (rr <= thresh2) {
          kconv = true;
          break;
        }
        b_cheb<W, U>(v, r0, r1, v.r, v.z, cf);
        rz = 0.0;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) rz += v.r[i] * v.z[i];
        double rho_new = bsum(rz, sh, &bc);
        double beta = bdiv(rho_new, rho_k, &bc);
        rho_k = rho_new;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x)
          v.p[i] = v.z[i] + beta * v.p[i];
        __syncthreads();
        b_spmv<W, U>(v, r0, r1, v.p, nullptr, v.q, 0);
      }
    }
    kry_total += it;
    if (!kconv) break;
    // a8 + a9: material solve with the new radiation energy, convergence test
    newton(v.x, v.E_l, v.e_l, v.e_new, ce, cE);
    ++outer;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      v.e_l[i] = v.e_new[i];
      v.E_l[i] = v.x[i];
    }
    __syncthreads();
    if (ce < ph.tol_outer_e && cE < ph.tol_outer_E) {
      status = 0;
      break;
    }
  }
  if (status == 0) {
    double src = 0.0, bnd = 0.0, after = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      v.e[i] = v.e_l[i];
      v.E[i] = v.E_l[i];
      src += v.V[i] * (v.Qe[i] + v.QE[i]);
      double acc = 0.0;
      for (int64_t kk = v.gh_ptr[i]; kk < v.gh_ptr[i + 1]; ++kk) {
        int32_t j = v.gh_slot[kk];
        acc += -v.gh_W[kk] * (v.D[i] + v.D[j]) * (v.E[j] - v.E_l[i]);
      }
      bnd += v.V[i] * acc;
      after += v.rho[i] * v.V[i] * v.e_l[i] + v.V[i] * v.E_l[i];
    }
    __syncthreads();
    for (int64_t i = r1 + threadIdx.x; i < s1; i += blockDim.x) {
      int32_t c = v.copysrc[i];
      if (c < 0) continue;
      v.e[i] = v.e[c];
      v.E[i] = v.E[c];
    }
    src = bsum(src, sh, &bc);
    bnd = bsum(bnd, sh, &bc);
    after = bsum(after, sh, &bc);
    if (threadIdx.x == 0) {
      v.energy[4 * k + 0] = energy_before;
      v.energy[4 * k + 1] = after;
      v.energy[4 * k + 2] = ph.dt * src;
      v.energy[4 * k + 3] = ph.dt * bnd;
    }
  }
  if (threadIdx.x == 0) {
    v.status[k] = status;
    v.outer[k] = outer;
    v.krylov[k] = kry_total;
  }
}

// ---------------------------------------------------------------------------
// host: packing problems into a batch
// ---------------------------------------------------------------------------
// After each step of a multi-step run: per-problem totals; a problem that did
// not converge is marked and skipped by the remaining steps.
__global__ void batch_accumulate_kernel(int K, const int32_t *status, const int32_t *outer,
                                        const int32_t *krylov, int32_t *run_status,
                                        int32_t *run_outer, int32_t *run_krylov) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K || run_status[k] != 0) return;
  run_outer[k] += outer[k];
  run_krylov[k] += krylov[k];
  if (status[k] != 0) run_status[k] = status[k];
}

__global__ void pack_ptr_kernel(const int64_t *ptr_k, int64_t n_int, int64_t n, int64_t nnz_k,
                                int64_t nnz_off, int64_t *ptr_out /* at slot offset */) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n;
       i += (int64_t)gridDim.x * blockDim.x)
    ptr_out[i] = nnz_off + (i <= n_int ? ptr_k[i] : nnz_k);
}
__global__ void offset_i32_kernel(const int32_t *in, int64_t n, int32_t off, int32_t *out,
                                  int keep_negative) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = in[i];
    out[i] = (keep_negative && v < 0) ? v : v + off;
  }
}

}  // namespace sphrt

using namespace sphrt;

struct BatchItem {
  int64_t n = 0, n_int = 0, nnz_nbr = 0, nnz_mat = 0, nnz_gh = 0;
  std::vector<int64_t> slot2caller;
};

struct sph_rt_batch {
  sph_rt *h = nullptr;  // owns the packed device data (allocator, stream)
  sph_rt_config cfg;
  std::vector<BatchItem> items;
  std::vector<sph_rt *> staging;  // per-problem set-up handles until packed
  bool packed = false;
  BatchView view{};
  int64_t *d_slot_off = nullptr, *d_nint = nullptr;
  int32_t *d_status = nullptr, *d_outer = nullptr, *d_krylov = nullptr;
  double *d_energy = nullptr;
  int W = 16, U = 6;
  // multi-step runs (sph_rt_batch_run): accumulators and the captured graph
  int32_t *d_run_status = nullptr, *d_run_outer = nullptr, *d_run_krylov = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  double graph_dt = 0.0;
  int32_t graph_steps = 0;
  int64_t graph_kernels = 0;
};

static void batch_graph_release(sph_rt_batch *B) {
  if (B->graph_exec) cudaGraphExecDestroy(B->graph_exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  B->graph_exec = nullptr;
  B->graph = nullptr;
}

extern "C" sph_rt_status sph_rt_batch_create(const sph_rt_config *cfg, sph_rt_batch **out) {
  if (!cfg || !out) return SPH_RT_EINVAL;
  *out = nullptr;
  sph_rt *h = nullptr;
  sph_rt_status rc = sph_rt_create(cfg, &h);
  if (rc) return rc;
  sph_rt_batch *B = new (std::nothrow) sph_rt_batch();
  if (!B) {
    sph_rt_destroy(h);
    return SPH_RT_ENOMEM;
  }
  B->h = h;
  B->cfg = *cfg;
  *out = B;
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_batch_add(sph_rt_batch *B, int64_t n_total, const double *pos,
                                          const double *mass, const double *rho, const double *h,
                                          const double *sigma0, const int32_t *kind,
                                          const int64_t *copy_of, const double *e0,
                                          const double *E0, int32_t *index) {
  if (!B) return SPH_RT_EINVAL;
  if (B->packed) return set_error(B->h, SPH_RT_ESTATE, "batch already stepped; create a new one");
  sph_rt_config c = B->cfg;
  c.stream = nullptr;
  sph_rt *t = nullptr;
  sph_rt_status rc = sph_rt_create(&c, &t);
  if (rc) return rc;
  // the staging handle runs on the batch's stream once that exists
  rc = sph_rt_set_particles(t, n_total, pos, mass, rho, h, sigma0, kind, copy_of, e0, E0);
  if (rc) {
    set_error(B->h, rc, sph_rt_last_error(t));
    sph_rt_destroy(t);
    return rc;
  }
  BatchItem it;
  it.n = t->n;
  it.n_int = t->n_int;
  it.nnz_nbr = t->nnz_nbr;
  it.nnz_mat = t->nnz_mat;
  it.nnz_gh = t->nnz_gh;
  B->items.push_back(it);
  B->staging.push_back(t);
  if (index) *index = (int32_t)(B->items.size() - 1);
  return SPH_RT_OK;
}

static sph_rt_status batch_pack(sph_rt_batch *B) {
  sph_rt *s = B->h;
  const int K = (int)B->items.size();
  if (K == 0) return set_error(s, SPH_RT_ESTATE, "empty batch");
  if (K > 65535) return set_error(s, SPH_RT_EINVAL, "too many problems in one batch");
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  if (!s->cuda_ready) {
    // the packed handle needs its stream and host mirror
    SPH_CUDA(s, cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
    SPH_CUDA(s, cudaMallocHost(&s->sc_host, sizeof(Scalars)));
    s->cuda_ready = true;
  }
  int64_t n_all = 0, nb = 0, nm = 0, ng = 0;
  std::vector<int64_t> so(K + 1), nint(K), nbo(K), nmo(K), ngo(K);
  for (int k = 0; k < K; ++k) {
    so[k] = n_all;
    nbo[k] = nb;
    nmo[k] = nm;
    ngo[k] = ng;
    n_all += B->items[k].n;
    nb += B->items[k].nnz_nbr;
    nm += B->items[k].nnz_mat;
    ng += B->items[k].nnz_gh;
    nint[k] = B->items[k].n_int;
  }
  so[K] = n_all;
  if (n_all >= ((int64_t)1 << 31) - 1) return set_error(s, SPH_RT_EINVAL, "batch too large");
  BatchView &v = B->view;
  auto D = [&](size_t cnt) { return dalloc<double>(s, cnt); };
  v.K = K;
  double **dd[] = {(double **)&v.px, (double **)&v.py, (double **)&v.pz, (double **)&v.V,
                   (double **)&v.invV, (double **)&v.rho, (double **)&v.sigma0, &v.e, &v.E,
                   (double **)&v.Qe, (double **)&v.QE, &v.T, &v.sigma, &v.f, &v.R, &v.lam, &v.D,
                   &v.diag, &v.invdiag, &v.gb, &v.b, &v.x, &v.r, &v.z, &v.p, &v.q, &v.d, &v.t,
                   &v.e_old, &v.E_old, &v.e_l, &v.E_l, &v.e_new};
  for (double **p : dd)
    if (!(*p = D(n_all))) return SPH_RT_ENOMEM;
  int32_t *kind = dalloc<int32_t>(s, n_all), *copysrc = dalloc<int32_t>(s, n_all);
  int64_t *nbr_ptr = dalloc<int64_t>(s, n_all + 1), *mat_ptr = dalloc<int64_t>(s, n_all + 1),
          *gh_ptr = dalloc<int64_t>(s, n_all + 1);
  int32_t *nbr_col = dalloc<int32_t>(s, nb), *mat_col = dalloc<int32_t>(s, nm),
          *gh_slot = dalloc<int32_t>(s, ng);
  double *nbr_F = D(nb), *mat_G = D(nm), *mat_val = D(nm), *gh_W = D(ng);
  B->d_slot_off = dalloc<int64_t>(s, K + 1);
  B->d_nint = dalloc<int64_t>(s, K);
  B->d_status = dalloc<int32_t>(s, K);
  B->d_outer = dalloc<int32_t>(s, K);
  B->d_krylov = dalloc<int32_t>(s, K);
  B->d_energy = D(4 * (size_t)K);
  if (!kind || !copysrc || !nbr_ptr || !mat_ptr || !gh_ptr || !nbr_col || !mat_col ||
      !gh_slot || !nbr_F || !mat_G || !mat_val || !gh_W || !B->d_slot_off || !B->d_nint ||
      !B->d_status || !B->d_outer || !B->d_krylov || !B->d_energy)
    return SPH_RT_ENOMEM;
  cudaStream_t st = s->stream;
  const auto h2d = cudaMemcpyHostToDevice;
  const auto d2d = cudaMemcpyDeviceToDevice;
  SPH_CUDA(s, cudaMemcpyAsync(B->d_slot_off, so.data(), sizeof(int64_t) * (K + 1), h2d, st));
  SPH_CUDA(s, cudaMemcpyAsync(B->d_nint, nint.data(), sizeof(int64_t) * K, h2d, st));
  SPH_CUDA(s, cudaMemsetAsync((void *)v.Qe, 0, sizeof(double) * n_all, st));
  SPH_CUDA(s, cudaMemsetAsync((void *)v.QE, 0, sizeof(double) * n_all, st));
  for (int k = 0; k < K; ++k) {
    sph_rt *t = B->staging[k];
    SPH_CUDA(s, cudaStreamSynchronize(t->stream));
    const BatchItem &it = B->items[k];
    const int64_t o = so[k], n = it.n;
    const double *srcs[] = {t->px, t->py, t->pz, t->V, t->invV, t->rho, t->sigma0, t->e, t->E};
    double *dsts[] = {(double *)v.px + o, (double *)v.py + o, (double *)v.pz + o,
                      (double *)v.V + o, (double *)v.invV + o, (double *)v.rho + o,
                      (double *)v.sigma0 + o, v.e + o, v.E + o};
    for (int a = 0; a < 9; ++a)
      SPH_CUDA(s, cudaMemcpyAsync(dsts[a], srcs[a], sizeof(double) * n, d2d, st));
    SPH_CUDA(s, cudaMemcpyAsync(kind + o, t->kind, sizeof(int32_t) * n, d2d, st));
    const int g = 64;
    offset_i32_kernel<<<g, kBlock, 0, st>>>(t->copysrc, n, (int32_t)o, copysrc + o, 1);
    SPH_LAUNCHED(s);
    pack_ptr_kernel<<<g, kBlock, 0, st>>>(t->nbr_ptr, it.n_int, n, it.nnz_nbr, nbo[k], nbr_ptr + o);
    SPH_LAUNCHED(s);
    pack_ptr_kernel<<<g, kBlock, 0, st>>>(t->mat_ptr, it.n_int, n, it.nnz_mat, nmo[k], mat_ptr + o);
    SPH_LAUNCHED(s);
    pack_ptr_kernel<<<g, kBlock, 0, st>>>(t->gh_ptr, it.n_int, n, it.nnz_gh, ngo[k], gh_ptr + o);
    SPH_LAUNCHED(s);
    offset_i32_kernel<<<g, kBlock, 0, st>>>(t->nbr_col, it.nnz_nbr, (int32_t)o, nbr_col + nbo[k], 0);
    SPH_LAUNCHED(s);
    offset_i32_kernel<<<g, kBlock, 0, st>>>(t->mat_col, it.nnz_mat, (int32_t)o, mat_col + nmo[k], 0);
    SPH_LAUNCHED(s);
    offset_i32_kernel<<<g, kBlock, 0, st>>>(t->gh_slot, it.nnz_gh, (int32_t)o, gh_slot + ngo[k], 0);
    SPH_LAUNCHED(s);
    if (it.nnz_nbr)
      SPH_CUDA(s, cudaMemcpyAsync(nbr_F + nbo[k], t->nbr_F, sizeof(double) * it.nnz_nbr, d2d, st));
    if (it.nnz_mat)
      SPH_CUDA(s, cudaMemcpyAsync(mat_G + nmo[k], t->mat_G, sizeof(double) * it.nnz_mat, d2d, st));
    if (it.nnz_gh)
      SPH_CUDA(s, cudaMemcpyAsync(gh_W + ngo[k], t->gh_W, sizeof(double) * it.nnz_gh, d2d, st));
    B->items[k].slot2caller.resize(n);
    SPH_CUDA(s, cudaMemcpyAsync(B->items[k].slot2caller.data(), t->slot2caller,
                                sizeof(int64_t) * n, cudaMemcpyDeviceToHost, st));
    SPH_CUDA(s, cudaStreamSynchronize(st));
    sph_rt_destroy(t);
    B->staging[k] = nullptr;
  }
  B->staging.clear();
  v.slot_off = B->d_slot_off;
  v.n_int = B->d_nint;
  v.kind = kind;
  v.copysrc = copysrc;
  v.nbr_ptr = nbr_ptr;
  v.nbr_col = nbr_col;
  v.nbr_F = nbr_F;
  v.mat_ptr = mat_ptr;
  v.mat_col = mat_col;
  v.mat_G = mat_G;
  v.mat_val = mat_val;
  v.gh_ptr = gh_ptr;
  v.gh_slot = gh_slot;
  v.gh_W = gh_W;
  v.status = B->d_status;
  v.outer = B->d_outer;
  v.krylov = B->d_krylov;
  v.energy = B->d_energy;
  int64_t ni_all = 0;
  for (int k = 0; k < K; ++k) ni_all += nint[k];
  RowShape sh = shape_for_mean(ni_all ? (double)nm / (double)ni_all : 0.0);
  B->W = sh.W;
  B->U = sh.U;
  s->n = n_all;
  B->packed = true;
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_batch_set_sources(sph_rt_batch *B, int32_t index,
                                                  const double *Qe, const double *QE) {
  if (!B) return SPH_RT_EINVAL;
  sph_rt_status rc;
  if (!B->packed && (rc = batch_pack(B))) return rc;
  sph_rt *s = B->h;
  if (index < 0 || index >= (int32_t)B->items.size())
    return set_error(s, SPH_RT_EINVAL, "problem index out of range");
  const BatchItem &it = B->items[index];
  int64_t o = 0;
  for (int k = 0; k < index; ++k) o += B->items[k].n;
  std::vector<double> tmp((size_t)it.n);
  const double *src[2] = {Qe, QE};
  double *dst[2] = {(double *)B->view.Qe + o, (double *)B->view.QE + o};
  for (int a = 0; a < 2; ++a) {
    if (!src[a]) {
      SPH_CUDA(s, cudaMemsetAsync(dst[a], 0, sizeof(double) * it.n, s->stream));
      continue;
    }
    for (int64_t i = 0; i < it.n; ++i) {
      double val = src[a][it.slot2caller[i]];
      if (!isfinite(val) && i < it.n_int) return set_error(s, SPH_RT_EINVAL, "non-finite source");
      tmp[i] = val;
    }
    SPH_CUDA(s, cudaMemcpyAsync(dst[a], tmp.data(), sizeof(double) * it.n, cudaMemcpyHostToDevice,
                                s->stream));
    SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  }
  return SPH_RT_OK;
}

static BatchPhys batch_phys(const sph_rt_batch *B, double dt) {
  const sph_rt_config &c = B->h->cfg;
  BatchPhys ph;
  ph.a = c.a;
  ph.c = c.c;
  ph.cv = c.cv;
  ph.p = c.opacity_exp;
  ph.T_floor = c.T_floor;
  ph.larsen_k = c.larsen_k;
  ph.dt = dt;
  ph.tol_inner = c.tol_inner_e;
  ph.tol_outer_e = c.tol_outer_e;
  ph.tol_outer_E = c.tol_outer_E;
  ph.tol_krylov = c.tol_krylov;
  ph.limiter = c.limiter;
  ph.max_inner = c.max_inner_e;
  ph.max_outer = c.max_outer;
  ph.max_krylov = c.max_krylov;
  ph.cheb_degree = c.cheb_degree;
  return ph;
}

static sph_rt_status launch_batch_step(sph_rt_batch *B, const BatchView &v, const BatchPhys &ph) {
  sph_rt *s = B->h;
  if (B->W <= 4)
    batch_step_kernel<4, 8><<<v.K, 512, 0, s->stream>>>(v, ph);
  else
    batch_step_kernel<8, 8><<<v.K, 512, 0, s->stream>>>(v, ph);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_batch_run(sph_rt_batch *B, double dt, int32_t steps,
                                          int32_t *status, int32_t *outer_total,
                                          int32_t *krylov_total) {
  if (!B) return SPH_RT_EINVAL;
  if (!isfinite(dt) || dt <= 0.0) return set_error(B->h, SPH_RT_EINVAL, "dt must be finite and > 0");
  if (steps < 1) return set_error(B->h, SPH_RT_EINVAL, "steps must be >= 1");
  sph_rt_status rc;
  if (!B->packed && (rc = batch_pack(B))) return rc;
  sph_rt *s = B->h;
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  const int K = B->view.K;
  if (!B->d_run_status) {
    B->d_run_status = dalloc<int32_t>(s, K);
    B->d_run_outer = dalloc<int32_t>(s, K);
    B->d_run_krylov = dalloc<int32_t>(s, K);
    if (!B->d_run_status || !B->d_run_outer || !B->d_run_krylov) return SPH_RT_ENOMEM;
  }
  if (!B->graph_exec || B->graph_dt != dt || B->graph_steps != steps) {
    batch_graph_release(B);
    BatchView v = B->view;
    v.run_status = B->d_run_status;
    const BatchPhys ph = batch_phys(B, dt);
    const int64_t l0 = s->launches;
    SPH_CUDA(s, cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeRelaxed));
    auto body = [&]() -> sph_rt_status {
      SPH_CUDA(s, cudaMemsetAsync(B->d_run_status, 0, sizeof(int32_t) * K, s->stream));
      SPH_CUDA(s, cudaMemsetAsync(B->d_run_outer, 0, sizeof(int32_t) * K, s->stream));
      SPH_CUDA(s, cudaMemsetAsync(B->d_run_krylov, 0, sizeof(int32_t) * K, s->stream));
      for (int32_t k = 0; k < steps; ++k) {
        sph_rt_status r2 = launch_batch_step(B, v, ph);
        if (r2) return r2;
        batch_accumulate_kernel<<<(K + 255) / 256, 256, 0, s->stream>>>(
            K, B->d_status, B->d_outer, B->d_krylov, B->d_run_status, B->d_run_outer,
            B->d_run_krylov);
        SPH_LAUNCHED(s);
      }
      return SPH_RT_OK;
    };
    rc = body();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->stream, &g);
    B->graph_kernels = s->launches - l0;
    s->launches = l0;
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) {
      cuda_ok(s, e, "cudaStreamEndCapture");
      return SPH_RT_EDEVICE;
    }
    B->graph = g;
    SPH_CUDA(s, cudaGraphInstantiate(&B->graph_exec, g, 0));
    B->graph_dt = dt;
    B->graph_steps = steps;
  }
  SPH_CUDA(s, cudaGraphLaunch(B->graph_exec, s->stream));
  s->launches += B->graph_kernels;
  std::vector<int32_t> st(K), ou(K), kr(K);
  SPH_CUDA(s, cudaMemcpyAsync(st.data(), B->d_run_status, sizeof(int32_t) * K, cudaMemcpyDeviceToHost, s->stream));
  SPH_CUDA(s, cudaMemcpyAsync(ou.data(), B->d_run_outer, sizeof(int32_t) * K, cudaMemcpyDeviceToHost, s->stream));
  SPH_CUDA(s, cudaMemcpyAsync(kr.data(), B->d_run_krylov, sizeof(int32_t) * K, cudaMemcpyDeviceToHost, s->stream));
  SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  bool all_ok = true;
  for (int k = 0; k < K; ++k) {
    if (status) status[k] = st[k];
    if (outer_total) outer_total[k] = ou[k];
    if (krylov_total) krylov_total[k] = kr[k];
    all_ok = all_ok && st[k] == 0;
  }
  return all_ok ? SPH_RT_OK : set_error(s, SPH_RT_ENOTCONV, "some problems did not converge");
}

extern "C" sph_rt_status sph_rt_batch_step(sph_rt_batch *B, double dt, int32_t *status,
                                           int32_t *outer_iters, int32_t *krylov_iters,
                                           double *energy) {
  if (!B) return SPH_RT_EINVAL;
  if (!isfinite(dt) || dt <= 0.0) return set_error(B->h, SPH_RT_EINVAL, "dt must be finite and > 0");
  sph_rt_status rc;
  if (!B->packed && (rc = batch_pack(B))) return rc;
  sph_rt *s = B->h;
  SPH_CUDA(s, cudaSetDevice(s->cfg.device));
  const int K = B->view.K;
  BatchView v = B->view;
  v.run_status = nullptr;
  // the failed problems keep their state: batch_step_kernel only commits on success
  if ((rc = launch_batch_step(B, v, batch_phys(B, dt)))) return rc;
  std::vector<int32_t> st(K), ou(K), kr(K);
  SPH_CUDA(s, cudaMemcpyAsync(st.data(), B->d_status, sizeof(int32_t) * K, cudaMemcpyDeviceToHost, s->stream));
  SPH_CUDA(s, cudaMemcpyAsync(ou.data(), B->d_outer, sizeof(int32_t) * K, cudaMemcpyDeviceToHost, s->stream));
  SPH_CUDA(s, cudaMemcpyAsync(kr.data(), B->d_krylov, sizeof(int32_t) * K, cudaMemcpyDeviceToHost, s->stream));
  if (energy)
    SPH_CUDA(s, cudaMemcpyAsync(energy, B->d_energy, sizeof(double) * 4 * K, cudaMemcpyDeviceToHost, s->stream));
  SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  bool all_ok = true;
  for (int k = 0; k < K; ++k) {
    if (status) status[k] = st[k];
    if (outer_iters) outer_iters[k] = ou[k];
    if (krylov_iters) krylov_iters[k] = kr[k];
    all_ok = all_ok && st[k] == 0;
  }
  return all_ok ? SPH_RT_OK : set_error(s, SPH_RT_ENOTCONV, "some problems did not converge");
}

extern "C" sph_rt_status sph_rt_batch_get_energies(sph_rt_batch *B, int32_t index, double *e,
                                                   double *E) {
  if (!B) return SPH_RT_EINVAL;
  sph_rt_status rc;
  if (!B->packed && (rc = batch_pack(B))) return rc;
  sph_rt *s = B->h;
  if (index < 0 || index >= (int32_t)B->items.size())
    return set_error(s, SPH_RT_EINVAL, "problem index out of range");
  const BatchItem &it = B->items[index];
  int64_t o = 0;
  for (int k = 0; k < index; ++k) o += B->items[k].n;
  std::vector<double> tmp((size_t)it.n);
  double *outs[2] = {e, E};
  const double *srcs[2] = {B->view.e + o, B->view.E + o};
  for (int a = 0; a < 2; ++a) {
    if (!outs[a]) continue;
    SPH_CUDA(s, cudaMemcpyAsync(tmp.data(), srcs[a], sizeof(double) * it.n, cudaMemcpyDeviceToHost,
                                s->stream));
    SPH_CUDA(s, cudaStreamSynchronize(s->stream));
    for (int64_t i = 0; i < it.n; ++i) outs[a][it.slot2caller[i]] = tmp[i];
  }
  return SPH_RT_OK;
}

extern "C" int32_t sph_rt_batch_size(const sph_rt_batch *B) {
  return B ? (int32_t)B->items.size() : 0;
}

extern "C" const char *sph_rt_batch_last_error(const sph_rt_batch *B) {
  return B ? B->h->err.c_str() : "null batch";
}

extern "C" void sph_rt_batch_destroy(sph_rt_batch *B) {
  if (!B) return;
  if (B->graph_exec || B->graph) {
    cudaSetDevice(B->h->cfg.device);
    batch_graph_release(B);
  }
  for (sph_rt *t : B->staging)
    if (t) sph_rt_destroy(t);
  sph_rt_destroy(B->h);
  delete B;
}
