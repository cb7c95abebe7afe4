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
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

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
  const double *nbr_A;  // [3][nnz_nbr]: F_ij V_j (x_i - x_j), the limiter gradient's weights
  const int64_t *mat_ptr;
  const int32_t *mat_col;
  const double *mat_G;
  double *mat_val;
  const int64_t *gh_ptr;
  const int32_t *gh_slot;
  const double *gh_W;
  double *T, *sigma, *f, *R, *lam, *D, *diag, *invdiag, *gb, *b, *x, *r, *z, *p, *q, *d, *t;
  double *e_old, *E_old, *e_l, *E_l, *e_new;
  double *y;  // B x, kept through the CG updates for the next outer iteration's residual
  int32_t *status;   // [K] 0 ok, -3 not converged
  int32_t *outer;    // [K]
  int32_t *krylov;   // [K] total Krylov iterations of the step
  double *energy;    // [K*4] before, after, source, boundary
  const int32_t *run_status;  // [K] multi-step run: nonzero = failed earlier, skip (or NULL)
  const int32_t *order;       // [K] problem of each cluster of the launch, largest first
  // extrapolated Krylov start: per problem the consecutive converged steps behind
  // the state (capped at 3) and their sizes (newest first); between steps E_old
  // holds E^{n-2}, H0 E^{n-3} and H1 E^{n-4} of the problem's interior rows
  int32_t *hist;     // [K]
  double *dt_hist;   // [3K]
  double *H0, *H1;   // [n_all]
  int64_t nnz_nbr;            // neighbour entries of the whole batch (stride of nbr_A)
};

struct BatchPhys {
  double a, c, cv, inv_cv, p, T_floor, larsen_k, dt, tol_inner, tol_outer_e, tol_outer_E,
      tol_krylov;
  int limiter, max_inner, max_outer, max_krylov, cheb_degree, dim;
  int krylov_start;  // p > 0: first solve from the extrapolation in time of order <= p
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

// ---------------------------------------------------------------------------
// Work split.  A problem runs on the C CTAs of one thread-block cluster (C = 1,
// 2, 4 or 8, by its size): CTA `rank` owns the contiguous interior rows
// [q0, q1) (chunks of a multiple of 32 rows), slot loops are strided over all
// C * blockDim threads of the cluster, and every value another CTA reads is
// published by a cluster barrier (barrier.cluster arrive.release /
// wait.acquire, which orders global as well as shared memory) before it is
// read.  Control flow is uniform over the cluster: every branch depends on
// per-problem data or on cluster-reduced values, which every CTA combines in
// the same order, so all CTAs reach every barrier.
// ---------------------------------------------------------------------------
struct Part {
  int rank, C;
  int64_t s0, s1;  // the problem's slots
  int64_t r0, r1;  // its interior rows
  int64_t q0, q1;  // this CTA's rows
  int64_t ct, cn;  // this thread's index in the cluster, threads in the cluster
};

__device__ __forceinline__ Part make_part(int64_t s0, int64_t s1, int64_t nint, int rank, int C) {
  Part P;
  P.rank = rank;
  P.C = C;
  P.s0 = s0;
  P.s1 = s1;
  P.r0 = s0;
  P.r1 = s0 + nint;
  const int64_t chunk = ((nint + C - 1) / C + 31) / 32 * 32;
  P.q0 = P.r0 + (int64_t)rank * chunk;
  if (P.q0 > P.r1) P.q0 = P.r1;
  P.q1 = P.q0 + chunk;
  if (P.q1 > P.r1) P.q1 = P.r1;
  P.ct = (int64_t)rank * blockDim.x + threadIdx.x;
  P.cn = (int64_t)C * blockDim.x;
  return P;
}

// Cluster reductions: each warp reduces its values, lane 0 stores them in one
// of two CTA buffers, after a CTA barrier thread a combines value a over the
// warps (in warp order) into one of two cluster-visible slots, and after the
// cluster barrier every thread of the cluster reads the C CTA totals in rank
// order (distributed shared memory), so all hold the same fixed-order result.
// The buffers alternate between calls: a buffer is written again two calls
// later, after the barriers of the call between, which every thread reaches
// only after it has read the buffer.  All threads make the same calls.
constexpr int kBRedWarps = 16, kBRedVals = 3;
struct CRed {
  double *wbuf;  // shared, [2][kBRedVals][kBRedWarps]
  double *cbuf;  // shared, [2][kBRedVals], read by the whole cluster
  int par;
};

template <int N>
__device__ __forceinline__ void cred(CRed &R, const Part &P, double (&v)[N],
                                     const bool (&is_max)[N]) {
  static_assert(N <= kBRedVals, "too many values in one reduction");
  cg::cluster_group cl = cg::this_cluster();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int a = 0; a < N; ++a) v[a] = is_max[a] ? warp_max(v[a]) : warp_sum(v[a]);
  double *wb = R.wbuf + R.par * (kBRedVals * kBRedWarps);
  double *cb = R.cbuf + R.par * kBRedVals;
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < N; ++a) wb[a * kBRedWarps + wid] = v[a];
  }
  __syncthreads();
  if (threadIdx.x < N) {
    const int a = threadIdx.x;
    double s = wb[a * kBRedWarps];
    for (int w = 1; w < nw; ++w) {
      const double t = wb[a * kBRedWarps + w];
      s = is_max[a] ? fmax(s, t) : s + t;
    }
    cb[a] = s;
  }
  cl.sync();
#pragma unroll
  for (int a = 0; a < N; ++a) {
    double s = *cl.map_shared_rank(cb + a, 0);
    for (int r = 1; r < P.C; ++r) {
      const double t = *cl.map_shared_rank(cb + a, r);
      s = is_max[a] ? fmax(s, t) : s + t;
    }
    v[a] = s;
  }
  R.par ^= 1;
}
__device__ __forceinline__ double csum(CRed &R, const Part &P, double x) {
  double v[1] = {x};
  const bool m[1] = {false};
  cred<1>(R, P, v, m);
  return v[0];
}
// barrier over the cluster, publishing every earlier write to all its CTAs
__device__ __forceinline__ void csync() { cg::this_cluster().sync(); }

// num / den computed by one thread of each CTA (identical inputs in every CTA
// of the cluster, so identical results) and broadcast with one CTA barrier;
// an FP64 division costs tens of FP64-pipe operations per warp.  Alternating
// slots, as in cred.
__device__ __forceinline__ double bdiv(double num, double den, double *bc, int &par) {
  if (threadIdx.x == 0) bc[par] = num / den;
  __syncthreads();
  const double out = bc[par];
  par ^= 1;
  return out;
}

// Row dot product of the batched kernel: the values and x are written earlier
// in the same launch by other threads, so they are read with plain (coherent)
// loads, not through the read-only path; the columns are read-only.  Same
// order of operations as row_dot.
template <int W, int U>
__device__ __forceinline__ double b_row_dot(int64_t beg, int64_t end, const int32_t *col,
                                            const double *val, const double *x, int sub) {
  double s = 0.0;
  for (int64_t k = beg + sub; k < end; k += (int64_t)W * U) {
    int32_t c[U];
    double a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t kk = k + (int64_t)u * W;
      c[u] = kk < end ? __ldg(col + kk) : -1;
      a[u] = kk < end ? val[kk] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (c[u] >= 0) s = fma(a[u], x[c[u]], s);
  }
  return s;
}

// Operator sweep over this CTA's rows (W lanes per row, U entries in flight
// per lane).  MODE 0: y = B xin, returns this thread's part of (xin, y);
// MODE 1: y = rhs - B xin and bx = B xin, returns its part of ||y / V||^2.
// No barrier at the end: the reduction that follows is the barrier before y
// is read.
template <int W, int U, int MODE>
__device__ __forceinline__ double b_spmv(const BatchView &v, const Part &P, const double *xin,
                                         const double *rhs, double *y, double *bxout = nullptr) {
  const int sub = threadIdx.x % W;
  const int grp = threadIdx.x / W, ngrp = blockDim.x / W;
  double part = 0.0;
  for (int64_t wb = P.q0 + warp_first_group<W>(grp); wb < P.q1; wb += ngrp) {
    const int64_t i = wb + group_in_warp<W>(grp);
    const bool active = i < P.q1;
    double s = active ? b_row_dot<W, U>(v.mat_ptr[i], v.mat_ptr[i + 1], v.mat_col, v.mat_val, xin, sub)
                      : 0.0;
    s = row_reduce<W>(s);
    if (active && sub == 0) {
      const double bx = v.diag[i] * xin[i] + s;
      if (MODE == 0) {
        y[i] = bx;
        part += xin[i] * bx;
      } else {
        const double yi = rhs[i] - bx;
        y[i] = yi;
        bxout[i] = bx;
        const double yu = yi * v.invV[i];
        part += yu * yu;
      }
    }
  }
  return part;
}

// Chebyshev preconditioner z = p(D^{-1}B) D^{-1} r on [lo, hi], zero guess, on
// this CTA's rows; ping-pong between z and v.t, result in z.  Returns this
// thread's part of (r, z); no barrier at the end (the reduction of (r, z) is
// the barrier).
template <int W, int U>
__device__ double b_cheb(const BatchView &v, const Part &P, const double *r, double *z,
                         const ChebCoef &cf) {
  const int degree = cf.degree;
  double *buf[2] = {z, v.t};
  int at = (degree - 1) % 2;
  double rz = 0.0;
  for (int64_t i = P.q0 + threadIdx.x; i < P.q1; i += blockDim.x) {
    const double di = cf.inv_theta * v.invdiag[i] * r[i];
    v.d[i] = di;
    buf[at][i] = di;
    if (degree == 1) rz += r[i] * di;
  }
  const int sub = threadIdx.x % W;
  const int grp = threadIdx.x / W, ngrp = blockDim.x / W;
  for (int k = 1; k < degree; ++k) {
    csync();  // the previous iterate, all rows of the problem
    const double c1 = cf.c1[k], c2 = cf.c2[k];
    const double *zin = buf[at];
    double *zout = buf[at ^ 1];
    const bool last = k == degree - 1;
    for (int64_t wb = P.q0 + warp_first_group<W>(grp); wb < P.q1; wb += ngrp) {
      const int64_t i = wb + group_in_warp<W>(grp);
      const bool active = i < P.q1;
      double s = active ? b_row_dot<W, U>(v.mat_ptr[i], v.mat_ptr[i + 1], v.mat_col, v.mat_val,
                                          zin, sub)
                        : 0.0;
      s = row_reduce<W>(s);
      if (active && sub == 0) {
        const double res = r[i] - (v.diag[i] * zin[i] + s);
        const double di = c1 * v.d[i] + c2 * v.invdiag[i] * res;
        v.d[i] = di;
        const double zi = zin[i] + di;
        zout[i] = zi;
        if (last) rz += r[i] * zi;
      }
    }
    at ^= 1;
  }
  return rz;
}

// MINB resident blocks per SM: 1 leaves the compiler ~128 registers a thread,
// 2 caps it at 64 (a few spilled values in the limiter and opacity code) so
// that twice as many CTAs are in flight; the arithmetic is the same.  Launched
// with a cluster dimension C (1, 2, 4 or 8): cluster c runs problem
// v.order[c] on its C CTAs.
template <int W, int U, int MINB>
__global__ void __launch_bounds__(512, MINB) batch_step_kernel(BatchView v, BatchPhys ph) {
  __shared__ double wred[2 * kBRedVals * kBRedWarps];
  __shared__ double cred_slots[2 * kBRedVals];
  __shared__ double bc[2];
  __shared__ ChebCoef cf;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int cid = blockIdx.x / C;  // clusters are C consecutive blocks
  if (cid >= v.K) return;          // the grid is exactly v.K clusters: never taken
  const int k = v.order[cid];
  if (v.run_status && v.run_status[k] != 0) return;  // failed in an earlier step of the run
  CRed R{wred, cred_slots, 0};
  int bpar = 0;
  const Part P = make_part(v.slot_off[k], v.slot_off[k + 1], v.n_int[k], (int)cl.block_rank(), C);
  const int sub = threadIdx.x % W;
  const int grp = threadIdx.x / W, ngrp = blockDim.x / W;

  // a3: material data from the state at the start of the step (every slot but
  // copy ghosts), energy before; Eg = E at each slot's value source (a copy
  // ghost's interior particle)
  double ea = 0.0;
  for (int64_t i = P.s0 + P.ct; i < P.s1; i += P.cn) {
    const bool copy = v.kind[i] == SPH_RT_COPY;
    v.t[i] = v.E[copy ? v.copysrc[i] : i];
    if (copy) continue;
    if (i < P.r1) ea += v.rho[i] * v.V[i] * v.e[i] + v.V[i] * v.E[i];
    double Ti = v.e[i] * ph.inv_cv;
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
  const double energy_before = csum(R, P, ea);  // also the barrier after a3
  if (ph.limiter != SPH_RT_LIMITER_NONE) {
    // grad E_i = sum_j F_ij V_j (E_j - E_i) (x_i - x_j), with the constant
    // weights F_ij V_j (x_i - x_j) stored per pair: 4 FP64 operations a pair
    // (3 in 2-D) instead of 9 -- the FP64 pipe bounds this kernel
    constexpr int UL = 4;
    const double *Eg = v.t;
    const bool d3 = ph.dim == 3;
    const int64_t na = v.nnz_nbr;
    for (int64_t wb = P.q0 + warp_first_group<W>(grp); wb < P.q1; wb += ngrp) {
      const int64_t i = wb + group_in_warp<W>(grp);
      const bool active = i < P.q1;
      const int64_t ia = active ? i : P.r0;
      const double Ei = v.E[ia];
      double gx = 0.0, gy = 0.0, gz = 0.0;
      const int64_t kb = active ? v.nbr_ptr[i] : 0, ke = active ? v.nbr_ptr[i + 1] : 0;
      for (int64_t kk = kb + sub; kk < ke; kk += (int64_t)W * UL) {
        int32_t jj[UL];
        double ax[UL], ay[UL], az[UL];
#pragma unroll
        for (int u = 0; u < UL; ++u) {
          const int64_t q = kk + (int64_t)u * W;
          const bool in = q < ke;
          jj[u] = in ? __ldg(v.nbr_col + q) : -1;
          ax[u] = in ? __ldg(v.nbr_A + q) : 0.0;
          ay[u] = in ? __ldg(v.nbr_A + na + q) : 0.0;
          az[u] = in && d3 ? __ldg(v.nbr_A + 2 * na + q) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < UL; ++u) {
          if (jj[u] < 0) continue;
          const double d = Eg[jj[u]] - Ei;
          gx = fma(ax[u], d, gx);
          gy = fma(ay[u], d, gy);
          if (d3) gz = fma(az[u], d, gz);  // 2-D: no z weights
        }
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
    csync();  // the copy ghosts read their sources' D
  }
  for (int64_t i = P.r1 + P.ct; i < P.s1; i += P.cn) {
    int32_t c = v.copysrc[i];
    if (c < 0) continue;
    v.T[i] = v.T[c];
    v.sigma[i] = v.sigma[c];
    v.f[i] = v.f[c];
    v.R[i] = v.R[c];
    v.lam[i] = v.lam[c];
    v.D[i] = v.D[c];
  }
  csync();  // the assembly reads D at every neighbour

  // a4: operator values, diagonal, Dirichlet coupling, Gershgorin bound
  double gmax = 0.0;
  for (int64_t wb = P.q0 + warp_first_group<W>(grp); wb < P.q1; wb += ngrp) {
    const int64_t i = wb + group_in_warp<W>(grp);
    const bool active = i < P.q1;
    const double Di = active ? v.D[i] : 0.0;
    double off = 0.0;
    const int64_t mb = active ? v.mat_ptr[i] : 0, me = active ? v.mat_ptr[i + 1] : 0;
    for (int64_t kk = mb + sub; kk < me; kk += (int64_t)W * U) {
      int32_t jj[U];
      double G[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t q = kk + (int64_t)u * W;
        jj[u] = q < me ? __ldg(v.mat_col + q) : -1;
        G[u] = q < me ? __ldg(v.mat_G + q) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (jj[u] < 0) continue;
        const double val = G[u] * (Di + v.D[jj[u]]);
        v.mat_val[kk + (int64_t)u * W] = val;
        off += val;
      }
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
      const double inv = 1.0 / dd;
      v.diag[i] = dd;
      v.invdiag[i] = inv;
      v.gb[i] = gbs;
      gmax = fmax(gmax, -off * inv);
    }
  }
  // Alg. 1: e^{n,0} = e^{n-1}, E^{n,0} = E^{n-1}.  The first Krylov solve starts
  // from the extrapolation in time of order min(p, converged steps behind)
  // through E^{n-1} and E^{n-2} (E_old, still the last step's start here),
  // E^{n-3} (H0), E^{n-4} (H1); the history then moves down one place.
  const int kp = ph.krylov_start;
  const int ord = min(kp, v.hist[k]);
  double gw[4] = {1.0, 0.0, 0.0, 0.0};
  if (ord >= 1) extrap_weights(ord, ph.dt, v.dt_hist + 3 * k, gw);
  for (int64_t i = P.q0 + threadIdx.x; i < P.q1; i += blockDim.x) {
    const double Ei = v.E[i], E2 = v.E_old[i];
    if (ord >= 1) {
      double xi = gw[0] * Ei + gw[1] * E2;
      if (ord >= 2) xi += gw[2] * v.H0[i];
      if (ord >= 3) xi += gw[3] * v.H1[i];
      v.x[i] = xi;
    }
    if (kp >= 3) v.H1[i] = v.H0[i];
    if (kp >= 2) v.H0[i] = E2;
    v.e_old[i] = v.e[i];
    v.E_old[i] = Ei;
    v.E_l[i] = Ei;
  }
  {
    double m[1] = {gmax};
    const bool mx[1] = {true};
    cred<1>(R, P, m, mx);
    if (threadIdx.x == 0) cheb_coefficients(ph.cheb_degree, 1.0 - m[0], 1.0 + m[0], &cf);
  }
  // (cf is read after the next barrier: the material solve's reduction)

  // per-particle nonlinear elimination on this CTA's rows; returns the two
  // convergence measures of the problem
  auto newton = [&](const double *E_new, const double *E_prev, const double *e_start,
                    double *e_out, double &ce, double &cE) {
    double mc[2] = {0.0, 0.0};
    for (int64_t i = P.q0 + threadIdx.x; i < P.q1; i += blockDim.x) {
      const double cs = ph.c * v.sigma[i];
      const double Pw = cs * E_new[i] + v.Qe[i];
      const double rdt = v.rho[i] / ph.dt, eo = v.e_old[i], e0 = e_start[i];
      // one FP64 division an iteration: T = e / c_v as a product, the
      // Jacobian's factor 4 c sigma a / c_v hoisted out of the loop
      const double ca = cs * ph.a, k1 = 4.0 * ca * ph.inv_cv;
      double ei = e0;
      for (int it = 0; it < ph.max_inner; ++it) {
        const double T = ei * ph.inv_cv, T3 = T * T * T;
        const double u = rdt * (ei - eo) + ca * T3 * T - Pw;
        const double J = rdt + k1 * T3;
        const double de = u / J;
        ei -= de;
        if (fabs(de) <= ph.tol_inner * fabs(ei)) break;
      }
      e_out[i] = ei;
      mc[0] = fmax(mc[0], fabs(ei - e0) / fmax(fabs(ei), 1e-300));
      mc[1] = fmax(mc[1], fabs(E_new[i] - E_prev[i]) / fmax(fabs(E_new[i]), 1e-300));
    }
    const bool mx[2] = {true, true};
    cred<2>(R, P, mc, mx);
    ce = mc[0];
    cE = mc[1];
  };
  double ce = 0.0, cE = 0.0;
  newton(v.E_l, v.E_l, v.e_old, v.e_l, ce, cE);

  int outer = 0, kry_total = 0, status = -3;
  while (outer < ph.max_outer) {
    // a7: right-hand side (B-scaled), warm start, ||b||
    double bb = 0.0;
    for (int64_t i = P.q0 + threadIdx.x; i < P.q1; i += blockDim.x) {
      double Tl = v.e_l[i] * ph.inv_cv;
      double cs = ph.c * v.sigma[i];
      double bi = v.E_old[i] / ph.dt + cs * ph.a * Tl * Tl * Tl * Tl - (1.0 - v.f[i]) * cs * v.E_l[i] +
                  v.QE[i] + v.gb[i];
      v.b[i] = v.V[i] * bi;
      if (outer > 0 || ord == 0) v.x[i] = v.E_l[i];  // else the extrapolated start
      bb += bi * bi;
    }
    const double thresh2 = ph.tol_krylov * ph.tol_krylov * csum(R, P, bb);
    // a6: Chebyshev-preconditioned CG on B.  The start x is the last outer
    // iteration's solution, whose product y = B x the CG updates carried
    // (y += alpha q), so only the first outer iteration of the step sweeps
    // the operator for its residual.
    double rr;
    if (outer == 0) {
      rr = csum(R, P, b_spmv<W, U, 1>(v, P, v.x, v.b, v.r, v.y));
    } else {
      double part = 0.0;
      for (int64_t i = P.q0 + threadIdx.x; i < P.q1; i += blockDim.x) {
        const double ri = v.b[i] - v.y[i];
        v.r[i] = ri;
        const double ru = ri * v.invV[i];
        part += ru * ru;
      }
      rr = csum(R, P, part);
    }
    int it = 0;
    bool kconv = rr <= thresh2;
    if (!kconv) {
      double rho_k = csum(R, P, b_cheb<W, U>(v, P, v.r, v.z, cf));
      for (int64_t i = P.q0 + threadIdx.x; i < P.q1; i += blockDim.x) v.p[i] = v.z[i];
      csync();  // p at every neighbour
      double pq = csum(R, P, b_spmv<W, U, 0>(v, P, v.p, nullptr, v.q));
      while (it < ph.max_krylov) {
        if (!(pq > 0.0) || !(pq < 1e308)) break;  // breakdown
        const double alpha = bdiv(rho_k, pq, bc, bpar);
        rr = 0.0;
        for (int64_t i = P.q0 + threadIdx.x; i < P.q1; i += blockDim.x) {
          v.x[i] += alpha * v.p[i];
          v.y[i] += alpha * v.q[i];
          double ri = v.r[i] - alpha * v.q[i];
          v.r[i] = ri;
          double ru = ri * v.invV[i];
          rr += ru * ru;
        }
        rr = csum(R, P, rr);
        ++it;
        if (rr <= thresh2) {
          kconv = true;
          break;
        }
        const double rho_new = csum(R, P, b_cheb<W, U>(v, P, v.r, v.z, cf));
        const double beta = bdiv(rho_new, rho_k, bc, bpar);
        rho_k = rho_new;
        for (int64_t i = P.q0 + threadIdx.x; i < P.q1; i += blockDim.x)
          v.p[i] = v.z[i] + beta * v.p[i];
        csync();  // p at every neighbour
        pq = csum(R, P, b_spmv<W, U, 0>(v, P, v.p, nullptr, v.q));
      }
    }
    kry_total += it;
    if (!kconv) break;
    // a8 + a9: material solve with the new radiation energy, convergence test
    newton(v.x, v.E_l, v.e_l, v.e_new, ce, cE);
    ++outer;
    for (int64_t i = P.q0 + threadIdx.x; i < P.q1; i += blockDim.x) {
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
    double tot[3] = {0.0, 0.0, 0.0};  // source, boundary, after
    for (int64_t i = P.q0 + threadIdx.x; i < P.q1; i += blockDim.x) {
      v.e[i] = v.e_l[i];
      v.E[i] = v.E_l[i];
      tot[0] += v.V[i] * (v.Qe[i] + v.QE[i]);
      double acc = 0.0;
      for (int64_t kk = v.gh_ptr[i]; kk < v.gh_ptr[i + 1]; ++kk) {
        int32_t j = v.gh_slot[kk];
        acc += -v.gh_W[kk] * (v.D[i] + v.D[j]) * (v.E[j] - v.E_l[i]);
      }
      tot[1] += v.V[i] * acc;
      tot[2] += v.rho[i] * v.V[i] * v.e_l[i] + v.V[i] * v.E_l[i];
    }
    const bool mx[3] = {false, false, false};
    cred<3>(R, P, tot, mx);  // also the barrier before the copy ghosts read e, E
    for (int64_t i = P.r1 + P.ct; i < P.s1; i += P.cn) {
      int32_t c = v.copysrc[i];
      if (c < 0) continue;
      v.e[i] = v.e[c];
      v.E[i] = v.E[c];
    }
    if (P.rank == 0 && threadIdx.x == 0) {
      v.energy[4 * k + 0] = energy_before;
      v.energy[4 * k + 1] = tot[2];
      v.energy[4 * k + 2] = ph.dt * tot[0];
      v.energy[4 * k + 3] = ph.dt * tot[1];
    }
  }
  if (P.rank == 0 && threadIdx.x == 0) {
    v.status[k] = status;
    v.outer[k] = outer;
    v.krylov[k] = kry_total;
    // read above by every CTA of the cluster, many cluster barriers ago
    v.hist[k] = status == 0 ? min(v.hist[k] + 1, 3) : 0;
    double *d = v.dt_hist + 3 * k;
    d[2] = d[1];
    d[1] = d[0];
    d[0] = ph.dt;
  }
  csync();  // no CTA leaves while another may still read its reduction slots
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

// Weights of the limiter gradient, one per neighbour pair (i, j):
// A_ij = F_ij V_j (x_i - x_j), stored as three arrays of nnz entries.  Rows
// without neighbours (ghost slots) are empty.  A warp per row.
__global__ void limiter_weights_kernel(int64_t n, const int64_t *nbr_ptr, const int32_t *nbr_col,
                                       const double *nbr_F, const double *V, const double *px,
                                       const double *py, const double *pz, int64_t nnz,
                                       double *A) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < n; i += nw) {
    const double xi = px[i], yi = py[i], zi = pz[i];
    for (int64_t k = nbr_ptr[i] + lane; k < nbr_ptr[i + 1]; k += 32) {
      const int32_t j = nbr_col[k];
      const double fv = nbr_F[k] * V[j];
      A[k] = fv * (xi - px[j]);
      A[nnz + k] = fv * (yi - py[j]);
      A[2 * nnz + k] = fv * (zi - pz[j]);
    }
  }
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

sph_rt_status ensure_cuda(sph_rt *s);

constexpr int kClusterKinds = 4;  // cluster sizes 1, 2, 4, 8
constexpr int kDefaultRowsPerCta = 4096;

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
  // launch shape: lanes per row W (32 / W rows per warp), Chebyshev degree and
  // resident blocks per SM; from the mean row length, cfg.cheb_degree and the
  // batch size, set by the caller, or tuned
  int W = 4, degree = 1, blocks_per_sm = 1;
  // rows per CTA: a problem of n interior rows runs on a cluster of
  // C = pow2ceil(n / rows_per_cta) CTAs (at most max_cluster); 0 = one CTA each
  int rows_per_cta = kDefaultRowsPerCta, max_cluster = 8;
  // problems grouped by cluster size (1, 2, 4, 8): one launch per group, the
  // groups' launches on forked streams so that they run side by side
  int32_t *d_order = nullptr;  // [K] problems of group 0, then group 1, ...
  int cls_off[kClusterKinds] = {}, cls_cnt[kClusterKinds] = {};
  int cls_split = -1;  // rows_per_cta the groups were built for
  cudaStream_t side[kClusterKinds - 1] = {};
  cudaEvent_t fork = nullptr, join[kClusterKinds - 1] = {};
  bool shape_set = false, tuned = false;
  double *d_e_save = nullptr, *d_E_save = nullptr;  // state kept across tuning trials
  // multi-step runs (sph_rt_batch_run): accumulators and the captured graph
  int32_t *d_run_status = nullptr, *d_run_outer = nullptr, *d_run_krylov = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  double graph_dt = 0.0;
  int32_t graph_steps = 0, graph_W = 0, graph_degree = 0, graph_bps = 0, graph_split = -1;
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
  B->degree = h->cfg.cheb_degree;
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

extern "C" sph_rt_status sph_rt_batch_add_many(sph_rt_batch *B, int32_t count,
                                               const sph_rt_problem *problems, int32_t threads,
                                               int32_t *first_index) {
  if (!B || count < 0 || (count > 0 && !problems)) return SPH_RT_EINVAL;
  if (B->packed) return set_error(B->h, SPH_RT_ESTATE, "batch already stepped; create a new one");
  if (first_index) *first_index = (int32_t)B->items.size();
  if (count == 0) return SPH_RT_OK;
  sph_rt_config c = B->cfg;
  c.stream = nullptr;
  // one staging handle per problem (own stream), set up by `threads` host
  // threads; their buffers come from the library's cache of freed device
  // memory once an earlier batch has been destroyed (measured, 120 3-D
  // problems of 1k-20k particles: 0.091 s with 1 thread, 0.042 s with 4)
  std::vector<sph_rt *> hs((size_t)count, nullptr);
  std::vector<sph_rt_status> rcs((size_t)count, SPH_RT_OK);
  std::vector<std::string> errs((size_t)count);
  std::atomic<int> next{0};
  auto work = [&]() {
    cudaSetDevice(c.device);
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= count) break;
      const sph_rt_problem &q = problems[k];
      sph_rt *t = nullptr;
      sph_rt_status rc = sph_rt_create(&c, &t);
      if (rc) {
        rcs[k] = rc;
        errs[k] = sph_rt_last_error(nullptr);
        continue;
      }
      rc = sph_rt_set_particles(t, q.n_total, q.pos, q.mass, q.rho, q.h, q.sigma0, q.kind,
                                q.copy_of, q.e0, q.E0);
      if (rc) {
        rcs[k] = rc;
        errs[k] = sph_rt_last_error(t);
        sph_rt_destroy(t);
        continue;
      }
      hs[k] = t;
    }
  };
  int nt = threads > 0 ? threads : 1;
  if (nt > count) nt = count;
  std::vector<std::thread> pool;
  for (int a = 1; a < nt; ++a) pool.emplace_back(work);
  work();
  for (auto &th : pool) th.join();
  for (int k = 0; k < count; ++k) {
    if (rcs[k] == SPH_RT_OK) continue;
    for (sph_rt *t : hs)
      if (t) sph_rt_destroy(t);
    return set_error(B->h, rcs[k], "problem " + std::to_string(k) + ": " + errs[k]);
  }
  for (int k = 0; k < count; ++k) {
    sph_rt *t = hs[k];
    BatchItem it;
    it.n = t->n;
    it.n_int = t->n_int;
    it.nnz_nbr = t->nnz_nbr;
    it.nnz_mat = t->nnz_mat;
    it.nnz_gh = t->nnz_gh;
    B->items.push_back(it);
    B->staging.push_back(t);
  }
  return SPH_RT_OK;
}

static int max_cluster_for(int bps);

static sph_rt_status batch_pack(sph_rt_batch *B) {
  sph_rt *s = B->h;
  const int K = (int)B->items.size();
  if (K == 0) return set_error(s, SPH_RT_ESTATE, "empty batch");
  if (K > 65535) return set_error(s, SPH_RT_EINVAL, "too many problems in one batch");
  sph_rt_status rc0 = ensure_cuda(s);  // the packed handle's stream, host mirror, SM count
  if (rc0) return rc0;
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
                   &v.e_old, &v.E_old, &v.e_l, &v.E_l, &v.e_new, &v.y};
  for (double **p : dd)
    if (!(*p = D(n_all))) return SPH_RT_ENOMEM;
  int32_t *kind = dalloc<int32_t>(s, n_all), *copysrc = dalloc<int32_t>(s, n_all);
  int64_t *nbr_ptr = dalloc<int64_t>(s, n_all + 1), *mat_ptr = dalloc<int64_t>(s, n_all + 1),
          *gh_ptr = dalloc<int64_t>(s, n_all + 1);
  int32_t *nbr_col = dalloc<int32_t>(s, nb), *mat_col = dalloc<int32_t>(s, nm),
          *gh_slot = dalloc<int32_t>(s, ng);
  double *nbr_F = D(nb), *nbr_A = D(3 * (size_t)nb), *mat_G = D(nm), *mat_val = D(nm),
         *gh_W = D(ng);
  B->d_slot_off = dalloc<int64_t>(s, K + 1);
  B->d_nint = dalloc<int64_t>(s, K);
  B->d_status = dalloc<int32_t>(s, K);
  B->d_outer = dalloc<int32_t>(s, K);
  B->d_krylov = dalloc<int32_t>(s, K);
  B->d_energy = D(4 * (size_t)K);
  B->d_order = dalloc<int32_t>(s, K);
  v.hist = dalloc<int32_t>(s, K);
  v.dt_hist = D(3 * (size_t)K);
  v.H0 = D(n_all);
  v.H1 = D(n_all);
  if (!B->d_order || !v.hist || !v.dt_hist || !v.H0 || !v.H1) return SPH_RT_ENOMEM;
  SPH_CUDA(s, cudaMemsetAsync(v.hist, 0, sizeof(int32_t) * K, s->stream));
  SPH_CUDA(s, cudaMemsetAsync(v.dt_hist, 0, sizeof(double) * 3 * K, s->stream));
  for (int c = 0; c < kClusterKinds - 1; ++c)
    SPH_CUDA(s, cudaStreamCreateWithFlags(&B->side[c], cudaStreamNonBlocking));
  SPH_CUDA(s, cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming));
  for (int c = 0; c < kClusterKinds - 1; ++c)
    SPH_CUDA(s, cudaEventCreateWithFlags(&B->join[c], cudaEventDisableTiming));
  if (!kind || !copysrc || !nbr_ptr || !mat_ptr || !gh_ptr || !nbr_col || !mat_col ||
      !gh_slot || !nbr_F || !nbr_A || !mat_G || !mat_val || !gh_W || !B->d_slot_off || !B->d_nint ||
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
  }
  // one wait for all the copies, then the staging handles go
  SPH_CUDA(s, cudaStreamSynchronize(st));
  for (int k = 0; k < K; ++k) {
    sph_rt_destroy(B->staging[k]);
    B->staging[k] = nullptr;
  }
  B->staging.clear();
  v.slot_off = B->d_slot_off;
  v.n_int = B->d_nint;
  v.kind = kind;
  v.copysrc = copysrc;
  v.nbr_ptr = nbr_ptr;
  v.nbr_col = nbr_col;
  v.nbr_A = nbr_A;
  v.nnz_nbr = nb;
  if (nb > 0) {
    limiter_weights_kernel<<<std::max(1, std::min<int>((int)((n_all + 7) / 8), s->num_sms * 16)),
                             256, 0, s->stream>>>(n_all, nbr_ptr, nbr_col, nbr_F, v.V, v.px, v.py,
                                                  v.pz, nb, nbr_A);
    SPH_LAUNCHED(s);
    SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  }
  dfree(s, nbr_F);  // only the weights are used by the steps
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
  v.order = B->d_order;
  int64_t ni_all = 0;
  for (int k = 0; k < K; ++k) ni_all += nint[k];
  B->max_cluster = std::min(max_cluster_for(1), max_cluster_for(2));
  if (!B->shape_set) {
    B->W = lanes_for_mean(ni_all ? (double)nm / (double)ni_all : 0.0);
    // more problems than SMs: two blocks per SM keep them all in flight
    B->blocks_per_sm = K > s->num_sms ? 2 : 1;
  }
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
  ph.inv_cv = 1.0 / c.cv;
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
  ph.cheb_degree = B->degree;
  ph.dim = c.dim;
  ph.krylov_start = c.krylov_start;
  return ph;
}

static bool batch_lanes_ok(int W) { return W == 1 || W == 2 || W == 4 || W == 8; }

template <int W, int MINB>
static cudaError_t launch_cluster(const BatchView &v, const BatchPhys &ph, int C, cudaStream_t st) {
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)v.K * (unsigned)C);
  lc.blockDim = dim3(512);
  lc.dynamicSmemBytes = 0;
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, batch_step_kernel<W, 8, MINB>, v, ph);
}

template <int MINB>
static cudaError_t launch_cluster_w(int W, const BatchView &v, const BatchPhys &ph, int C,
                                    cudaStream_t st) {
  if (W == 1) return launch_cluster<1, MINB>(v, ph, C, st);
  if (W == 2) return launch_cluster<2, MINB>(v, ph, C, st);
  if (W == 4) return launch_cluster<4, MINB>(v, ph, C, st);
  return launch_cluster<8, MINB>(v, ph, C, st);
}

// Largest cluster (<= 8) of which at least one fits on the GPU with this
// kernel variant's registers (1 or 2 CTAs per SM).
static int max_cluster_for(int bps) {
  int best = 1;
  for (int C = 2; C <= 8; C *= 2) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)C);
    lc.blockDim = dim3(512);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    int n = 0;
    cudaError_t e = bps == 2 ? cudaOccupancyMaxActiveClusters(&n, batch_step_kernel<4, 8, 2>, &lc)
                             : cudaOccupancyMaxActiveClusters(&n, batch_step_kernel<4, 8, 1>, &lc);
    if (e != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    if (n < 1) break;
    best = C;
  }
  return best;
}

// Cluster size of a problem of n interior rows.
static int cluster_of(int64_t n, int rows_per_cta, int max_cluster) {
  if (rows_per_cta <= 0) return 1;
  int C = 1;
  while (C < max_cluster && (int64_t)C * rows_per_cta < n) C *= 2;
  return C;
}

// Group the problems by cluster size (each group largest first, ties by
// index) and upload the launch order.  A problem's cluster size depends on
// its own size only, so its result does not depend on the rest of the batch.
static sph_rt_status batch_groups(sph_rt_batch *B) {
  if (B->cls_split == B->rows_per_cta) return SPH_RT_OK;
  sph_rt *s = B->h;
  const int K = (int)B->items.size();
  std::vector<int32_t> order;
  order.reserve(K);
  for (int g = 0; g < kClusterKinds; ++g) {
    const int C = 1 << g;
    std::vector<int32_t> mem;
    for (int k = 0; k < K; ++k)
      if (cluster_of(B->items[k].n_int, B->rows_per_cta, B->max_cluster) == C) mem.push_back(k);
    auto work = [&](int k) { return B->items[k].nnz_mat + 4 * B->items[k].n_int; };
    std::stable_sort(mem.begin(), mem.end(), [&](int a, int b) { return work(a) > work(b); });
    B->cls_off[g] = (int)order.size();
    B->cls_cnt[g] = (int)mem.size();
    order.insert(order.end(), mem.begin(), mem.end());
  }
  SPH_CUDA(s, cudaMemcpyAsync(B->d_order, order.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice,
                              s->stream));
  SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  B->cls_split = B->rows_per_cta;
  return SPH_RT_OK;
}

// One batched step: a launch per cluster-size group.  The first group runs on
// the batch's stream, the others on side streams forked from it and joined
// back, so the groups overlap (also inside a captured graph: parallel
// branches).
// The groups must be current (batch_groups) before the call, which may be
// inside a stream capture.
static sph_rt_status launch_batch_step(sph_rt_batch *B, const BatchView &v, const BatchPhys &ph) {
  sph_rt *s = B->h;
  int used[kClusterKinds], nu = 0;
  for (int g = 0; g < kClusterKinds; ++g)
    if (B->cls_cnt[g] > 0) used[nu++] = g;
  if (nu > 1) {
    SPH_CUDA(s, cudaEventRecord(B->fork, s->stream));
    for (int a = 1; a < nu; ++a) SPH_CUDA(s, cudaStreamWaitEvent(B->side[a - 1], B->fork, 0));
  }
  for (int a = 0; a < nu; ++a) {
    const int g = used[a];
    BatchView vg = v;
    vg.K = B->cls_cnt[g];
    vg.order = B->d_order + B->cls_off[g];
    cudaStream_t st = a == 0 ? s->stream : B->side[a - 1];
    cudaError_t e = B->blocks_per_sm == 2 ? launch_cluster_w<2>(B->W, vg, ph, 1 << g, st)
                                          : launch_cluster_w<1>(B->W, vg, ph, 1 << g, st);
    SPH_CUDA(s, e);
    SPH_LAUNCHED(s);
  }
  for (int a = 1; a < nu; ++a) {
    SPH_CUDA(s, cudaEventRecord(B->join[a - 1], B->side[a - 1]));
    SPH_CUDA(s, cudaStreamWaitEvent(s->stream, B->join[a - 1], 0));
  }
  return SPH_RT_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the batched launch: lanes per row W (32 / W rows per warp),
// the Chebyshev degree, resident blocks per SM, and rows per CTA (how large
// a cluster each problem gets).  The degree trades Krylov iterations (fewer
// as the polynomial gets stronger) against operator sweeps per iteration, W
// trades idle lanes on short rows against more rows per reduction, two blocks
// per SM trade spilled registers against CTAs in flight, and smaller row
// chunks trade cluster barriers against the time of the largest problem,
// which bounds the step; none of these balances is known before the batch's
// operators are.  Every candidate runs one step from the same state (restored
// after each trial, so the tuning leaves the problems where they were) and is
// timed with CUDA events on the batch's stream; a candidate counts only if
// every problem converged, and the fastest one is kept.  The first three
// dimensions are searched as a grid at the current rows per CTA, then the
// rows per CTA at the best of them.  A first untimed launch of each kernel
// variant takes module loading and cold caches out of the comparison.
// ---------------------------------------------------------------------------
static const int kTuneBlocks[] = {1, 2};
static const int kTuneLanes[] = {1, 2, 4, 8};
static const int kTuneDegrees[] = {1, 2, 3, 4, 6};
static const int kTuneRows[] = {0, 2048, 4096, 8192};
constexpr int kNB = 2, kNW = 4, kND = 5, kNR = 4;
static_assert(kNB * kNW * kND + kNR == SPH_RT_BATCH_TUNE_CANDIDATES,
              "candidate table and header disagree");

static sph_rt_status batch_restore(sph_rt_batch *B) {
  sph_rt *s = B->h;
  const size_t bytes = sizeof(double) * (size_t)s->n;
  SPH_CUDA(s, cudaMemcpyAsync(B->view.e, B->d_e_save, bytes, cudaMemcpyDeviceToDevice, s->stream));
  SPH_CUDA(s, cudaMemcpyAsync(B->view.E, B->d_E_save, bytes, cudaMemcpyDeviceToDevice, s->stream));
  // E_old now holds the trial's start, not E^{n-2}: the next step starts from E^{n-1}
  SPH_CUDA(s, cudaMemsetAsync(B->view.hist, 0, sizeof(int32_t) * B->view.K, s->stream));
  return SPH_RT_OK;
}

static sph_rt_status batch_autotune(sph_rt_batch *B, double dt, float *times_ms) {
  sph_rt *s = B->h;
  const int K = B->view.K;
  const size_t bytes = sizeof(double) * (size_t)s->n;
  if (!B->d_e_save) {
    B->d_e_save = dalloc<double>(s, s->n);
    B->d_E_save = dalloc<double>(s, s->n);
    if (!B->d_e_save || !B->d_E_save) return SPH_RT_ENOMEM;
  }
  SPH_CUDA(s, cudaMemcpyAsync(B->d_e_save, B->view.e, bytes, cudaMemcpyDeviceToDevice, s->stream));
  SPH_CUDA(s, cudaMemcpyAsync(B->d_E_save, B->view.E, bytes, cudaMemcpyDeviceToDevice, s->stream));
  BatchView v = B->view;
  v.run_status = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  SPH_CUDA(s, cudaEventCreate(&ev[0]));
  if (cudaEventCreate(&ev[1]) != cudaSuccess) {
    cudaEventDestroy(ev[0]);
    return set_error(s, SPH_RT_EDEVICE, "autotune: cudaEventCreate failed");
  }
  std::vector<int32_t> st(K);
  float best = -1.0f;
  int bestW = B->W, bestDeg = B->degree, bestB = B->blocks_per_sm, bestR = B->rows_per_cta;
  const int deg0 = B->degree;
  sph_rt_status rc = SPH_RT_OK;
  // one timed trial of the current shape; ms < 0 if some problem did not converge
  auto trial = [&](float *slot) -> sph_rt_status {
    sph_rt_status r2;
    if ((r2 = batch_groups(B))) return r2;
    float ms = -1.0f;
    if (cudaEventRecord(ev[0], s->stream) != cudaSuccess ||
        (r2 = launch_batch_step(B, v, batch_phys(B, dt))) ||
        cudaEventRecord(ev[1], s->stream) != cudaSuccess ||
        cudaMemcpyAsync(st.data(), B->d_status, sizeof(int32_t) * K, cudaMemcpyDeviceToHost,
                        s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess ||
        cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess)
      return r2 ? r2 : set_error(s, SPH_RT_EDEVICE, "autotune: CUDA error in a trial");
    bool ok = true;
    for (int k = 0; k < K; ++k) ok = ok && st[k] == 0;
    if (slot) *slot = ok ? ms : -1.0f;
    if (ok && (best < 0.0f || ms < best)) {
      best = ms;
      bestW = B->W;
      bestDeg = B->degree;
      bestB = B->blocks_per_sm;
      bestR = B->rows_per_cta;
    }
    return batch_restore(B);
  };
  for (int c = 0; c < kNB * kNW && !rc; ++c) {
    B->blocks_per_sm = kTuneBlocks[c / kNW];
    B->W = kTuneLanes[c % kNW];
    B->degree = deg0;
    if ((rc = batch_groups(B)) || (rc = launch_batch_step(B, v, batch_phys(B, dt))) ||
        (rc = batch_restore(B)))
      break;
    for (int d = 0; d < kND && !rc; ++d) {
      B->degree = kTuneDegrees[d];
      rc = trial(times_ms ? times_ms + c * kND + d : nullptr);
    }
  }
  for (int r = 0; r < kNR && !rc; ++r) {
    B->W = bestW;
    B->degree = bestDeg;
    B->blocks_per_sm = bestB;
    B->rows_per_cta = kTuneRows[r];
    rc = trial(times_ms ? times_ms + kNB * kNW * kND + r : nullptr);
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  B->W = bestW;
  B->degree = bestDeg;
  B->blocks_per_sm = bestB;
  B->rows_per_cta = bestR;
  B->tuned = true;
  if (rc) return rc;
  if ((rc = batch_groups(B))) return rc;
  SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  return SPH_RT_OK;
}

// pack on first use, then tune once if the configuration asks for it
static sph_rt_status batch_ready(sph_rt_batch *B, double dt) {
  sph_rt_status rc;
  if (!B->packed && (rc = batch_pack(B))) return rc;
  SPH_CUDA(B->h, cudaSetDevice(B->h->cfg.device));
  if (B->cfg.autotune == 1 && !B->tuned && !B->shape_set && (rc = batch_autotune(B, dt, nullptr)))
    return rc;
  return batch_groups(B);
}

extern "C" sph_rt_status sph_rt_batch_run(sph_rt_batch *B, double dt, int32_t steps,
                                          int32_t *status, int32_t *outer_total,
                                          int32_t *krylov_total) {
  if (!B) return SPH_RT_EINVAL;
  if (!isfinite(dt) || dt <= 0.0) return set_error(B->h, SPH_RT_EINVAL, "dt must be finite and > 0");
  if (steps < 1) return set_error(B->h, SPH_RT_EINVAL, "steps must be >= 1");
  sph_rt_status rc;
  if ((rc = batch_ready(B, dt))) return rc;
  sph_rt *s = B->h;
  const int K = B->view.K;
  if (!B->d_run_status) {
    B->d_run_status = dalloc<int32_t>(s, K);
    B->d_run_outer = dalloc<int32_t>(s, K);
    B->d_run_krylov = dalloc<int32_t>(s, K);
    if (!B->d_run_status || !B->d_run_outer || !B->d_run_krylov) return SPH_RT_ENOMEM;
  }
  if (!B->graph_exec || B->graph_dt != dt || B->graph_steps != steps || B->graph_W != B->W ||
      B->graph_degree != B->degree || B->graph_bps != B->blocks_per_sm ||
      B->graph_split != B->rows_per_cta) {
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
    B->graph_W = B->W;
    B->graph_degree = B->degree;
    B->graph_bps = B->blocks_per_sm;
    B->graph_split = B->rows_per_cta;
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
  if ((rc = batch_ready(B, dt))) return rc;
  sph_rt *s = B->h;
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

extern "C" sph_rt_status sph_rt_batch_set_shape(sph_rt_batch *B, const sph_rt_batch_shape *shape) {
  if (!B || !shape) return SPH_RT_EINVAL;
  if (!batch_lanes_ok(shape->lanes_per_row))
    return set_error(B->h, SPH_RT_EINVAL, "lanes_per_row must be 1, 2, 4 or 8");
  if (shape->cheb_degree < 1 || shape->cheb_degree > 16)
    return set_error(B->h, SPH_RT_EINVAL, "cheb_degree must be in [1, 16]");
  if (shape->blocks_per_sm != 1 && shape->blocks_per_sm != 2)
    return set_error(B->h, SPH_RT_EINVAL, "blocks_per_sm must be 1 or 2");
  if (shape->rows_per_cta < 0 || (shape->rows_per_cta > 0 && shape->rows_per_cta < 64))
    return set_error(B->h, SPH_RT_EINVAL, "rows_per_cta must be 0 or >= 64");
  B->W = shape->lanes_per_row;
  B->degree = shape->cheb_degree;
  B->blocks_per_sm = shape->blocks_per_sm;
  B->rows_per_cta = shape->rows_per_cta;
  B->shape_set = true;
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_batch_get_shape(const sph_rt_batch *B, sph_rt_batch_shape *shape) {
  if (!B || !shape) return SPH_RT_EINVAL;
  shape->lanes_per_row = B->W;
  shape->cheb_degree = B->degree;
  shape->blocks_per_sm = B->blocks_per_sm;
  shape->rows_per_cta = B->rows_per_cta;
  return SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_batch_autotune(sph_rt_batch *B, double dt, float *times_ms,
                                               sph_rt_batch_shape *chosen) {
  if (!B) return SPH_RT_EINVAL;
  if (!isfinite(dt) || dt <= 0.0) return set_error(B->h, SPH_RT_EINVAL, "dt must be finite and > 0");
  sph_rt_status rc;
  if (!B->packed && (rc = batch_pack(B))) return rc;
  SPH_CUDA(B->h, cudaSetDevice(B->h->cfg.device));
  if ((rc = batch_autotune(B, dt, times_ms))) return rc;
  B->shape_set = true;
  return chosen ? sph_rt_batch_get_shape(B, chosen) : SPH_RT_OK;
}

extern "C" sph_rt_status sph_rt_batch_problem_info(const sph_rt_batch *B, int32_t index,
                                                   int64_t info[5]) {
  if (!B || !info) return SPH_RT_EINVAL;
  if (index < 0 || index >= (int32_t)B->items.size()) return SPH_RT_EINVAL;
  const BatchItem &it = B->items[index];
  info[0] = it.n;
  info[1] = it.n_int;
  info[2] = it.nnz_mat;
  info[3] = it.nnz_nbr;
  info[4] = cluster_of(it.n_int, B->rows_per_cta, B->max_cluster);
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
  if (B->graph_exec || B->graph || B->fork) {
    cudaSetDevice(B->h->cfg.device);
    if (B->h->cuda_ready) cudaStreamSynchronize(B->h->stream);
    batch_graph_release(B);
    for (int c = 0; c < kClusterKinds - 1; ++c) {
      if (B->side[c]) cudaStreamDestroy(B->side[c]);
      if (B->join[c]) cudaEventDestroy(B->join[c]);
    }
    if (B->fork) cudaEventDestroy(B->fork);
  }
  for (sph_rt *t : B->staging)
    if (t) sph_rt_destroy(t);
  sph_rt_destroy(B->h);
  delete B;
}
