// physics.cu -- per-particle and per-row kernels of one time step
// (rows a3, a4, a7, a8, a9 of the hot path).
//
//  a3  material data, frozen for the step (Sec. 3.2):
//        T = e/c_v, sigma = sigma0 T^p, Fleck factor f = 1/(1 + c sigma dt 4aT^3/(rho c_v))
//        (Sec. 2.2), SPH gradient grad E_i = sum_j V_j (E_j - E_i) F_ij x_ij (Sec. 2.3),
//        R = |grad E|/(sigma_t E), flux limiter lambda(R) (Sec. 2.1), D = c lambda / sigma_t,
//        sigma_t = sigma_a + sigma_s (constant scattering opacity sigma_s).
//  a4  operator of Eq. diffusion-solve scaled by V:  B_ij = V_i V_j F_ij (D_i + D_j) for
//        j != i, B_ii = V_i (1/dt + c sigma_i f_i) + sum over all neighbours of
//        V_i w_ij, w_ij = -V_j (D_i + D_j) F_ij >= 0; Dirichlet neighbours move to
//        the right-hand side as gb_i = sum_j w_ij E_j.
//  a7  right-hand side (Sec. 3.2, operators S and N):
//        b_i = E_i^{n-1}/dt + c sigma_i a T_i^4 - (1 - f_i) c sigma_i E_i + Q_E,i + gb_i.
//  a8  material solve M^{-1} (Eq. material-energy-update), one thread per particle.
//  a9  outer convergence (Eq. mat-rad-convergence) and energy totals (Sec. 2.5).
#include <cuda_runtime.h>

#include "common.cuh"

namespace sphrt {

struct Phys {
  double a, c, cv, p, T_floor, larsen_k, dt;
  double sigma_s;  // scattering opacity: sigma_t = sigma_a + sigma_s (R and D, Sec. 2.1)
  double inv_cv, inv_dt;  // 1/cv, 1/dt (the Newton loop multiplies instead of dividing)
  double tol_inner;
  int limiter, max_inner;
};

__device__ __forceinline__ double opacity(double sigma0, double Ts, double p) {
  if (p == 0.0) return sigma0;
  if (p == -3.0) return sigma0 / (Ts * Ts * Ts);
  return sigma0 * pow(Ts, p);
}

__device__ __forceinline__ double limiter_lambda(int limiter, double k, double R) {
  if (limiter == SPH_RT_LIMITER_LEVERMORE) return (2.0 + R) / (6.0 + 3.0 * R + R * R);
  if (limiter == SPH_RT_LIMITER_LARSEN) {
    if (k == 2.0) return 1.0 / sqrt(9.0 + R * R);
    return 1.0 / pow(pow(3.0, k) + pow(R, k), 1.0 / k);
  }
  return 1.0 / 3.0;
}

// a3, point part: every non-copy slot (interior and Dirichlet ghosts).
__global__ void props_point_kernel(Phys ph, int64_t n, const int32_t *kind, const double *rho,
                                   const double *sigma0, const double *e, double *T,
                                   double *sigma, double *f, double *R, double *lambda,
                                   double *D) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (kind[i] == SPH_RT_COPY) continue;
    double Ti = e[i] / ph.cv;
    double Ts = Ti > ph.T_floor ? Ti : ph.T_floor;
    double sig = opacity(sigma0[i], Ts, ph.p);
    double fi = 1.0 / (1.0 + ph.c * sig * ph.dt * 4.0 * ph.a * Ti * Ti * Ti / (rho[i] * ph.cv));
    T[i] = Ti;
    sigma[i] = sig;
    f[i] = fi;
    // R = 0 here; interior rows with a limiter are overwritten by the gradient kernel
    double lam = limiter_lambda(ph.limiter, ph.larsen_k, 0.0);
    R[i] = 0.0;
    lambda[i] = lam;
    D[i] = ph.c * lam / (sig + ph.sigma_s);
  }
}

// a3, gradient part: one group of W lanes per interior row.
template <int W>
__global__ void props_grad_kernel(Phys ph, int64_t n_int, const int64_t *nbr_ptr,
                                  const int32_t *nbr_col, const double *nbr_F, const double *px,
                                  const double *py, const double *pz, const double *V,
                                  const int32_t *kind, const int32_t *copysrc, const double *E,
                                  const double *sigma, double *R, double *lambda, double *D) {
  const int sub = threadIdx.x % W;
  const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / W;
  const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / W;
  for (int64_t wb = warp_first_group<W>(grp); wb < n_int; wb += ngrp) {
    const int64_t i = wb + group_in_warp<W>(grp);
    const bool active = i < n_int;
    const int64_t ia = active ? i : 0;
    double xi = px[ia], yi = py[ia], zi = pz[ia], Ei = E[ia];
    double gx = 0.0, gy = 0.0, gz = 0.0;
    const int64_t kbeg = active ? nbr_ptr[i] : 0, kend = active ? nbr_ptr[i + 1] : 0;
    for (int64_t k = kbeg + sub; k < kend; k += W) {
      int32_t j = nbr_col[k];
      int32_t js = kind[j] == SPH_RT_COPY ? copysrc[j] : j;
      double s = V[j] * (E[js] - Ei) * nbr_F[k];
      gx += s * (xi - px[j]);
      gy += s * (yi - py[j]);
      gz += s * (zi - pz[j]);
    }
    gx = group_sum<W>(gx);
    gy = group_sum<W>(gy);
    gz = group_sum<W>(gz);
    if (active && sub == 0) {
      double gn = sqrt(gx * gx + gy * gy + gz * gz);
      double Es = Ei > 1e-300 ? Ei : 1e-300;
      const double sig_t = sigma[i] + ph.sigma_s;
      double Ri = gn / (sig_t * Es);
      double lam = limiter_lambda(ph.limiter, ph.larsen_k, Ri);
      R[i] = Ri;
      lambda[i] = lam;
      D[i] = ph.c * lam / sig_t;
    }
  }
}

// Gradient sums of one row by its W-lane group (a row-tile round): entries
// beg + sub + j W, j < nmax (nmax warp-uniform; see row_dot_n), each adding
// (E_j - E_i) g_ij to the three components.  Slots past the row's end add
// fma(0, 0, g) = g.
template <int W, int U>
__device__ __forceinline__ Sum3 grad_row_n(int64_t beg, int64_t end, const int32_t *__restrict__ gcol,
                                           const double *__restrict__ gvx,
                                           const double *__restrict__ gvy,
                                           const double *__restrict__ gvz,
                                           const double *__restrict__ E, double Ei, int sub,
                                           int nmax) {
  double gx = 0.0, gy = 0.0, gz = 0.0;
  int64_t k = beg + sub;
  int j = 0;
  for (; j + U <= nmax; j += U, k += (int64_t)W * U) {
    int32_t c[U];
    double ax[U], ay[U], az[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t kk = k + (int64_t)u * W;
      const bool ok = kk < end;
      c[u] = ok ? __ldg(gcol + kk) : -1;
      ax[u] = ok ? __ldg(gvx + kk) : 0.0;
      ay[u] = ok ? __ldg(gvy + kk) : 0.0;
      az[u] = ok ? __ldg(gvz + kk) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (c[u] < 0) continue;
      const double dE = __ldg(E + c[u]) - Ei;
      gx = fmadd(dE, ax[u], gx);
      gy = fmadd(dE, ay[u], gy);
      gz = fmadd(dE, az[u], gz);
    }
  }
  const int rem = nmax - j;  // warp-uniform, < U
  if (rem > 0) {
    double dE[U], ax[U], ay[U], az[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t kk = k + (int64_t)u * W;
      const bool ok = kk < end;
      const int32_t c = ok ? __ldg(gcol + kk) : -1;
      ax[u] = ok ? __ldg(gvx + kk) : 0.0;
      ay[u] = ok ? __ldg(gvy + kk) : 0.0;
      az[u] = ok ? __ldg(gvz + kk) : 0.0;
      dE[u] = c >= 0 ? __ldg(E + c) - Ei : 0.0;
    }
#pragma unroll 1
    for (int u = 0; u < rem; ++u) {
      gx = fmadd(dE[0], ax[0], gx);
      gy = fmadd(dE[0], ay[0], gy);
      gz = fmadd(dE[0], az[0], gz);
#pragma unroll
      for (int q = 0; q + 1 < U; ++q) {
        dE[q] = dE[q + 1];
        ax[q] = ax[q + 1];
        ay[q] = ay[q + 1];
        az[q] = az[q + 1];
      }
    }
  }
  return {gx, gy, gz};
}

// a3, gradient part with precomputed pair geometry g_ij = V_j F_ij x_ij and
// the slot whose E a neighbour carries (its own, or the copied particle's):
// grad E_i = sum_j (E_j - E_i) g_ij.  Row tiles (common.cuh): 32 rows per warp,
// the row epilogue (|grad E|, R, the limiter, D) on all 32 lanes.
// Resident blocks per SM the row-tile gradient and assembly kernels are
// compiled for (80 registers: their rounds carry three sums and, at the end of
// a row, up to U slots of pair data).
constexpr int kPairMinBlocks = 3;

template <int W, int U>
__global__ void __launch_bounds__(kBlock, kPairMinBlocks)
    props_grad_pre_kernel(Phys ph, int64_t n_int, const int64_t *nbr_ptr, const int32_t *gcol,
                          const double *gvx, const double *gvy, const double *gvz,
                          const double *E, const double *sigma, double *R, double *lambda,
                          double *D) {
  const int lane = threadIdx.x & 31, sub = lane % W, own = tile_own_row<W>(lane);
  int64_t r0, r1;
  warp_rows<W>(n_int, r0, r1);
  for (int64_t base = r0; base < r1; base += 32) {
    const int rows = (int)(r1 - base < 32 ? r1 - base : 32);
    const int64_t i = base + own;
    const bool active = own < rows;
    int64_t b = 0, e = 0;
    double Eo = 0.0;
    if (active) {
      b = nbr_ptr[i];
      e = nbr_ptr[i + 1];
      Eo = E[i];
    }
    const Sum3 g = tile_tree<W, 1, Sum3>(0, rows, sub, [&](int t) -> Sum3 {
      const int64_t rb = __shfl_sync(0xffffffffu, b, t, W);
      const int64_t re = __shfl_sync(0xffffffffu, e, t, W);
      const double Ei = __shfl_sync(0xffffffffu, Eo, t, W);
      return grad_row_n<W, U>(rb, re, gcol, gvx, gvy, gvz, E, Ei, sub,
                              tile_nmax<W>(rb, re, sub));
    });
    if (active) {
      const double gx = g.a, gy = g.b, gz = g.c;
      double gn = sqrt(gx * gx + gy * gy + gz * gz);
      double Es = Eo > 1e-300 ? Eo : 1e-300;
      const double sig_t = sigma[i] + ph.sigma_s;
      double Ri = gn / (sig_t * Es);
      double lam = limiter_lambda(ph.limiter, ph.larsen_k, Ri);
      R[i] = Ri;
      lambda[i] = lam;
      D[i] = ph.c * lam / sig_t;
    }
  }
}

// pair geometry for the gradient (once per particle set)
__global__ void grad_geom_kernel(int64_t n_int, const int64_t *nbr_ptr, const int32_t *nbr_col,
                                 const double *nbr_F, const double *px, const double *py,
                                 const double *pz, const double *V, const int32_t *kind,
                                 const int32_t *copysrc, int32_t *gcol, double *gvx, double *gvy,
                                 double *gvz) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_int;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double xi = px[i], yi = py[i], zi = pz[i];
    for (int64_t k = nbr_ptr[i]; k < nbr_ptr[i + 1]; ++k) {
      const int32_t j = nbr_col[k];
      gcol[k] = kind[j] == SPH_RT_COPY ? copysrc[j] : j;
      const double vf = V[j] * nbr_F[k];
      gvx[k] = vf * (xi - px[j]);
      gvy[k] = vf * (yi - py[j]);
      gvz[k] = vf * (zi - pz[j]);
    }
  }
}

// copy ghosts take every property of the particle they copy
__global__ void props_copy_kernel(int64_t n_int, int64_t n, const int32_t *copysrc, double *T,
                                  double *sigma, double *f, double *R, double *lambda, double *D) {
  for (int64_t i = n_int + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t s = copysrc[i];
    if (s < 0) continue;
    T[i] = T[s];
    sigma[i] = sigma[s];
    f[i] = f[s];
    R[i] = R[s];
    lambda[i] = lambda[s];
    D[i] = D[s];
  }
}

// Off-diagonal values of one row of B by its W-lane group (a row-tile round):
// B_ij = G_ij (D_i + D_j) written for entries beg + sub + j W, j < nmax
// (nmax warp-uniform), and this lane's sum of them.  Slots past the row's end
// store nothing and add +0.
// F32: also write the FP32 copy of the mixed form.
template <int W, int U, bool F32>
__device__ __forceinline__ double assemble_row_n(int64_t beg, int64_t end,
                                                 const int32_t *__restrict__ mat_col,
                                                 const double *__restrict__ mat_G,
                                                 const double *__restrict__ D, double Di,
                                                 double *__restrict__ mat_val,
                                                 float *__restrict__ mat_val32, int sub,
                                                 int nmax) {
  double offsum = 0.0;
  int64_t k = beg + sub;
  int j = 0;
  for (; j + U <= nmax; j += U, k += (int64_t)W * U) {
    int32_t c[U];
    double g[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t kk = k + (int64_t)u * W;
      c[u] = kk < end ? __ldg(mat_col + kk) : -1;
      g[u] = kk < end ? __ldg(mat_G + kk) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (c[u] < 0) continue;
      const double v = g[u] * (Di + __ldg(D + c[u]));
      mat_val[k + (int64_t)u * W] = v;
      if (F32) mat_val32[k + (int64_t)u * W] = (float)v;
      offsum += v;
    }
  }
  const int rem = nmax - j;  // warp-uniform, < U
  if (rem > 0) {
    double g[U], dj[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t kk = k + (int64_t)u * W;
      const int32_t c = kk < end ? __ldg(mat_col + kk) : -1;
      g[u] = c >= 0 ? __ldg(mat_G + kk) : 0.0;
      dj[u] = c >= 0 ? __ldg(D + c) : 0.0;
    }
#pragma unroll 1
    for (int u = 0; u < rem; ++u, k += W) {
      if (k < end) {
        const double v = g[0] * (Di + dj[0]);
        mat_val[k] = v;
        if (F32) mat_val32[k] = (float)v;
        offsum += v;
      }
#pragma unroll
      for (int q = 0; q + 1 < U; ++q) {
        g[q] = g[q + 1];
        dj[q] = dj[q + 1];
      }
    }
  }
  return offsum;
}

// a4: values of B for the step.  Row tiles (common.cuh): in each round a
// W-lane group writes one row's off-diagonal values and sums them, then adds
// up its Dirichlet-ghost couplings (few rows have any); the diagonal, its
// inverse, the ghost right-hand side and the Gershgorin ratio are computed on
// all 32 lanes.
template <int W, int U, bool F32>
__global__ void __launch_bounds__(kBlock, kPairMinBlocks)
    assemble_kernel(Phys ph, int64_t n_int, const int64_t *mat_ptr, const int32_t *mat_col,
                    const double *mat_G, double *mat_val, const int64_t *gh_ptr,
                    const int32_t *gh_slot, const double *gh_W, const double *V,
                    const double *sigma, const double *f, const double *D, const double *E,
                    double *diag, double *invdiag, double *gb, double *partials,
                    unsigned *counter, double *gersh_out, float *mat_val32, float *diag32,
                    float *invdiag32) {
  // gersh_out = max_i sum_{j != i} |B_ij| / B_ii: the eigenvalues of D^{-1} B
  // lie in [1 - gersh, 1 + gersh] (Gershgorin; B is symmetric, so real).
  const int lane = threadIdx.x & 31, sub = lane % W, own = tile_own_row<W>(lane);
  int64_t r0, r1;
  warp_rows<W>(n_int, r0, r1);
  double gmax = 0.0;
  for (int64_t base = r0; base < r1; base += 32) {
    const int rows = (int)(r1 - base < 32 ? r1 - base : 32);
    const int64_t i = base + own;
    const bool active = own < rows;
    int64_t b = 0, e = 0, hb = 0, he = 0;
    double Do = 0.0;
    if (active) {
      b = mat_ptr[i];
      e = mat_ptr[i + 1];
      hb = gh_ptr[i];
      he = gh_ptr[i + 1];
      Do = D[i];
    }
    const Sum3 acc = tile_tree<W, 1, Sum3>(0, rows, sub, [&](int t) -> Sum3 {
      const int64_t rb = __shfl_sync(0xffffffffu, b, t, W);
      const int64_t re = __shfl_sync(0xffffffffu, e, t, W);
      const int64_t gb0 = __shfl_sync(0xffffffffu, hb, t, W);
      const int64_t ge0 = __shfl_sync(0xffffffffu, he, t, W);
      const double Di = __shfl_sync(0xffffffffu, Do, t, W);
      const double offsum = assemble_row_n<W, U, F32>(rb, re, mat_col, mat_G, D, Di, mat_val,
                                                      mat_val32, sub, tile_nmax<W>(rb, re, sub));
      double wsum = 0.0, gbs = 0.0;
      const int ng = tile_nmax<W>(gb0, ge0, sub);
      for (int jj = 0; jj < ng; ++jj) {
        const int64_t k = gb0 + sub + (int64_t)jj * W;
        if (k < ge0) {
          const int32_t j = gh_slot[k];
          const double wk = -gh_W[k] * (Di + D[j]);
          wsum += wk;
          gbs += wk * E[j];
        }
      }
      return {offsum, wsum, gbs};
    });
    if (active) {
      const double offsum = acc.a, wsum = acc.b, gbs = acc.c;
      double d = V[i] * (1.0 / ph.dt + ph.c * sigma[i] * f[i] + wsum) - offsum;
      diag[i] = d;
      invdiag[i] = 1.0 / d;
      if (F32) {
        diag32[i] = (float)d;
        invdiag32[i] = (float)(1.0 / d);
      }
      gb[i] = gbs;
      gmax = fmax(gmax, -offsum / d);  // off-diagonals are <= 0
    }
  }
  __shared__ double sh[32];
  gmax = block_max(gmax, sh);
  double part[1] = {gmax}, out[1];
  const bool mx[1] = {true};
  if (last_block_combine<1>(part, partials, counter, out, mx) && threadIdx.x == 0)
    *gersh_out = out[0];
}

// a7: right-hand side of the diffusion solve (B-scaled), the warm start x = E^l,
// ||b||^2 of the unscaled rows, and reset of the Krylov scalars.
__global__ void rhs_kernel(Phys ph, int64_t n_int, const double *V, const double *sigma,
                           const double *f, const double *E_old, const double *e_l,
                           const double *E_l, const double *QE, const double *gb, double *b,
                           double *x, double tol, Scalars *sc, double *partials,
                           const double *H0, const double *H1, const double *H2) {
  // the first outer iteration's solve may start from the extrapolation in time
  // through E^l = E^{n-1} and H0, H1, H2 = E^{n-2}, E^{n-3}, E^{n-4}
  const int ord = sc->outer_iters == 0 ? sc->guess_order : 0;
  const double w0 = sc->guess_w[0], w1 = sc->guess_w[1], w2 = sc->guess_w[2],
               w3 = sc->guess_w[3];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_int;
       i += (int64_t)gridDim.x * blockDim.x) {
    double Tl = e_l[i] / ph.cv;
    double B = ph.a * Tl * Tl * Tl * Tl;
    double cs = ph.c * sigma[i];
    double bi = E_old[i] / ph.dt + cs * B - (1.0 - f[i]) * cs * E_l[i] + QE[i] + gb[i];
    b[i] = V[i] * bi;
    double xi = E_l[i];
    if (ord >= 1) {
      xi = w0 * xi + w1 * H0[i];
      if (ord >= 2) xi += w2 * H1[i];
      if (ord >= 3) xi += w3 * H2[i];
    }
    x[i] = xi;
    acc += bi * bi;
  }
  __shared__ double sh[32];
  double bs = block_sum(acc, sh);
  double part[1] = {bs}, out[1];
  const bool mx[1] = {false};
  if (last_block_combine<1>(part, partials, &sc->counter, out, mx) && threadIdx.x == 0) {
    sc->bnorm2 = out[0];
    sc->thresh2 = tol * tol * out[0];
    sc->done = 0;
    sc->iters = 0;
    sc->breakdown = 0;
  }
}

// a8 + a9: material solve with the new radiation energy and the outer
// convergence measures.  P_i = c sigma_i E_i + Q_e,i (Eq. material-energy-solve);
// Newton from e_start.  red[0] = max |e_new - e_start|/|e_new|,
// red[1] = max |E_new - E_prev|/|E_new|, red[2] = max Newton iterations,
// red[3] = number of particles that hit the iteration limit.
__global__ void newton_kernel(Phys ph, int64_t n_int, const double *rho, const double *sigma,
                              const double *e_old, const double *Qe, const double *E_new,
                              const double *E_prev, const double *e_start, double *e_new,
                              Scalars *sc, double *partials) {
  double ce = 0.0, cE = 0.0, itmax = 0.0, fails = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_int;
       i += (int64_t)gridDim.x * blockDim.x) {
    double cs = ph.c * sigma[i];
    double P = cs * E_new[i] + Qe[i];
    // per-particle constants of u(e) = rho/dt (e - e_old) + c sigma a T^4 - P and
    // J = rho/dt + 4 c sigma a T^3 / cv, hoisted out of the loop: one FP64
    // division (u / J) per iteration is left, on a part whose FP64 pipe is narrow
    double rdt = rho[i] * ph.inv_dt;
    double csa = cs * ph.a;
    double k4 = 4.0 * csa * ph.inv_cv;
    double eo = e_old[i];
    double e0 = e_start[i];
    double ei = e0;
    int it = 0;
    bool ok = false;
    while (it < ph.max_inner) {
      double T = ei * ph.inv_cv;
      double T3 = T * T * T;
      double u = rdt * (ei - eo) + csa * T3 * T - P;
      double J = rdt + k4 * T3;
      double de = u / J;
      ei = ei - de;
      ++it;
      if (fabs(de) <= ph.tol_inner * fabs(ei)) {
        ok = true;
        break;
      }
    }
    e_new[i] = ei;
    ce = fmax(ce, fabs(ei - e0) / fmax(fabs(ei), 1e-300));
    cE = fmax(cE, fabs(E_new[i] - E_prev[i]) / fmax(fabs(E_new[i]), 1e-300));
    itmax = fmax(itmax, (double)it);
    if (!ok) fails += 1.0;
  }
  __shared__ double sh[32];
  double p0 = block_max(ce, sh);
  __syncthreads();
  double p1 = block_max(cE, sh);
  __syncthreads();
  double p2 = block_max(itmax, sh);
  __syncthreads();
  double p3 = block_sum(fails, sh);
  double part[4] = {p0, p1, p2, p3}, out[4];
  const bool mx[4] = {true, true, true, false};
  if (last_block_combine<4>(part, partials, &sc->counter, out, mx) && threadIdx.x == 0) {
    sc->red[0] = out[0];
    sc->red[1] = out[1];
    sc->red[2] = out[2];
    sc->red[3] = out[3];
  }
}

// Step inputs must be finite: sources of interior particles, ghost values of
// Dirichlet ghosts (caller order).  Sets sc->bad_input.
__global__ void check_inputs_kernel(int64_t n, const int64_t *caller2slot, const int32_t *kind,
                                    const double *Qe, const double *QE, const double *ge,
                                    const double *gE, Scalars *sc) {
  int bad = 0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int k = kind[caller2slot[c]];
    if (k == SPH_RT_INTERIOR) {
      if ((Qe && !isfinite(Qe[c])) || (QE && !isfinite(QE[c]))) bad = 1;
    } else if (k == SPH_RT_DIRICHLET) {
      if ((ge && !isfinite(ge[c])) || (gE && !isfinite(gE[c]))) bad = 1;
    }
  }
  if (bad) atomicExch(&sc->bad_input, 1);
}

// Totals over interior particles: red[4] = sum m e, red[5] = sum V E.
__global__ void totals_kernel(int64_t n_int, const double *mass, const double *V, const double *e,
                              const double *E, Scalars *sc, double *partials) {
  double a = 0.0, b = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_int;
       i += (int64_t)gridDim.x * blockDim.x) {
    a += mass[i] * e[i];
    b += V[i] * E[i];
  }
  __shared__ double sh[32];
  double pa = block_sum(a, sh);
  __syncthreads();
  double pb = block_sum(b, sh);
  double part[2] = {pa, pb}, out[2];
  const bool mx[2] = {false, false};
  if (last_block_combine<2>(part, partials, &sc->counter, out, mx) && threadIdx.x == 0) {
    sc->red[4] = out[0];
    sc->red[5] = out[1];
  }
}

// Energy added over the step: red[6] = dt sum V (Q_e + Q_E);
// red[7] = dt sum_i V_i sum_{Dirichlet j} w_ij (E_j - E_i).
__global__ void balance_kernel(Phys ph, int64_t n_int, const double *V, const double *Qe,
                               const double *QE, const int64_t *gh_ptr, const int32_t *gh_slot,
                               const double *gh_W, const double *D, const double *E,
                               Scalars *sc, double *partials) {
  double a = 0.0, b = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_int;
       i += (int64_t)gridDim.x * blockDim.x) {
    a += V[i] * (Qe[i] + QE[i]);
    double acc = 0.0;
    for (int64_t k = gh_ptr[i]; k < gh_ptr[i + 1]; ++k) {
      int32_t j = gh_slot[k];
      acc += -gh_W[k] * (D[i] + D[j]) * (E[j] - E[i]);
    }
    b += V[i] * acc;
  }
  __shared__ double sh[32];
  double pa = block_sum(a, sh);
  __syncthreads();
  double pb = block_sum(b, sh);
  double part[2] = {pa, pb}, out[2];
  const bool mx[2] = {false, false};
  if (last_block_combine<2>(part, partials, &sc->counter, out, mx) && threadIdx.x == 0) {
    sc->red[6] = ph.dt * out[0];
    sc->red[7] = ph.dt * out[1];
  }
}

// Install Dirichlet ghost values (slot order) from caller-order arrays.
__global__ void ghost_install_kernel(int64_t n_int, int64_t n, const int32_t *kind,
                                     const int64_t *slot2caller, const double *ge_c,
                                     const double *gE_c, double *e, double *E) {
  for (int64_t s = n_int + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    if (kind[s] != SPH_RT_DIRICHLET) continue;
    int64_t c = slot2caller[s];
    if (ge_c) e[s] = ge_c[c];
    if (gE_c) E[s] = gE_c[c];
  }
}

__global__ void copy_ghost_sync_kernel(int64_t n_int, int64_t n, const int32_t *copysrc,
                                       double *e, double *E) {
  for (int64_t s = n_int + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    int32_t c = copysrc[s];
    if (c < 0) continue;
    e[s] = e[c];
    E[s] = E[c];
  }
}

// caller-order source -> slot order (interior part); NULL source gives zeros
__global__ void gather_interior_kernel(const double *in_c, const int64_t *slot2caller,
                                       int64_t n_int, double *out) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_int;
       s += (int64_t)gridDim.x * blockDim.x)
    out[s] = in_c ? in_c[slot2caller[s]] : 0.0;
}

__global__ void scatter_caller_kernel(const double *in_s, const int64_t *slot2caller, int64_t n,
                                      double *out_c) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x)
    out_c[slot2caller[s]] = in_s[s];
}

// End of a step: a converged step with valid inputs commits its interior
// state; any other step restores the snapshot taken at its start (ghost
// entries included), so a failed step leaves the state unchanged.
__global__ void finish_kernel(int64_t n_int, int64_t n, const double *e_new, const double *E_new,
                              const double *e_bak, const double *E_bak, double *e, double *E,
                              const Scalars *sc) {
  const bool commit = sc->outer_status == 1 && !sc->bad_input;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (commit) {
      if (i < n_int) {
        e[i] = e_new[i];
        E[i] = E_new[i];
      }
    } else {
      e[i] = e_bak[i];
      E[i] = E_bak[i];
    }
  }
}

// the totals just reduced (red[4], red[5]) are the energy before the step
__global__ void save_before_kernel(Scalars *sc) {
  sc->energy_before_e = sc->red[4];
  sc->energy_before_E = sc->red[5];
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static int grid_items(const sph_rt *s, int64_t n, int per_block) {
  int64_t g = ceil_div(n > 0 ? n : 1, per_block);
  int64_t cap = (int64_t)s->num_sms * 8;
  if (cap > kMaxRedBlocks) cap = kMaxRedBlocks;
  return (int)(g < cap ? g : cap);
}

Phys make_phys(const sph_rt *s, double dt) {
  Phys ph;
  ph.a = s->cfg.a;
  ph.c = s->cfg.c;
  ph.cv = s->cfg.cv;
  ph.inv_cv = 1.0 / s->cfg.cv;
  ph.inv_dt = 1.0 / dt;
  ph.p = s->cfg.opacity_exp;
  ph.T_floor = s->cfg.T_floor;
  ph.larsen_k = s->cfg.larsen_k;
  ph.sigma_s = s->cfg.sigma_s;
  ph.dt = dt;
  ph.tol_inner = s->cfg.tol_inner_e;
  ph.limiter = s->cfg.limiter;
  ph.max_inner = s->cfg.max_inner_e;
  return ph;
}

// rows per group of the warp-per-row kernels, from the mean row length
int row_width(int64_t nnz, int64_t rows) {
  double mean = rows > 0 ? (double)nnz / (double)rows : 0.0;
  if (mean > 48) return 32;
  if (mean > 12) return 16;
  return 8;
}

#define SPH_ROWS_LAUNCH(KERNEL, W, grid, s, ...)                              \
  do {                                                                        \
    if ((W) == 32) KERNEL<32><<<grid, kBlock, 0, (s)->stream>>>(__VA_ARGS__); \
    else if ((W) == 16) KERNEL<16><<<grid, kBlock, 0, (s)->stream>>>(__VA_ARGS__); \
    else KERNEL<8><<<grid, kBlock, 0, (s)->stream>>>(__VA_ARGS__);            \
    SPH_LAUNCHED(s);                                                          \
  } while (0)

sph_rt_status launch_properties(sph_rt *s, double dt) {
  Phys ph = make_phys(s, dt);
  int g = grid_items(s, s->n, kBlock);
  props_point_kernel<<<g, kBlock, 0, s->stream>>>(ph, s->n, s->kind, s->rho, s->sigma0, s->e,
                                                   s->T, s->sigma, s->f, s->R, s->lambda, s->D);
  SPH_LAUNCHED(s);
  if (s->cfg.limiter != SPH_RT_LIMITER_NONE) {
    // pair geometry once per particle set, if it fits a modest share of memory
    const double geom_bytes = 28.0 * (double)s->nnz_nbr;
    if (!s->gvx && geom_bytes < 24e9) {
      s->gcol = dalloc<int32_t>(s, s->nnz_nbr);
      s->gvx = dalloc<double>(s, s->nnz_nbr);
      s->gvy = dalloc<double>(s, s->nnz_nbr);
      s->gvz = dalloc<double>(s, s->nnz_nbr);
      if (!s->gcol || !s->gvx || !s->gvy || !s->gvz) return SPH_RT_ENOMEM;
      grad_geom_kernel<<<grid_items(s, s->n_int, kBlock), kBlock, 0, s->stream>>>(
          s->n_int, s->nbr_ptr, s->nbr_col, s->nbr_F, s->px, s->py, s->pz, s->V, s->kind,
          s->copysrc, s->gcol, s->gvx, s->gvy, s->gvz);
      SPH_LAUNCHED(s);
    }
    if (s->gvx) {
      RowShape sh = shape_for_mean(s->n_int ? (double)s->nnz_nbr / (double)s->n_int : 0.0);
      int gr = row_grid_blocks(s->num_sms, s->n_int, sh.W, kPairMinBlocks);
      SPH_DISPATCH_SHAPE(sh.W, sh.U,
                         (props_grad_pre_kernel<W, U><<<gr, kBlock, 0, s->stream>>>(
                             ph, s->n_int, s->nbr_ptr, s->gcol, s->gvx, s->gvy, s->gvz, s->E,
                             s->sigma, s->R, s->lambda, s->D)));
      SPH_LAUNCHED(s);
    } else {
      int W = row_width(s->nnz_nbr, s->n_int);
      int gr = grid_items(s, s->n_int, kBlock / W);
      SPH_ROWS_LAUNCH(props_grad_kernel, W, gr, s, ph, s->n_int, s->nbr_ptr, s->nbr_col,
                      s->nbr_F, s->px, s->py, s->pz, s->V, s->kind, s->copysrc, s->E, s->sigma,
                      s->R, s->lambda, s->D);
    }
  }
  if (s->n > s->n_int) {
    props_copy_kernel<<<grid_items(s, s->n - s->n_int, kBlock), kBlock, 0, s->stream>>>(
        s->n_int, s->n, s->copysrc, s->T, s->sigma, s->f, s->R, s->lambda, s->D);
    SPH_LAUNCHED(s);
  }
  return SPH_RT_OK;
}

sph_rt_status launch_assembly(sph_rt *s, double dt, double *gersh_out) {
  Phys ph = make_phys(s, dt);
  RowShape sh = shape_for_mean(s->n_int ? (double)s->nnz_mat / (double)s->n_int : 0.0);
  int gr = row_grid_blocks(s->num_sms, s->n_int, sh.W, kPairMinBlocks);
  // the mixed form gets its FP32 copy of the fine operator in the same pass
  if (s->mat_val32)
    SPH_DISPATCH_SHAPE(sh.W, sh.U,
                       (assemble_kernel<W, U, true><<<gr, kBlock, 0, s->stream>>>(
                           ph, s->n_int, s->mat_ptr, s->mat_col, s->mat_G, s->mat_val, s->gh_ptr,
                           s->gh_slot, s->gh_W, s->V, s->sigma, s->f, s->D, s->E, s->diag,
                           s->invdiag, s->gb, s->partials, &s->sc->counter, gersh_out,
                           s->mat_val32, s->diag32, s->invdiag32)));
  else
    SPH_DISPATCH_SHAPE(sh.W, sh.U,
                       (assemble_kernel<W, U, false><<<gr, kBlock, 0, s->stream>>>(
                           ph, s->n_int, s->mat_ptr, s->mat_col, s->mat_G, s->mat_val, s->gh_ptr,
                           s->gh_slot, s->gh_W, s->V, s->sigma, s->f, s->D, s->E, s->diag,
                           s->invdiag, s->gb, s->partials, &s->sc->counter, gersh_out,
                           nullptr, nullptr, nullptr)));
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

sph_rt_status launch_rhs(sph_rt *s, double dt) {
  Phys ph = make_phys(s, dt);
  int g = grid_items(s, s->n_int, kBlock);
  rhs_kernel<<<g, kBlock, 0, s->stream>>>(ph, s->n_int, s->V, s->sigma, s->f, s->E_old, s->e_l,
                                           s->E_l, s->QE, s->gb, s->b, s->x, s->cfg.tol_krylov,
                                           s->sc, s->partials, s->E_hist[0], s->E_hist[1],
                                           s->E_hist[2]);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

__global__ void set_guess_kernel(Scalars *sc, int order, double w0, double w1, double w2,
                                 double w3) {
  sc->guess_order = order;
  sc->guess_w[0] = w0;
  sc->guess_w[1] = w1;
  sc->guess_w[2] = w2;
  sc->guess_w[3] = w3;
}

// order and weights of the extrapolated start of the step's first solve (order 0: E^l)
sph_rt_status launch_set_guess(sph_rt *s, int order, const double *w) {
  set_guess_kernel<<<1, 1, 0, s->stream>>>(s->sc, order, w[0], w[1], w[2], w[3]);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

sph_rt_status launch_newton(sph_rt *s, double dt, const double *E_new, const double *E_prev,
                            const double *e_start, double *e_out) {
  Phys ph = make_phys(s, dt);
  int g = grid_items(s, s->n_int, kBlock);
  newton_kernel<<<g, kBlock, 0, s->stream>>>(ph, s->n_int, s->rho, s->sigma, s->e_old, s->Qe,
                                              E_new, E_prev, e_start, e_out, s->sc, s->partials);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

sph_rt_status launch_check_inputs(sph_rt *s, const double *Qe, const double *QE,
                                  const double *ge, const double *gE) {
  SPH_CUDA(s, cudaMemsetAsync(&s->sc->bad_input, 0, sizeof(int), s->stream));
  if (!Qe && !QE && !ge && !gE) return SPH_RT_OK;
  check_inputs_kernel<<<grid_items(s, s->n, kBlock), kBlock, 0, s->stream>>>(
      s->n, s->caller2slot, s->kind, Qe, QE, ge, gE, s->sc);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

// ---------------------------------------------------------------------------
// Time step choice (Sec. 3.3, Eq. energy-fractional), after a converged step:
//   xbar = sum_i x_i^n V_i / sum_i V_i                       (volume average)
//   eta_x = max_i |x_i^n - x_i^{n-1}| / (x_i^n + target xbar + floor)
//   dt_x = dt (target / eta_x)^(1/2)
//   dt_next = min(dt_e, dt_E, growth dt, dt_max), at least dt_min
// for x = e and x = E over the interior particles.  x^{n-1} is the snapshot
// taken at the start of the step.
// ---------------------------------------------------------------------------
__global__ void dtc_sums_kernel(int64_t n_int, const double *V, const double *e, const double *E,
                                Scalars *sc, double *partials) {
  double a = 0.0, b = 0.0, v = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_int;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double Vi = V[i];
    a += e[i] * Vi;
    b += E[i] * Vi;
    v += Vi;
  }
  __shared__ double sh[32];
  double part[3];
  part[0] = block_sum(a, sh);
  __syncthreads();
  part[1] = block_sum(b, sh);
  __syncthreads();
  part[2] = block_sum(v, sh);
  double out[3];
  const bool mx[3] = {false, false, false};
  if (last_block_combine<3>(part, partials, &sc->counter, out, mx) && threadIdx.x == 0) {
    sc->dtc_ebar = out[0] / out[2];
    sc->dtc_Ebar = out[1] / out[2];
  }
}

struct DtControl {
  double dt, target, growth, dt_min, dt_max, floor;
};

__global__ void dtc_eta_kernel(int64_t n_int, const double *e, const double *E,
                               const double *e_old, const double *E_old, DtControl c, Scalars *sc,
                               double *partials) {
  const double de = c.target * sc->dtc_ebar + c.floor, dE = c.target * sc->dtc_Ebar + c.floor;
  double me = 0.0, mE = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_int;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double en = e[i], En = E[i];
    me = fmax(me, fabs(en - e_old[i]) / (en + de));
    mE = fmax(mE, fabs(En - E_old[i]) / (En + dE));
  }
  __shared__ double sh[32];
  double part[2];
  part[0] = block_max(me, sh);
  __syncthreads();
  part[1] = block_max(mE, sh);
  double out[2];
  const bool mx[2] = {true, true};
  if (last_block_combine<2>(part, partials, &sc->counter, out, mx) && threadIdx.x == 0) {
    double next = fmin(c.growth * c.dt, c.dt_max);
    if (out[0] > 0.0) next = fmin(next, c.dt * sqrt(c.target / out[0]));
    if (out[1] > 0.0) next = fmin(next, c.dt * sqrt(c.target / out[1]));
    sc->dtc_eta_e = out[0];
    sc->dtc_eta_E = out[1];
    sc->dtc_next = fmax(next, c.dt_min);
  }
}

sph_rt_status launch_dt_control(sph_rt *s, double dt) {
  const int g = grid_items(s, s->n_int, kBlock);
  dtc_sums_kernel<<<g, kBlock, 0, s->stream>>>(s->n_int, s->V, s->e, s->E, s->sc, s->partials);
  SPH_LAUNCHED(s);
  const DtControl c = {dt, s->cfg.dt_target, s->cfg.dt_growth, s->cfg.dt_min, s->cfg.dt_max,
                       s->cfg.dt_eta_floor};
  dtc_eta_kernel<<<g, kBlock, 0, s->stream>>>(s->n_int, s->e, s->E, s->e_bak, s->E_bak, c, s->sc,
                                              s->partials);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

sph_rt_status launch_totals(sph_rt *s, const double *e, const double *E) {
  int g = grid_items(s, s->n_int, kBlock);
  totals_kernel<<<g, kBlock, 0, s->stream>>>(s->n_int, s->mass, s->V, e, E, s->sc, s->partials);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

sph_rt_status launch_balance(sph_rt *s, double dt, const double *E) {
  Phys ph = make_phys(s, dt);
  int g = grid_items(s, s->n_int, kBlock);
  balance_kernel<<<g, kBlock, 0, s->stream>>>(ph, s->n_int, s->V, s->Qe, s->QE, s->gh_ptr,
                                               s->gh_slot, s->gh_W, s->D, E, s->sc, s->partials);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

sph_rt_status launch_ghost_install(sph_rt *s, const double *ge_c, const double *gE_c) {
  if (s->n == s->n_int || (!ge_c && !gE_c)) return SPH_RT_OK;
  int g = grid_items(s, s->n - s->n_int, kBlock);
  ghost_install_kernel<<<g, kBlock, 0, s->stream>>>(s->n_int, s->n, s->kind, s->slot2caller,
                                                     ge_c, gE_c, s->e, s->E);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

sph_rt_status launch_copy_sync(sph_rt *s) {
  if (s->n == s->n_int) return SPH_RT_OK;
  int g = grid_items(s, s->n - s->n_int, kBlock);
  copy_ghost_sync_kernel<<<g, kBlock, 0, s->stream>>>(s->n_int, s->n, s->copysrc, s->e, s->E);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

sph_rt_status launch_gather_interior(sph_rt *s, const double *in_c, double *out) {
  int g = grid_items(s, s->n_int, kBlock);
  gather_interior_kernel<<<g, kBlock, 0, s->stream>>>(in_c, s->slot2caller, s->n_int, out);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

sph_rt_status launch_scatter_caller(sph_rt *s, const double *in_s, int64_t count, double *out_c) {
  int g = grid_items(s, count, kBlock);
  scatter_caller_kernel<<<g, kBlock, 0, s->stream>>>(in_s, s->slot2caller, count, out_c);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

sph_rt_status launch_finish(sph_rt *s, const double *e_new, const double *E_new) {
  int g = grid_items(s, s->n, kBlock);
  finish_kernel<<<g, kBlock, 0, s->stream>>>(s->n_int, s->n, e_new, E_new, s->e_bak, s->E_bak,
                                             s->e, s->E, s->sc);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

sph_rt_status launch_save_before(sph_rt *s) {
  save_before_kernel<<<1, 1, 0, s->stream>>>(s->sc);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

}  // namespace sphrt
