// common.cuh -- shared device helpers and the internal handle of libsphrt.
//
// Index spaces.  Particles are sorted once by (ghost flag, Morton code of the
// cell, caller index), so "slots" [0, n_int) are the interior particles in
// Morton order and [n_int, n) the ghosts.  Unknowns of the radiation system
// are the interior slots, so an unknown's index IS its slot and the solver
// needs no index maps.
//
// Operator scaling.  The library stores B = V A, V = diag(m/rho), where A is
// the paper's row operator of Eq. diffusion-solve.  B_ij = V_i V_j F_ij (D_i +
// D_j) is bitwise symmetric (V_i V_j commutes, F_ij is the symmetric two-h
// average) and B is an M-matrix, so the Krylov solver is CG and the AMG
// hierarchy is built from symmetric Galerkin products.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <cstring>

#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/sph_rt.h"

namespace sphrt {

constexpr int kBlock = 256;          // threads per block of the 1-D kernels
constexpr int kWarpsPerBlock = kBlock / 32;
constexpr int kMaxRedBlocks = 2048;  // upper bound on blocks of a reducing kernel
// Resident blocks per SM the SpMV-class sweeps are compiled for, i.e. their
// register cap (65536 / (kBlock * blocks)): 5 blocks (48 registers) with U = 4
// loads in flight per lane, 4 blocks (64 registers) with U = 8.  Their grids
// never exceed this many blocks per SM (row_grid), so one wave covers all rows.
__host__ __device__ constexpr int sweep_min_blocks(int U) { return U >= 8 ? 4 : 5; }
// The coarse levels' sweeps (a few thousand to a few tens of thousands of
// L2-resident rows: latency-bound, not throughput-bound) also load their row
// operands before the row sums, which takes them to 64 registers.
constexpr int kCoarseMinBlocks = 4;

// --------------------------------------------------------------------------
// Scalars of one Krylov solve and of the outer loop, kept on the device so
// that the iteration runs without host round trips between kernels.
// --------------------------------------------------------------------------
struct Scalars {
  double rho;      // (r, z)
  double alpha;    // rho / (p, q)
  double beta;     // rho_new / rho
  double pq;       // (p, B p)
  double rnorm2;   // ||r / V||^2 (unscaled residual)
  double bnorm2;   // ||b||^2 (unscaled right-hand side)
  double thresh2;  // tol^2 ||b||^2
  double red[8];   // results of generic reductions
  int done;        // Krylov converged (or aborted)
  int iters;       // Krylov iterations taken
  int breakdown;   // non-positive curvature / NaN seen
  int bad_input;   // a step input (source or ghost value) was not finite
  int gate_timeout;  // a timing gate gave up waiting for the host (timing only)
  unsigned int counter;  // arrival counter of the last-block reductions
  // outer (nonlinear-elimination) loop of Alg. 1, advanced by outer_check_kernel
  int outer_iters;       // completed outer iterations
  int outer_status;      // 0 running, 1 converged, 2 Krylov failure, 3 max_outer reached
  int outer_trips;       // loop trips (termination guard of the device-driven loop)
  int krylov_total;      // Krylov iterations over the converged outer iterations
  int krylov_trips;      // Krylov loop trips over all outer iterations (launch count)
  int krylov_solve_trips;  // Krylov loop trips of the current solve (termination guard)
  int newton_max;        // largest material Newton iteration count
  int krylov_per_outer[64];
  double last_change_e, last_change_E;
  double energy_before_e, energy_before_E;  // interior totals at the start of the step
  // CG with the V-cycle's product (fine_post_smooth = 0)
  int pfirst;      // the next update starts the directions: p = z, q = B z
  int ru;          // mixed form: the next launch replaces r by the FP64 residual
  double rmax2;    // mixed form: largest ||r / V||^2 since the last replacement
  int yvalid;      // mixed form: the last solve ended on a verified residual whose B x
                   // (kept in the handle's w) is that of the next solve's start
  // time step choice of the last converged step (config.dt_target > 0)
  double dtc_ebar, dtc_Ebar, dtc_eta_e, dtc_eta_E, dtc_next;
  // start of the first solve of a step: x = sum_j guess_w[j] E^{n-1-j}, j <= guess_order
  // (E^{n-1} = E^l; guess_order 0: x = E^l)
  double guess_w[4];
  int guess_order;
};

// Lagrange extrapolation in time of order p (0..3): the weights w[0..p] with
// sum_j w[j] E(t_{n-1-j}) the value at t_n of the polynomial of degree p through
// E^{n-1}, ..., E^{n-1-p}.  dt is t_n - t_{n-1}; d[j] = t_{n-1-j} - t_{n-2-j}
// are the previous steps' sizes.  p = 1: w = (1 + dt/d0, -dt/d0).
__host__ __device__ inline void extrap_weights(int p, double dt, const double *d, double *w) {
  double tau[4];  // node times relative to t_{n-1}
  tau[0] = 0.0;
  for (int j = 1; j <= p; ++j) tau[j] = tau[j - 1] - d[j - 1];
  for (int j = 0; j <= p; ++j) {
    double num = 1.0, den = 1.0;
    for (int m = 0; m <= p; ++m) {
      if (m == j) continue;
      num *= dt - tau[m];
      den *= tau[j] - tau[m];
    }
    w[j] = num / den;
  }
}

// --------------------------------------------------------------------------
// Warp and block reductions (fixed order: deterministic).
// --------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
template <int W>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, W);
  return v;
}

// Sum of v over the block; result valid in thread 0.  `sh` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double *sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) {
    int nw = (blockDim.x + 31) >> 5;
    s = lane < nw ? sh[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;
}
__device__ __forceinline__ double block_max(double v, double *sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) {
    int nw = (blockDim.x + 31) >> 5;
    s = lane < nw ? sh[lane] : 0.0;
    s = warp_max(s);
  }
  return s;
}

// Last-block reduction: every block stores its NV partial values, the block
// that arrives last combines all partials in block order (so the result does
// not depend on scheduling) and returns true in all its threads; `out` then
// holds the NV totals in thread 0 (sums, or maxima where is_max[k]).
template <int NV>
__device__ bool last_block_combine(const double (&part)[NV], double *partials, unsigned *counter,
                                   double (&out)[NV], const bool (&is_max)[NV]) {
  __shared__ bool am_last;
  __shared__ double sh[32];
  if (threadIdx.x == 0) {
    for (int k = 0; k < NV; ++k) partials[(size_t)k * gridDim.x + blockIdx.x] = part[k];
    __threadfence();
    unsigned ticket = atomicAdd(counter, 1u);
    am_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  for (int k = 0; k < NV; ++k) {
    double acc = 0.0;  // partial maxima are of non-negative quantities
    // each thread folds a strided subset in order, then a fixed-shape tree
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
      double v = ((volatile double *)partials)[(size_t)k * gridDim.x + b];
      acc = is_max[k] ? fmax(acc, v) : acc + v;
    }
    acc = is_max[k] ? block_max(acc, sh) : block_sum(acc, sh);
    if (threadIdx.x == 0) out[k] = acc;
    __syncthreads();
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Off-diagonal part of one CSR row times a gathered vector, computed by the W
// lanes of a row group (this lane's partial sum; reduce over the group after).
// Each pass first issues U independent column/value loads per lane and then U
// independent gathers, so a row of up to W*U entries costs one dependent
// memory round trip instead of one per W entries.  Out-of-range slots load
// nothing and add nothing.
// Explicit fused multiply-add: the kernels that must agree bit for bit (the
// launched V-cycle and its cluster-resident tail) spell out every fusion
// instead of leaving the choice to the compiler's contraction.
__device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }

template <int W, int U, typename MT, typename VT>
__device__ __forceinline__ VT row_dot(int64_t beg, int64_t end, const int32_t *__restrict__ col,
                                      const MT *__restrict__ val, const VT *__restrict__ x,
                                      int sub) {
  VT s = VT(0);
  for (int64_t k = beg + sub; k < end; k += (int64_t)W * U) {
    int32_t c[U];
    MT v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t kk = k + (int64_t)u * W;
      c[u] = kk < end ? __ldg(col + kk) : -1;
      v[u] = kk < end ? __ldg(val + kk) : MT(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (c[u] >= 0) s = fmadd((VT)v[u], __ldg(x + c[u]), s);
  }
  return s;
}

// Row loops of W-lane row groups must be WARP-UNIFORM: row_reduce's full-mask
// shuffles need every lane of the warp, so all the groups of a warp make the
// same number of passes.  Loop over the warp's base row (the row of its first
// group) and give each group its offset; a group past the end of the range is
// inactive (an empty row) but still takes part in the shuffles.
//   for (int64_t wb = r0 + warp_first_group<W>(grp); wb < r1; wb += ngrp) {
//     const int64_t i = wb + group_in_warp<W>(grp);
//     const bool active = i < r1;  ...
template <int W>
__device__ __forceinline__ int64_t group_in_warp(int64_t grp) {
  return grp % (32 / W);
}
template <int W>
__device__ __forceinline__ int64_t warp_first_group(int64_t grp) {
  return grp - group_in_warp<W>(grp);
}

// Sum over the W lanes of a row group (W divides 32; groups are aligned).
template <int W, typename T>
__device__ __forceinline__ T row_reduce(T v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, W);
  return v;
}

// ---------------------------------------------------------------------------
// Row tiles: the layout of the SpMV-class sweeps.
//
// On this part an FP64 warp instruction occupies the narrow FP64 pipe for all
// 32 lanes whether or not a lane is active, so lanes left idle by a sweep cost
// as much as busy ones.  A warp therefore works on tiles of 32 consecutive rows
// in W rounds; in round t its G = 32/W row groups (W lanes each) take rows
// t G + g.  Per round the warp issues exactly as many FMA instructions as its
// longest row needs (not a multiple of the load batch); after the W rounds a
// transposed shuffle reduction leaves the sum of row (l mod W) G + l/W in lane
// l with W - 1 adds per lane instead of log2(W) adds per lane and row; and the
// row epilogue (diagonal term, vector updates, reductions) runs on all 32
// lanes instead of one lane per group, with its loads and stores coalesced.
//
// The arithmetic of a row is that of row_dot + row_reduce exactly: each lane
// sums its entries beg + sub + j W in increasing j, and the reduction adds the
// lane partials in the same tree (lanes W/2 apart first), so every row sum is
// bitwise that of the one-row-per-group form.
// ---------------------------------------------------------------------------

// Offset, within its tile, of the row whose sum and epilogue lane `lane` holds.
template <int W>
__device__ __forceinline__ int tile_own_row(int lane) {
  return (lane % W) * (32 / W) + lane / W;
}

// Contiguous rows [r0, r1) of this warp: the rows are cut into units of G =
// 32/W (one round of a tile) and the units are spread as evenly as possible
// over all warps of the grid.  Warp-uniform.
template <int W>
__device__ __forceinline__ void warp_rows(int64_t n, int64_t &r0, int64_t &r1) {
  constexpr int G = 32 / W;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t units = ceil_div(n, G), q = units / nwarps, rem = units % nwarps;
  const int64_t u0 = w * q + (w < rem ? w : rem);
  const int64_t u1 = u0 + q + (w < rem ? 1 : 0);
  r0 = u0 * G < n ? u0 * G : n;
  r1 = u1 * G < n ? u1 * G : n;
}

// Off-diagonal sum of one row by its W-lane group with a warp-uniform trip
// count: nmax = the largest per-lane entry count over the warp, so the warp
// issues nmax FMA instructions.  Full passes keep U column/value loads and U
// gathers in flight per lane; the last, partial pass loads its slots at once
// and then runs its FMAs in a loop of exactly (nmax mod U) trips, shifting the
// loaded slots down.  Slots past a lane's row end load nothing and contribute
// fma(0, 0, s) = s.
template <int W, int U, typename MT, typename VT>
__device__ __forceinline__ VT row_dot_n(int64_t beg, int64_t end, const int32_t *__restrict__ col,
                                        const MT *__restrict__ val, const VT *__restrict__ x,
                                        int sub, int nmax) {
  VT s = VT(0);
  int64_t k = beg + sub;
  int j = 0;
  for (; j + U <= nmax; j += U, k += (int64_t)W * U) {
    int32_t c[U];
    MT v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t kk = k + (int64_t)u * W;
      c[u] = kk < end ? __ldg(col + kk) : -1;
      v[u] = kk < end ? __ldg(val + kk) : MT(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (c[u] >= 0) s = fmadd((VT)v[u], __ldg(x + c[u]), s);
  }
  const int rem = nmax - j;  // warp-uniform, < U
  if (rem > 0) {
    VT a[U], g[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t kk = k + (int64_t)u * W;
      const int32_t c = kk < end ? __ldg(col + kk) : -1;
      a[u] = c >= 0 ? (VT)__ldg(val + kk) : VT(0);
      g[u] = c >= 0 ? __ldg(x + c) : VT(0);
    }
#pragma unroll 1
    for (int u = 0; u < rem; ++u) {
      s = fmadd(a[0], g[0], s);
#pragma unroll
      for (int q = 0; q + 1 < U; ++q) {
        a[q] = a[q + 1];
        g[q] = g[q + 1];
      }
    }
  }
  return s;
}

// Partial of a tile round that holds three sums (the gradient's components,
// or the assembly's off-diagonal, ghost-weight and ghost right-hand-side sums);
// added and shuffled component by component.
struct Sum3 {
  double a, b, c;
};
__device__ __forceinline__ Sum3 operator+(const Sum3 &x, const Sum3 &y) {
  return {x.a + y.a, x.b + y.b, x.c + y.c};
}
template <int W>
__device__ __forceinline__ double tile_shfl(double v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o, W);
}
template <int W>
__device__ __forceinline__ float tile_shfl(float v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o, W);
}
template <int W>
__device__ __forceinline__ Sum3 tile_shfl(const Sum3 &v, int o) {
  return {tile_shfl<W>(v.a, o), tile_shfl<W>(v.b, o), tile_shfl<W>(v.c, o)};
}

// One step of the transposed reduction at lane distance o: `lo` and `hi` are
// this lane's partials of two rounds that differ in bit o (lo: bit clear).
// The lane with bit o of its group index clear keeps round `lo` and adds its
// partner's partial of it; the partner keeps `hi`.  Both sides add the same
// two numbers, the lower lane's first, as row_reduce does.
template <int W, typename R>
__device__ __forceinline__ R tile_combine(const R &lo, const R &hi, int o, int sub) {
  const bool up = (sub & o) != 0;
  const R keep = up ? hi : lo, send = up ? lo : hi;
  const R recv = tile_shfl<W>(send, o);
  return up ? recv + keep : keep + recv;
}

// The reduction tree over the W rounds of a tile, evaluated depth first: the
// rounds are visited in bit-reversed order and each pair is combined as soon
// as both are done, so at most log2(W) + 1 partials are live at a time.
// Rounds t0 + j O (j = 0, 1, ...) are the subtree below bit O.  round(t)
// returns this lane's partial of round t; it is called by every lane of the
// warp, and only for rounds that hold rows (t G < rows, warp-uniform).  The
// result: lane sub of a group holds round sub, i.e. row sub G + g of the tile.
template <int W, int O, typename R, typename F>
__device__ __forceinline__ R tile_tree(int t0, int rows, int sub, const F &round) {
  if constexpr (O == W) {
    return t0 * (32 / W) < rows ? round(t0) : R{};
  } else {
    const R lo = tile_tree<W, 2 * O, R>(t0, rows, sub, round);
    const R hi = tile_tree<W, 2 * O, R>(t0 + O, rows, sub, round);
    return tile_combine<W, R>(lo, hi, O, sub);
  }
}

// Warp-uniform trip count of round t: the largest number of entries a lane
// of the warp has in its row [rb, re) (entries rb + sub + j W).
template <int W>
__device__ __forceinline__ int tile_nmax(int64_t rb, int64_t re, int sub) {
  const int cnt = (int)((re - rb - sub + W - 1) / W);  // >= 0
  return __reduce_max_sync(0xffffffffu, cnt);
}

// Row sums of the tile of `rows` (<= 32) rows starting at `base`: lane l gets
// the off-diagonal sum of row base + tile_own_row<W>(l) (0 past `rows`).  Every
// lane of the warp must call it with the same base and rows.
template <int W, int U, typename MT, typename VT>
__device__ __forceinline__ VT tile_row_sums(int64_t base, int rows, const int64_t *__restrict__ ptr,
                                            const int32_t *__restrict__ col,
                                            const MT *__restrict__ val, const VT *__restrict__ x) {
  const int lane = threadIdx.x & 31, sub = lane % W;
  const int own = tile_own_row<W>(lane);
  int64_t b = 0, e = 0;  // row extents, one coalesced load per lane
  if (own < rows) {
    b = __ldg(ptr + base + own);
    e = __ldg(ptr + base + own + 1);
  }
  return tile_tree<W, 1, VT>(0, rows, sub, [&](int t) -> VT {
    // round t's row of group g has its extents in lane g W + t
    const int64_t rb = __shfl_sync(0xffffffffu, b, t, W);
    const int64_t re = __shfl_sync(0xffffffffu, e, t, W);
    return row_dot_n<W, U, MT, VT>(rb, re, col, val, x, sub, tile_nmax<W>(rb, re, sub));
  });
}

// Chebyshev iteration coefficients on [lo, hi] (Saad, Iterative Methods,
// Alg. 12.1): the first step scales by 1/theta, step k >= 1 uses
// d = c1[k] d + c2[k] D^{-1} res.  Computed once per interval (host, or one
// thread) rather than per thread: an FP64 division costs tens of FP64-pipe
// operations, and the FP64 pipe is narrow on this part.
constexpr int kChebMaxDeg = 48;
struct ChebCoef {
  int degree;        // number of steps (the requested degree, clamped to [1, kChebMaxDeg])
  double inv_theta;  // 1 / theta, theta = (hi + lo) / 2
  double c1[kChebMaxDeg], c2[kChebMaxDeg];
};
// A collapsed interval means D^{-1} A = I (no off-diagonal coupling): the
// first (Jacobi) step is then exact and the recurrence is undefined, so the
// later steps get c1 = c2 = 0 (d = 0, z unchanged).  The number of steps never
// depends on the data, so a captured launch sequence stays valid.
__host__ __device__ inline void cheb_coefficients(int degree, double lo, double hi,
                                                  ChebCoef *cf) {
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
  const bool collapsed = !(delta > 1e-12 * theta);
  if (degree > kChebMaxDeg) degree = kChebMaxDeg;
  if (degree < 1) degree = 1;
  cf->degree = degree;
  cf->inv_theta = 1.0 / theta;
  const double sigma1 = collapsed ? 1.0 : theta / delta;
  double rho0 = 1.0 / sigma1;
  cf->c1[0] = 0.0;
  cf->c2[0] = cf->inv_theta;
  for (int k = 1; k < degree; ++k) {
    if (collapsed) {
      cf->c1[k] = 0.0;
      cf->c2[k] = 0.0;
      continue;
    }
    const double rho1 = 1.0 / (2.0 * sigma1 - rho0);
    cf->c1[k] = rho1 * rho0;
    cf->c2[k] = 2.0 * rho1 / delta;
    rho0 = rho1;
  }
}

// Fusions at the two ends of an AMG preconditioner application on the finest
// level (launches saved per CG iteration).
// FineInit: the zero-guess smoother start of the finest level
// (cheb_init_zero_kernel's arithmetic) fused into the CG update, in the
// V-cycle's precision IT; r_lo receives the narrowed residual when the V-cycle
// runs in FP32 (else nullptr).  d == nullptr: no fusion.
template <typename IT>
struct FineInit {
  IT *r_lo;
  const IT *invdiag;
  const ChebCoef *cf;
  IT *d, *z;
};
// DotFuse: the preconditioned inner product rho = (r, z) and beta -- for the
// flexible variant (r, z) - (r, z_old) with z widened from the FP32 V-cycle
// into z64, whose old contents are z_old -- fused into the last V-cycle sweep.
struct DotFuse {
  int first;  // first CG inner product (no beta)
  int flex;   // flexible (mixed) variant
  const double *r;
  double *z64;
  Scalars *sc;
  double *partials;
};

// Vectors of the CG with the V-cycle's product (fine_post_smooth = 0), in the
// hierarchy's precision T: residual r, preconditioned residual z, w = B z,
// direction p and q = B p, the finest level's smoother start zpre, and the
// finest level's 1 / diagonal in T.  The iterate x and b stay FP64.
template <typename T>
struct FcgSet {
  T *r, *z, *w, *p, *q, *zpre;
  const T *invdiag;
};
struct FcgVecs {
  FcgSet<double> f64;
  FcgSet<float> f32;
  const ChebCoef *cf;  // the finest level's smoother coefficients (zpre = cf->inv_theta D^{-1} r)
};

// Chebyshev coefficient slots of a handle (device array): slot 0 belongs to
// the fine-level Chebyshev preconditioner, slot 1 + l to AMG level l (its
// smoother, or the coarse solve on the last level).
constexpr int kChebSlots = 1 + 32;

// Row-group shape of the SpMV-class kernels: W lanes per row, U loads in flight
// per lane.  A lane sums its entries (beg + sub + j W, j = 0, 1, ...) in
// increasing j whatever U is, so results depend on W only.  W follows from the
// mean row length (deterministic); U may be picked by the autotuner.
struct RowShape {
  int W, U;
};
// W = 4 lanes per row: loads stay sector-coalesced (4 x 8 B = one 32 B sector
// per row per instruction) while the FP64 reduction costs W - 1 = 3 adds per
// lane and tile (tile_row_sums) -- on GB300 the FP64 pipe, not HBM, limits a
// wide-warp CSR sweep.  Very long rows (coarse AMG levels) use 8 lanes.
__host__ inline int lanes_for_mean(double mean) { return mean <= 160 ? 4 : 8; }
// U = 4: with row tiles the sweeps are FP64-pipe-bound before they are
// latency-bound, and U = 4 keeps them at 48 registers (5 resident blocks per SM
// instead of 4 at U = 8); on the 64^3 and 128^3 operators it is 2-3 % faster.
__host__ inline RowShape shape_for_mean(double mean) {
  return {lanes_for_mean(mean), 4};
}
// Grid of a row-tile sweep (W lanes per row, kBlock threads per block): one
// wave of sweep_min_blocks(U) resident blocks per SM at most (the sweeps are
// compiled with that register cap); warp_rows splits the rows over its warps.
__host__ inline int row_grid_blocks(int num_sms, int64_t n, int W, int blocks_per_sm) {
  int64_t g = ceil_div(n > 0 ? n : 1, kBlock / W);
  int64_t cap = (int64_t)num_sms * blocks_per_sm;
  return (int)(g < cap ? g : cap);
}
__host__ inline int row_grid(int num_sms, int64_t n, int W, int U) {
  return row_grid_blocks(num_sms, n, W, sweep_min_blocks(U));
}

// Launch CALL with constexpr W and U set to the supported row-group shape:
// W in {4, 8}; U in {4, 8}.
#define SPH_DISPATCH_SHAPE(W_, U_, CALL)            \
  do {                                              \
    if ((W_) <= 4) {                                \
      if ((U_) <= 4) {                              \
        constexpr int W = 4, U = 4;                 \
        CALL;                                       \
      } else {                                      \
        constexpr int W = 4, U = 8;                 \
        CALL;                                       \
      }                                             \
    } else {                                        \
      if ((U_) <= 4) {                              \
        constexpr int W = 8, U = 4;                 \
        CALL;                                       \
      } else {                                      \
        constexpr int W = 8, U = 8;                 \
        CALL;                                       \
      }                                             \
    }                                               \
  } while (0)

// A CSR operator as seen by the SpMV-shaped kernels: off-diagonal entries in
// (ptr, col, val) and the diagonal apart.  (W, U) = row-group shape.
template <typename T>
struct CsrView {
  int64_t n = 0;
  const int64_t *ptr = nullptr;
  const int32_t *col = nullptr;
  const T *val = nullptr;
  const T *diag = nullptr;
  const T *invdiag = nullptr;
  int64_t nnz = 0;
  int W = 32;
  int U = 4;
};

}  // namespace sphrt

// --------------------------------------------------------------------------
// Internal handle.
// --------------------------------------------------------------------------
struct SphLevel;  // AMG level (amg.cu)

struct sph_rt {
  sph_rt_config cfg;
  std::string err;
  int64_t launches = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool cuda_ready = false;
  int num_sms = 152;
  std::vector<void *> allocs;  // device allocations of the current particle set
  std::unordered_map<void *, size_t> alloc_size;
  std::multimap<size_t, void *> pool;  // released buffers kept for reuse

  // sizes
  bool have_particles = false;
  bool have_operator = false;
  int64_t n = 0, n_int = 0;
  int64_t nnz_nbr = 0, nnz_mat = 0, nnz_gh = 0;
  int dim = 3;

  // permutation
  int64_t *slot2caller = nullptr;  // [n]
  int64_t *caller2slot = nullptr;  // [n]

  // particle data, slot order
  double *px = nullptr, *py = nullptr, *pz = nullptr;
  double *mass = nullptr, *rho = nullptr, *h = nullptr, *sigma0 = nullptr;
  double *V = nullptr, *invV = nullptr;
  int32_t *kind = nullptr;      // [n]
  int32_t *copysrc = nullptr;   // [n] slot of the copied interior particle, else -1
  double *e = nullptr, *E = nullptr;  // state [n] (ghost entries hold ghost values)

  // neighbour lists (interior rows)
  int64_t *nbr_ptr = nullptr;  // [n_int + 1]
  int32_t *nbr_col = nullptr;  // slot of the neighbour
  double *nbr_F = nullptr;     // F_ij = W'(r)/r, two-h average
  int32_t *gcol = nullptr;     // slot whose E neighbour k carries (copy ghosts: the copied one)
  double *gvx = nullptr, *gvy = nullptr, *gvz = nullptr;  // V_j F_ij x_ij (limiter only)

  // operator B = V A (interior rows; unknown index == slot)
  int64_t *mat_ptr = nullptr;
  int32_t *mat_col = nullptr;
  double *mat_G = nullptr;     // V_i V_j F_ij
  double *mat_val = nullptr;   // B_ij of the current step
  float *mat_val32 = nullptr;  // FP32 copy for the mixed form (written by the assembly)
  float *diag32 = nullptr, *invdiag32 = nullptr;
  double *diag = nullptr, *invdiag = nullptr;
  int64_t *gh_ptr = nullptr;   // Dirichlet-ghost couplings
  int32_t *gh_slot = nullptr;
  double *gh_W = nullptr;      // V_j F_ij
  double *gb = nullptr;        // unscaled Dirichlet coupling sum_j w_ij E_j

  // material data of the step, slot order [n]
  double *T = nullptr, *sigma = nullptr, *f = nullptr, *R = nullptr, *lambda = nullptr,
         *D = nullptr;

  // step vectors (interior)
  double *e_old = nullptr, *E_old = nullptr, *e_l = nullptr, *E_l = nullptr;
  double *e_new = nullptr;
  double *Qe = nullptr, *QE = nullptr;  // slot order [n]
  double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr,
         *w = nullptr;
  double *z_old = nullptr;  // previous preconditioned residual (flexible CG)
  double *tmp_n = nullptr;   // [n] staging for caller-order transfers
  double *tmp_n2 = nullptr;  // [n] staging / Chebyshev scratch
  double *tmp_n3 = nullptr;
  double *e_bak = nullptr, *E_bak = nullptr;  // [n] state at the start of the step
  double *stage_ge = nullptr, *stage_gE = nullptr;  // [n] ghost values staged from the host

  // reductions
  sphrt::Scalars *sc = nullptr;  // device
  sphrt::Scalars *sc_host = nullptr;  // pinned mirror
  double *partials = nullptr;    // [8 * kMaxRedBlocks]

  // AMG hierarchy and Chebyshev data
  std::vector<SphLevel *> levels;
  bool amg_ready = false;
  int coarse_smem_optin = 0;                 // shared-memory opt-in done (bit per value type)
  int tail_level = 0;    // first AMG level of the cluster-resident V-cycle tail (0 = none)
  int tail_cluster = 0;  // thread blocks in the tail's cluster
  double *gersh = nullptr;                   // device scalar written by the assembly
  double *amg_gersh = nullptr;               // per-level Gershgorin bounds
  sphrt::ChebCoef *cheb_slots = nullptr;     // device [kChebSlots] (see kChebSlots)

  // device-driven outer loop: one CUDA graph with conditional WHILE nodes
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<uint64_t> graph_sig;  // launch parameters the graph was captured with
  cudaStream_t cap_stream = nullptr;
  int64_t graph_l_init = 0, graph_l_outer = 0, graph_l_inner = 0;  // kernels per part
  int64_t graph_builds = 0, graph_launches = 0;

  // row-group shape of the fine SpMV-class kernels (autotuned or from the mean row length)
  sphrt::RowShape fine_shape{16, 6};
  // extrapolated Krylov start (config.krylov_start = p > 0).  Between steps E_old
  // holds E^{n-2} (the last step's start) and E_hist[j] E^{n-3-j}; during a step
  // E_hist[j] holds E^{n-2-j}.  hist counts the consecutive converged steps of
  // this particle set (capped at 3), dt_hist[j] the sizes of the last ones.
  double *E_hist[3] = {nullptr, nullptr, nullptr};
  int hist = 0;
  double dt_hist[3] = {0.0, 0.0, 0.0};
  bool fine_shape_set = false;
  int64_t fine_shape_n = 0, fine_shape_nnz = 0;  // sizes the shape was tuned on
  // solver autotuner (config.autotune): done once per handle; its trials
  bool solver_tuned = false;
  std::vector<sph_rt_tune_trial> tune_trials;

  // kernel timing
  std::vector<cudaEvent_t> ev_pool;
  std::vector<double> ev_bytes;   // bytes of each event pair
  std::vector<int> ev_kind;       // kernel kind of each event pair (sphrt::TimedKind)
  int *ev_flags = nullptr;        // device: work flag of each event pair
  // timing gate: with kernel_timing the stream is held by gate_kernel until a
  // whole chunk of the solve is queued, so that the timed kernels run back to
  // back and an event pair measures the kernel, not the host's launch latency
  volatile int *gate_host = nullptr;  // mapped pinned word written by the host
  int *gate_dev = nullptr;            // its device address
  int gate_epoch = 0;
  int ev_used = 0;
  int64_t spmv_launches = 0;
  double spmv_ms = 0.0, spmv_bytes = 0.0;
  int64_t kind_launches[5] = {0, 0, 0, 0, 0};  // per sphrt::TimedKind
  double kind_ms[5] = {0, 0, 0, 0, 0}, kind_bytes[5] = {0, 0, 0, 0, 0};
};

// Helpers shared by the translation units (defined in sph_rt.cu).
namespace sphrt {
sph_rt_status set_error(sph_rt *s, sph_rt_status st, const std::string &msg);
bool cuda_ok(sph_rt *s, cudaError_t e, const char *what);
void *dalloc_bytes(sph_rt *s, size_t bytes);  // tracked cudaMalloc; nullptr on failure
template <typename T>
inline T *dalloc(sph_rt *s, size_t count) {
  return static_cast<T *>(dalloc_bytes(s, sizeof(T) * (count > 0 ? count : 1)));
}
void free_all(sph_rt *s);
void dfree(sph_rt *s, void *p);  // back to the free list (stream-ordered users must sync first)
// CUDA-event bracketing of fine-operator SpMV-class launches (config.kernel_timing).
// timing_begin returns the work flag of the launch (nullptr when timing is off):
// the kernel writes 1 there if it does work and 0 if it returns at once because
// the solve has converged; only launches that worked are counted.
// kinds of timed fine-operator launches (SPH_RT_KERNEL_* in sph_rt.h)
enum TimedKind { kTimedSpmvPQ = 0, kTimedResid = 1, kTimedCheb = 2, kTimedPost = 3,
                 kTimedTrueResid = 4 };
constexpr int kTimedKinds = 5;
int *timing_begin(sph_rt *s);
void timing_end(sph_rt *s, double bytes, int kind);
void timing_flush(sph_rt *s);
__device__ __forceinline__ void mark_work(int *wflag, int worked) {
  if (wflag && blockIdx.x == 0 && threadIdx.x == 0) *wflag = worked;
}
}  // namespace sphrt

// Host-side phase trace to stderr, enabled by the environment variable
// SPH_RT_TRACE=1 (diagnostics only; off by default).
namespace sphrt {
bool trace_enabled();
}
#define SPH_TRACE(...)                                \
  do {                                                \
    if (sphrt::trace_enabled()) {                     \
      fprintf(stderr, "[sphrt] " __VA_ARGS__);        \
      fputc('\n', stderr);                            \
      fflush(stderr);                                 \
    }                                                 \
  } while (0)

#define SPH_CUDA(s, call)                                          \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) {                                       \
      sphrt::cuda_ok((s), e_, #call);                              \
      return SPH_RT_EDEVICE;                                       \
    }                                                              \
  } while (0)

#define SPH_LAUNCHED(s)                                            \
  do {                                                             \
    (s)->launches++;                                               \
    cudaError_t e_ = cudaGetLastError();                           \
    if (e_ != cudaSuccess) {                                       \
      sphrt::cuda_ok((s), e_, "kernel launch");                    \
      return SPH_RT_EDEVICE;                                       \
    }                                                              \
  } while (0)

namespace sphrt {

// Programmatic dependent launch.  A kernel launched with pdl_launch may be
// launched while the previous kernel on the stream drains (its last blocks
// finishing, its writes being flushed); every such kernel calls pdl_wait() as
// its first statement, which returns once the previous kernel has completed
// and its writes are visible (at once for a kernel launched the ordinary way).
// Since every kernel of the chain waits before it does anything, each one still
// completes after all earlier ones.  (Allowing the next launch early, right
// after the wait, measured no faster and is not done.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch `kernel` on the handle's stream, with programmatic dependent launch
// when the configuration asks for it.  The caller checks with SPH_LAUNCHED.
template <typename... KP, typename... A>
inline void pdl_launch(const sph_rt *s, void (*kernel)(KP...), dim3 grid, dim3 block, size_t smem,
                       A... args) {
  cudaLaunchConfig_t lc;
  memset(&lc, 0, sizeof lc);
  lc.gridDim = grid;
  lc.blockDim = block;
  lc.dynamicSmemBytes = smem;
  lc.stream = s->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = attr;
  lc.numAttrs = s->cfg.pdl ? 1 : 0;
  cudaLaunchKernelEx(&lc, kernel, args...);
}

}  // namespace sphrt
