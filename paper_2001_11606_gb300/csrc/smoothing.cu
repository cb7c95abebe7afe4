// smoothing.cu -- smoothing lengths by the initialisation iteration of
// Sec. 3.1 of the paper: the support radius of every interior point is set to
// eta local point spacings (eta = 4 in the paper).
//
// The iteration works on the zeroth moment of the kernel,
//   S_i(h) = sum_j W(r_ij, h)   (all j within the support, i itself included),
// the SPH number density: for points of spacing dx, S = dx^-d, so
// (h^d S_i(h))^(1/d) estimates h / dx.  With s the support radius in units of h
// (2: cubic B-spline, 1: Wendland C4) the target is h / dx = eta / s, and every
// interior point is updated by
//   h_i <- h_i (eta / s) / (h_i^d S_i(h_i))^(1/d),  bounded to [h_i / 2, 2 h_i],
// until |dh_i| <= tol h_i or max_iter updates.  S_i depends on h_i alone, so a
// warp runs one point's whole iteration.  Copy ghosts then take the h of the
// point they copy; Dirichlet ghosts keep theirs.
//
// Candidates come from a uniform grid whose cells cover the support of any h
// up to a cap H; an update that would exceed H stops at H and the round is
// repeated with a coarser grid (at most kRounds rounds).  The membership test
// is the exact FP64 one of the neighbour search (r^2 summed in coordinate
// order without fused multiply-add, strict <), and every cell lists its
// members in slot order, so the sums are deterministic.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "common.cuh"

namespace sphrt {

sph_rt_status exclusive_scan(sph_rt *s, const int64_t *in, int64_t n, int64_t *out);

namespace {

constexpr int kRounds = 6;
// Largest number of points a grid cell may hold.  Cells cover the support of
// the largest h, so this bounds the candidates per point; starting h many times
// the point spacing would make the per-cell sort and the gathers quadratic.
constexpr unsigned kMaxCellPoints = 4096;

struct HGrid {
  double lo[3];
  double cell, inv_cell;
  int nc[3];
  int dim;
};

__device__ __forceinline__ int hcell(double x, double lo, double inv, int nc) {
  int c = (int)floor((x - lo) * inv);
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__device__ __forceinline__ int64_t hkey(const HGrid &g, int cx, int cy, int cz) {
  return ((int64_t)cz * g.nc[1] + cy) * g.nc[0] + cx;
}

__global__ void hkey_kernel(HGrid g, const double *px, const double *py, const double *pz,
                            int64_t n, int64_t *key, unsigned *count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = hkey(g, hcell(px[i], g.lo[0], g.inv_cell, g.nc[0]),
                           hcell(py[i], g.lo[1], g.inv_cell, g.nc[1]),
                           hcell(pz[i], g.lo[2], g.inv_cell, g.nc[2]));
    key[i] = k;
    atomicAdd(&count[k], 1u);
  }
}

// counts widened to int64 for the scan; the largest count goes to *most
__global__ void hcount64_kernel(int64_t n, const unsigned *in, int64_t *out, unsigned *most) {
  unsigned m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    out[i] = in[i];
    m = in[i] > m ? in[i] : m;
  }
  if (m) atomicMax(most, m);
}

__global__ void hscatter_kernel(int64_t n, const int64_t *key, const int64_t *start,
                                unsigned *cursor, int32_t *member) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = key[i];
    member[start[k] + atomicAdd(&cursor[k], 1u)] = (int32_t)i;
  }
}

// members of each cell in slot order (the scatter above is in arrival order)
__global__ void hsort_kernel(int64_t ncell, const int64_t *start, int32_t *member) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    int32_t *a = member + start[c];
    const int64_t m = start[c + 1] - start[c];
    for (int64_t t = 1; t < m; ++t) {
      const int32_t v = a[t];
      int64_t u = t - 1;
      while (u >= 0 && a[u] > v) {
        a[u + 1] = a[u];
        --u;
      }
      a[u + 1] = v;
    }
  }
}

__device__ __forceinline__ double hr2(double xi, double yi, double zi, double xj, double yj,
                                      double zj) {
  const double dx = __dsub_rn(xi, xj), dy = __dsub_rn(yi, yj), dz = __dsub_rn(zi, zj);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// W(r, h): cubic B-spline (support 2h) or Wendland C4 (support h), each
// normalised to a unit volume integral in dim dimensions (Sec. 2.3-2.4).
__device__ __forceinline__ double kernel_w(int kern, int dim, double r, double h) {
  const double pi = 3.141592653589793;
  const double q = r / h;
  double hd = h;
  if (dim >= 2) hd *= h;
  if (dim >= 3) hd *= h;
  if (kern == SPH_RT_WENDLAND_C4) {
    const double k = dim == 3 ? 45.0 / (4.0 * pi) : (dim == 2 ? 36.0 / (5.0 * pi) : 1.5);
    if (q > 1.0) return 0.0;
    const double t = 1.0 - q, t2 = t * t;
    return (k / hd) * (t2 * t2 * t) * (8.0 * q * q + 5.0 * q + 1.0);
  }
  const double k = dim == 3 ? 1.0 / pi : (dim == 2 ? 10.0 / (7.0 * pi) : 2.0 / 3.0);
  if (q < 1.0) return (k / hd) * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
  if (q < 2.0) {
    const double t = 2.0 - q;
    return (k / hd) * 0.25 * t * t * t;
  }
  return 0.0;
}

struct HIter {
  int kern;
  double support;  // support radius in units of h
  double target;   // eta / support
  double tol;
  double cap;      // largest h this round's grid covers
  int max_iter;
};

// One warp per interior slot: the point's whole iteration.  flags[0]: an update
// stopped at the cap; flags[1]: the largest number of updates.
__global__ void h_iterate_kernel(HGrid g, HIter it, int64_t n_int, const double *px,
                                 const double *py, const double *pz, const int64_t *start,
                                 const int32_t *member, double *h, int *flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int ncells = g.dim == 3 ? 27 : (g.dim == 2 ? 9 : 3);
  for (int64_t i = warp; i < n_int; i += nwarps) {
    const double xi = px[i], yi = py[i], zi = pz[i];
    const int c[3] = {hcell(xi, g.lo[0], g.inv_cell, g.nc[0]),
                      hcell(yi, g.lo[1], g.inv_cell, g.nc[1]),
                      hcell(zi, g.lo[2], g.inv_cell, g.nc[2])};
    double hi = h[i];
    int k = 0;
    bool capped = false;
    while (k < it.max_iter) {
      const double cut = it.support * hi, cut2 = __dmul_rn(cut, cut);
      double part = 0.0;
      for (int q = 0; q < ncells; ++q) {
        const int o[3] = {q % 3 - 1, (q / 3) % 3 - 1, q / 9 - 1};
        int cc[3];
        bool ok = true;
        for (int d = 0; d < 3; ++d) {
          cc[d] = d < g.dim ? c[d] + o[d] : 0;
          if (d < g.dim && (cc[d] < 0 || cc[d] >= g.nc[d])) ok = false;
        }
        if (!ok) continue;
        const int64_t key = hkey(g, cc[0], cc[1], cc[2]);
        const int64_t b = start[key], e = start[key + 1];
        for (int64_t m = b + lane; m < e; m += 32) {
          const int32_t j = member[m];
          if (j == i) continue;
          const double r2 = hr2(xi, yi, zi, px[j], py[j], pz[j]);
          if (r2 < cut2) part += kernel_w(it.kern, g.dim, sqrt(r2), hi);
        }
      }
      const double S = warp_sum(part) + kernel_w(it.kern, g.dim, 0.0, hi);
      // lane 0 holds the sum; every lane takes the update from it
      const double Sall = __shfl_sync(0xffffffffu, S, 0);
      const double ratio = pow(pow(hi, (double)g.dim) * Sall, 1.0 / g.dim);
      double hn = hi * it.target / ratio;
      if (hn > 2.0 * hi) hn = 2.0 * hi;
      if (hn < 0.5 * hi) hn = 0.5 * hi;
      if (hn > it.cap) {
        hn = it.cap;
        capped = true;
      }
      ++k;
      const double change = fabs(hn - hi);
      hi = hn;
      if (capped || change <= it.tol * hi) break;
    }
    if (lane == 0) {
      h[i] = hi;
      if (capped) atomicOr(&flags[0], 1);
      atomicMax(&flags[1], k);
    }
  }
}

__global__ void h_copy_ghost_kernel(int64_t n_int, int64_t n, const int32_t *kind,
                                    const int32_t *copysrc, double *h) {
  for (int64_t i = n_int + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (kind[i] == SPH_RT_COPY) h[i] = h[copysrc[i]];
}

__global__ void h_max_kernel(int64_t n, const double *h, unsigned long long *out) {
  double m = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, h[i]);
  m = warp_max(m);
  // h > 0: the bit pattern orders like the value
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void h_bbox_kernel(int64_t n, const double *px, const double *py, const double *pz,
                              unsigned long long *lo_hi) {
  // lo_hi[0..2]: order-preserving keys of -min, lo_hi[3..5]: of max
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double c[3] = {px[i], py[i], pz[i]};
    for (int d = 0; d < 3; ++d) {
      for (int side = 0; side < 2; ++side) {
        const double v = side == 0 ? -c[d] : c[d];
        // order-preserving map of a double to an unsigned key
        unsigned long long u = (unsigned long long)__double_as_longlong(v);
        u = (u >> 63) ? ~u : (u | 0x8000000000000000ull);
        atomicMax(&lo_hi[side * 3 + d], u);
      }
    }
  }
}

__host__ inline double key_to_double(unsigned long long u) {
  u = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
  double v;
  memcpy(&v, &u, sizeof v);
  return v;
}

int grid_blocks(const sph_rt *s, int64_t n) {
  int64_t g = ceil_div(n > 0 ? n : 1, kBlock), cap = (int64_t)s->num_sms * 8;
  return (int)(g < cap ? g : cap);
}

}  // namespace

// Iterate the smoothing lengths of the current particle set (slot order, in
// s->h) on the device.  *iters: the largest number of updates of a point.
sph_rt_status smoothing_iterate(sph_rt *s, double eta, double tol, int max_iter, int *iters) {
  const int64_t n = s->n, n_int = s->n_int;
  cudaStream_t st = s->stream;
  const int kern = s->cfg.kernel;
  const double support = kern == SPH_RT_WENDLAND_C4 ? 1.0 : 2.0;
  unsigned long long *scal = dalloc<unsigned long long>(s, 8);
  int *flags = dalloc<int>(s, 2);
  if (!scal || !flags) return SPH_RT_ENOMEM;
  SPH_CUDA(s, cudaMemsetAsync(scal, 0, 8 * sizeof(unsigned long long), st));
  h_bbox_kernel<<<grid_blocks(s, n), kBlock, 0, st>>>(n, s->px, s->py, s->pz, scal);
  SPH_LAUNCHED(s);
  unsigned long long hb[8];
  SPH_CUDA(s, cudaMemcpyAsync(hb, scal, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  SPH_CUDA(s, cudaStreamSynchronize(st));
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = -key_to_double(hb[d]);
    hi[d] = key_to_double(hb[3 + d]);
  }
  int most = 0;
  sph_rt_status rc = SPH_RT_OK;
  for (int round = 0; round < kRounds; ++round) {
    SPH_CUDA(s, cudaMemsetAsync(scal, 0, sizeof(unsigned long long), st));
    h_max_kernel<<<grid_blocks(s, n_int), kBlock, 0, st>>>(n_int, s->h, scal);
    SPH_LAUNCHED(s);
    unsigned long long hm_bits = 0;
    SPH_CUDA(s, cudaMemcpyAsync(&hm_bits, scal, sizeof hm_bits, cudaMemcpyDeviceToHost, st));
    SPH_CUDA(s, cudaStreamSynchronize(st));
    double hmax;
    memcpy(&hmax, &hm_bits, sizeof hmax);
    // this round covers any h up to 1.25 max h (larger steps take another round)
    HIter it = {kern, support, eta / support, tol, 1.25 * hmax, max_iter};
    HGrid g;
    g.dim = s->dim;
    g.cell = support * it.cap * (1.0 + 1e-9);
    g.inv_cell = 1.0 / g.cell;
    int64_t ncell = 1;
    for (int d = 0; d < 3; ++d) {
      g.lo[d] = lo[d];
      g.nc[d] = d < g.dim ? (int)((hi[d] - lo[d]) / g.cell) + 1 : 1;
      ncell *= g.nc[d];
    }
    if (ncell > ((int64_t)1 << 30))
      return set_error(s, SPH_RT_EINVAL, "smoothing-length grid too large for the point extent");
    int64_t *key = dalloc<int64_t>(s, n);
    unsigned *cnt = dalloc<unsigned>(s, ncell), *cur = dalloc<unsigned>(s, ncell);
    int64_t *cnt64 = dalloc<int64_t>(s, ncell), *start = dalloc<int64_t>(s, ncell + 1);
    int32_t *member = dalloc<int32_t>(s, n);
    if (!key || !cnt || !cur || !cnt64 || !start || !member) return SPH_RT_ENOMEM;
    SPH_CUDA(s, cudaMemsetAsync(cnt, 0, sizeof(unsigned) * ncell, st));
    SPH_CUDA(s, cudaMemsetAsync(cur, 0, sizeof(unsigned) * ncell, st));
    SPH_CUDA(s, cudaMemsetAsync(flags, 0, 2 * sizeof(int), st));
    hkey_kernel<<<grid_blocks(s, n), kBlock, 0, st>>>(g, s->px, s->py, s->pz, n, key, cnt);
    SPH_LAUNCHED(s);
    unsigned *most_dev = reinterpret_cast<unsigned *>(flags + 1);  // reset below
    SPH_CUDA(s, cudaMemsetAsync(most_dev, 0, sizeof(unsigned), st));
    hcount64_kernel<<<grid_blocks(s, ncell), kBlock, 0, st>>>(ncell, cnt, cnt64, most_dev);
    SPH_LAUNCHED(s);
    unsigned most_cell = 0;
    SPH_CUDA(s, cudaMemcpyAsync(&most_cell, most_dev, sizeof most_cell, cudaMemcpyDeviceToHost, st));
    SPH_CUDA(s, cudaStreamSynchronize(st));
    if (most_cell > kMaxCellPoints)
      return set_error(s, SPH_RT_EINVAL,
                       "starting smoothing lengths too large for the point spacing (more than " +
                           std::to_string(kMaxCellPoints) + " points within one support)");
    SPH_CUDA(s, cudaMemsetAsync(most_dev, 0, sizeof(unsigned), st));
    if ((rc = exclusive_scan(s, cnt64, ncell, start))) return rc;
    hscatter_kernel<<<grid_blocks(s, n), kBlock, 0, st>>>(n, key, start, cur, member);
    SPH_LAUNCHED(s);
    hsort_kernel<<<grid_blocks(s, ncell), kBlock, 0, st>>>(ncell, start, member);
    SPH_LAUNCHED(s);
    const int gw = (int)(ceil_div(n_int, kWarpsPerBlock) < (int64_t)s->num_sms * 8
                             ? ceil_div(n_int, kWarpsPerBlock)
                             : (int64_t)s->num_sms * 8);
    h_iterate_kernel<<<gw, kBlock, 0, st>>>(g, it, n_int, s->px, s->py, s->pz, start, member,
                                            s->h, flags);
    SPH_LAUNCHED(s);
    int hf[2] = {0, 0};
    SPH_CUDA(s, cudaMemcpyAsync(hf, flags, sizeof hf, cudaMemcpyDeviceToHost, st));
    SPH_CUDA(s, cudaStreamSynchronize(st));
    dfree(s, key);
    dfree(s, cnt);
    dfree(s, cur);
    dfree(s, cnt64);
    dfree(s, start);
    dfree(s, member);
    most = hf[1] > most ? hf[1] : most;
    if (!hf[0]) break;  // no point was held at the cap
    if (round + 1 == kRounds)
      return set_error(s, SPH_RT_ENOTCONV, "smoothing lengths still growing after the last grid");
  }
  if (n > n_int) {
    h_copy_ghost_kernel<<<grid_blocks(s, n - n_int), kBlock, 0, st>>>(n_int, n, s->kind,
                                                                      s->copysrc, s->h);
    SPH_LAUNCHED(s);
  }
  SPH_CUDA(s, cudaStreamSynchronize(st));
  dfree(s, scal);
  dfree(s, flags);
  *iters = most;
  return SPH_RT_OK;
}

}  // namespace sphrt
