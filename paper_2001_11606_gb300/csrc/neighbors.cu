// neighbors.cu -- Morton-sorted cell list, neighbour search and operator
// sparsity (rows a1-a2 of the hot path).
//
// Connectivity is the set of j != i with r_ij^2 < (s max(h_i, h_j))^2 for every
// interior particle i, s the kernel's support in units of h (2 for the cubic
// B-spline, 1 for the paper's Wendland C4 kernel; connectivity in the sense of
// Sec. 1 and Sec. 3.1 of the paper).  Distances are formed with
// explicit round-to-nearest double operations (no fused multiply-add) in the
// order dx*dx + dy*dy + dz*dz, so the neighbour sets are bit-identical to a
// host evaluation of the same expression.
//
// Layout: particles are sorted by key = (ghost flag, Morton code of the cell)
// with ties broken by caller index, giving "slots" with interior particles
// first.  Cells have edge >= s max h, so all neighbours of a particle lie in
// the 3^d cells around its own.  Two cell lists give the same slots: a dense
// table over all keys (counting sort, up to 2^27 keys), and for larger grids
// 64-bit keys with a stable radix sort, the occupied cells by run length and
// a hash table from cell key to cell (up to 2^58 cells).
#include <cuda_runtime.h>

#include "common.cuh"

namespace sphrt {

// --------------------------------------------------------------------------
// Exclusive scan of int64 counts: out[0..n] with out[n] = total.
// --------------------------------------------------------------------------
constexpr int kScanItems = 8;
constexpr int kScanTile = kBlock * kScanItems;

__global__ void scan_tile_sums(const int64_t *in, int64_t n, int64_t *tile_sums) {
  __shared__ int64_t sh[kWarpsPerBlock];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t acc = 0;
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)k * kBlock + threadIdx.x;
    if (i < n) acc += in[i];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < kWarpsPerBlock; ++w) t += sh[w];
    tile_sums[blockIdx.x] = t;
  }
}

// Single block: exclusive scan of the tile sums in place (sequential chunks).
__global__ void scan_tile_offsets(int64_t *tile_sums, int64_t ntiles, int64_t *total) {
  __shared__ int64_t sh[kBlock];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < ntiles; base += kBlock) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < ntiles ? tile_sums[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kBlock; o <<= 1) {
      int64_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < ntiles) tile_sums[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += sh[kBlock - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void scan_tiles(const int64_t *in, int64_t n, const int64_t *tile_off, int64_t *out) {
  __shared__ int64_t sh[kBlock];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t local = 0;
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    v[k] = i < n ? in[i] : 0;
    local += v[k];
  }
  sh[threadIdx.x] = local;
  __syncthreads();
  for (int o = 1; o < kBlock; o <<= 1) {
    int64_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  int64_t run = tile_off[blockIdx.x] + sh[threadIdx.x] - local;
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
}

sph_rt_status exclusive_scan(sph_rt *s, const int64_t *in, int64_t n, int64_t *out) {
  int64_t ntiles = ceil_div(n > 0 ? n : 1, kScanTile);
  int64_t *tiles = dalloc<int64_t>(s, (size_t)ntiles);
  if (!tiles) return SPH_RT_ENOMEM;
  scan_tile_sums<<<(unsigned)ntiles, kBlock, 0, s->stream>>>(in, n, tiles);
  SPH_LAUNCHED(s);
  scan_tile_offsets<<<1, kBlock, 0, s->stream>>>(tiles, ntiles, out + n);
  SPH_LAUNCHED(s);
  scan_tiles<<<(unsigned)ntiles, kBlock, 0, s->stream>>>(in, n, tiles, out);
  SPH_LAUNCHED(s);
  dfree(s, tiles);  // reuse is stream-ordered after the scan
  return SPH_RT_OK;
}

// --------------------------------------------------------------------------
// Bounding box and largest smoothing length.
// --------------------------------------------------------------------------
__global__ void bbox_kernel(const double *px, const double *py, const double *pz,
                            const double *h, int64_t n, double *partials, unsigned *counter,
                            double *out /* lo[3], hi[3], hmax */) {
  double lo[3] = {1e308, 1e308, 1e308}, hi[3] = {-1e308, -1e308, -1e308}, hm = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double c[3] = {px[i], py[i], pz[i]};
    for (int d = 0; d < 3; ++d) {
      lo[d] = fmin(lo[d], c[d]);
      hi[d] = fmax(hi[d], c[d]);
    }
    hm = fmax(hm, h[i]);
  }
  // maxima of (-lo, hi, h)
  double part[7] = {-lo[0], -lo[1], -lo[2], hi[0], hi[1], hi[2], hm};
  // Exact reduction (values may be negative): per-block serial fold in thread 0.
  __shared__ double vals[kBlock][7];
  for (int k = 0; k < 7; ++k) vals[threadIdx.x][k] = part[k];
  __syncthreads();
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    double m[7];
    for (int k = 0; k < 7; ++k) m[k] = vals[0][k];
    for (int t = 1; t < (int)blockDim.x; ++t)
      for (int k = 0; k < 7; ++k) m[k] = fmax(m[k], vals[t][k]);
    for (int k = 0; k < 7; ++k) partials[k * gridDim.x + blockIdx.x] = m[k];
    __threadfence();
    unsigned ticket = atomicAdd(counter, 1u);
    am_last = ticket == gridDim.x - 1;
  }
  __syncthreads();
  if (am_last && threadIdx.x == 0) {
    __threadfence();
    double m[7];
    for (int k = 0; k < 7; ++k) m[k] = ((volatile double *)partials)[k * gridDim.x];
    for (unsigned b = 1; b < gridDim.x; ++b)
      for (int k = 0; k < 7; ++k) m[k] = fmax(m[k], ((volatile double *)partials)[k * gridDim.x + b]);
    for (int d = 0; d < 3; ++d) {
      out[d] = -m[d];
      out[3 + d] = m[3 + d];
    }
    out[6] = m[6];
    *counter = 0u;
  }
}

// --------------------------------------------------------------------------
// Morton codes
// --------------------------------------------------------------------------
__host__ __device__ inline uint64_t spread3(uint64_t v) {  // 21 bits -> every 3rd bit
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}
__host__ __device__ inline uint64_t spread2(uint64_t v) {  // 32 bits -> every 2nd bit
  v &= 0xffffffffull;
  v = (v | (v << 16)) & 0x0000ffff0000ffffull;
  v = (v | (v << 8)) & 0x00ff00ff00ff00ffull;
  v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0full;
  v = (v | (v << 2)) & 0x3333333333333333ull;
  v = (v | (v << 1)) & 0x5555555555555555ull;
  return v;
}

struct Grid {
  double lo[3];
  double inv_cell;
  double cell;     // cell edge (>= support max h)
  double support;  // kernel support in units of h: 2 (cubic B-spline) or 1 (Wendland C4)
  int nc[3];
  int dim;
  int ghost_shift;  // key bit that marks ghosts
  int kernel;       // SPH_RT_M4_SPLINE or SPH_RT_WENDLAND_C4
};

__device__ __forceinline__ int cell_coord(double x, double lo, double inv, int nc) {
  int c = (int)floor((x - lo) * inv);
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}
__device__ __forceinline__ uint64_t morton(const Grid &g, int cx, int cy, int cz) {
  if (g.dim == 3) return spread3((uint64_t)cx) | (spread3((uint64_t)cy) << 1) | (spread3((uint64_t)cz) << 2);
  if (g.dim == 2) return spread2((uint64_t)cx) | (spread2((uint64_t)cy) << 1);
  return (uint64_t)cx;
}

// hash of a cell key (sorted cell list), and the free-entry marker
constexpr unsigned long long kEmptyCell = ~0ull;
__host__ __device__ inline uint64_t cell_hash(uint64_t k) {  // splitmix64 finaliser
  k ^= k >> 30;
  k *= 0xbf58476d1ce4e5b9ull;
  k ^= k >> 27;
  k *= 0x94d049bb133111ebull;
  k ^= k >> 31;
  return k;
}

__global__ void key_kernel(Grid g, const double *px, const double *py, const double *pz,
                           const int32_t *kind, int64_t n, uint32_t *key, unsigned *count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int cx = cell_coord(px[i], g.lo[0], g.inv_cell, g.nc[0]);
    int cy = cell_coord(py[i], g.lo[1], g.inv_cell, g.nc[1]);
    int cz = cell_coord(pz[i], g.lo[2], g.inv_cell, g.nc[2]);
    uint32_t k = (uint32_t)morton(g, cx, cy, cz);
    if (kind[i] != SPH_RT_INTERIOR) k |= (1u << g.ghost_shift);
    key[i] = k;
    atomicAdd(&count[k], 1u);
  }
}

__global__ void u32_to_i64(const unsigned *in, int64_t n, int64_t *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

__global__ void scatter_kernel(const uint32_t *key, int64_t n, const int64_t *start,
                               unsigned *cursor, int64_t *slot2caller) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t k = key[i];
    int64_t pos = start[k] + atomicAdd(&cursor[k], 1u);
    slot2caller[pos] = i;
  }
}

// Order each key's slice by caller index (insertion sort; slices are small).
__global__ void segment_sort_kernel(const int64_t *start, const unsigned *count, int64_t nkeys,
                                    int64_t *slot2caller) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nkeys;
       k += (int64_t)gridDim.x * blockDim.x) {
    unsigned c = count[k];
    if (c < 2) continue;
    int64_t *a = slot2caller + start[k];
    for (unsigned t = 1; t < c; ++t) {
      int64_t v = a[t];
      int u = (int)t - 1;
      while (u >= 0 && a[u] > v) {
        a[u + 1] = a[u];
        --u;
      }
      a[u + 1] = v;
    }
  }
}

// --------------------------------------------------------------------------
// Sorted-key cell list (grids beyond the dense key table)
// --------------------------------------------------------------------------
__global__ void key64_kernel(Grid g, const double *px, const double *py, const double *pz,
                             const int32_t *kind, int64_t n, uint64_t *key, int64_t *idx) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int cx = cell_coord(px[i], g.lo[0], g.inv_cell, g.nc[0]);
    int cy = cell_coord(py[i], g.lo[1], g.inv_cell, g.nc[1]);
    int cz = cell_coord(pz[i], g.lo[2], g.inv_cell, g.nc[2]);
    uint64_t k = morton(g, cx, cy, cz);
    if (kind[i] != SPH_RT_INTERIOR) k |= 1ull << g.ghost_shift;
    key[i] = k;
    idx[i] = i;
  }
}

// Stable LSD radix sort of (key, index) pairs, 8 bits a pass.  A block owns a
// contiguous tile of kRadixItems * blockDim items; pass 1 counts its digits
// (hist[d * nb + b]); after an exclusive scan over (digit, block) the scatter
// places the tile's items in order: round by round, each item's rank among
// the equal digits of its warp (match_any), after those of the earlier warps
// of the round and of the earlier rounds.  Equal keys keep their order, and
// the index starts as the caller index, so ties end in caller order.
constexpr int kRadixItems = 16;
constexpr int kRadixTile = kBlock * kRadixItems;
static_assert(kBlock == 256, "the radix kernels give each of the 256 digits one thread");

__global__ void radix_hist_kernel(const uint64_t *key, int64_t n, int shift, int64_t nb,
                                  int64_t *hist) {
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;  // blockDim == 256
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  for (int r = 0; r < kRadixItems; ++r) {
    const int64_t i = base + (int64_t)r * kBlock + threadIdx.x;
    if (i < n) atomicAdd(&h[(key[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

__global__ void radix_scatter_kernel(const uint64_t *kin, const int64_t *vin, int64_t n, int shift,
                                     int64_t nb, const int64_t *off, uint64_t *kout,
                                     int64_t *vout) {
  __shared__ unsigned wc[kWarpsPerBlock][256];
  __shared__ int64_t run[256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  run[threadIdx.x] = off[(int64_t)threadIdx.x * nb + blockIdx.x];
  for (int a = 0; a < kWarpsPerBlock; ++a) wc[a][threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  for (int r = 0; r < kRadixItems; ++r) {
    const int64_t i = base + (int64_t)r * kBlock + threadIdx.x;
    const bool valid = i < n;
    const uint64_t k = valid ? kin[i] : 0ull;
    const int d = valid ? (int)((k >> shift) & 255u) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    if (valid && lane == __ffs(peers) - 1) wc[w][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int64_t pos = run[d] + rank;
      for (int a = 0; a < w; ++a) pos += wc[a][d];
      kout[pos] = k;
      vout[pos] = vin[i];
    }
    __syncthreads();
    unsigned t = 0;
    for (int a = 0; a < kWarpsPerBlock; ++a) {
      t += wc[a][threadIdx.x];
      wc[a][threadIdx.x] = 0;
    }
    run[threadIdx.x] += t;
    __syncthreads();
  }
}

__global__ void cell_head_kernel(const uint64_t *key, int64_t n, int64_t *head) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    head[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

__global__ void cell_fill_kernel(const uint64_t *key, int64_t n, const int64_t *head,
                                 const int64_t *cidx, uint64_t *cell_key, int64_t *cell_start) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!head[i]) continue;
    cell_key[cidx[i]] = key[i];
    cell_start[cidx[i]] = i;
  }
}

__global__ void cell_hash_insert_kernel(const uint64_t *cell_key, int64_t ncells, uint64_t mask,
                                        unsigned long long *hkey, int64_t *hcell) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells;
       c += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = cell_key[c];
    uint64_t h = cell_hash(k) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {  // keys are distinct: ends at a free entry
      if (atomicCAS(&hkey[h], kEmptyCell, k) == kEmptyCell) {
        hcell[h] = c;
        break;
      }
      h = (h + 1) & mask;
    }
  }
}

__global__ void invert_perm(const int64_t *slot2caller, int64_t n, int64_t *caller2slot) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x)
    caller2slot[slot2caller[s]] = s;
}

template <typename T>
__global__ void gather_kernel(const T *in, const int64_t *slot2caller, int64_t n, T *out) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x)
    out[s] = in[slot2caller[s]];
}

// positions: caller row-major [n][dim] -> SoA slot order (missing dims = 0)
__global__ void gather_pos_kernel(const double *pos, int dim, const int64_t *slot2caller,
                                  int64_t n, double *px, double *py, double *pz) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = slot2caller[s];
    px[s] = pos[c * dim];
    py[s] = dim > 1 ? pos[c * dim + 1] : 0.0;
    pz[s] = dim > 2 ? pos[c * dim + 2] : 0.0;
  }
}

__global__ void caller_pos_to_soa(const double *pos, int dim, int64_t n, double *px, double *py,
                                  double *pz) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    px[i] = pos[i * dim];
    py[i] = dim > 1 ? pos[i * dim + 1] : 0.0;
    pz[i] = dim > 2 ? pos[i * dim + 2] : 0.0;
  }
}

__global__ void copysrc_kernel(const int64_t *copy_of, const int32_t *kind_slot,
                               const int64_t *slot2caller, const int64_t *caller2slot, int64_t n,
                               int32_t *copysrc) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = -1;
    if (kind_slot[s] == SPH_RT_COPY && copy_of) v = (int32_t)caller2slot[copy_of[slot2caller[s]]];
    copysrc[s] = v;
  }
}

__global__ void volume_kernel(const double *mass, const double *rho, int64_t n, double *V,
                              double *invV) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    double v = mass[s] / rho[s];
    V[s] = v;
    invV[s] = 1.0 / v;
  }
}

// --------------------------------------------------------------------------
// Neighbour search: one warp per interior particle.
// --------------------------------------------------------------------------
// Shape of dW/dq of the M4 cubic B-spline (support q < 2).
__device__ __forceinline__ double spline_dw(double q) {
  if (q < 1.0) return -3.0 * q + 2.25 * q * q;
  if (q < 2.0) {
    double t = 2.0 - q;
    return -0.75 * t * t;
  }
  return 0.0;
}

// Shape of dW/dq of the Wendland C4 kernel of Sec. 2.4 (Eq. wendlandc4): the
// printed polynomial (1 - q)^5 (8 q^2 + 5 q + 1) on q <= 1 has the derivative
// -14 q (1 + 4 q) (1 - q)^4.
__device__ __forceinline__ double wendland_dw(double q) {
  if (q <= 1.0) {
    const double t = 1.0 - q, t2 = t * t;
    return -14.0 * q * (1.0 + 4.0 * q) * (t2 * t2);
  }
  return 0.0;
}

// Per-particle kernel coefficients: 1/h and k_d / h^(d+1), so that
// dW/dr(r, h) = k_d / h^(d+1) * w'(r / h) needs no division per pair.  k_d makes
// the kernel's volume integral one (Sec. 2.3): for the cubic B-spline 2/3,
// 10/(7 pi), 1/pi; for the Wendland C4 polynomial as printed in every dimension
// 3/2, 36/(5 pi), 45/(4 pi).
__global__ void kernel_coef_kernel(int64_t n, int dim, int kern, const double *h, double *ih,
                                   double *cw) {
  const double pi = 3.141592653589793;
  const double sd =
      kern == SPH_RT_WENDLAND_C4
          ? (dim == 3 ? 45.0 / (4.0 * pi) : (dim == 2 ? 36.0 / (5.0 * pi) : 1.5))
          : (dim == 3 ? 1.0 / pi : (dim == 2 ? 10.0 / (7.0 * pi) : 2.0 / 3.0));
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double inv = 1.0 / h[i];
    double p = inv * inv;  // h^-2
    if (dim >= 2) p *= inv;
    if (dim >= 3) p *= inv;
    ih[i] = inv;
    cw[i] = sd * p;
  }
}

__device__ __forceinline__ double exact_r2(double xi, double yi, double zi, double xj, double yj,
                                           double zj) {
  double dx = __dsub_rn(xi, xj), dy = __dsub_rn(yi, yj), dz = __dsub_rn(zi, zj);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// FP32 pre-filter of the neighbour predicate.  GB300 issues FP64 arithmetic at
// ~1/64 of the FP32 rate, and a 3-D particle has ~729 candidates for ~113
// neighbours, so the candidate test runs in FP32 on positions relative to the
// particle's own cell: rel = x - (lo + c cell), |rel| <= ~cell, stored as
// float with the particle's (2h)^2 (the exact FP64 cut of a pair is
// max((2h_i)^2, (2h_j)^2), since rounding is monotonic).  For a candidate in
// the cell at offset o (-1, 0, 1 per axis) from the particle's,
//   dx = x_i - x_j = (rel_i - rel_j) - o cell.
// Error bound (cell = C, unit roundoff u = 2^-24): each rel carries <= 1.01 u C,
// the difference, the product o cell and the sum add <= 2.02 u C, u C and
// 3.03 u C, so |dx_f - dx| <= 8.1 u C = 4.8e-7 C; near the cut (r <= C) the
// squares and sums then differ from the exact r^2 by <= 2 sqrt(3) 4.8e-7 C^2 +
// 4 u 3 C^2 ~ 2.4e-6 C^2, and the FP32 cut by <= u C^2.  A candidate farther
// than kNbrBand C^2 (12x that bound) from the cut is decided in FP32; the
// rest take the exact FP64 predicate, so the neighbour sets are bitwise those
// of the exact test.
constexpr float kNbrBand = 3e-5f;

__global__ void rel_kernel(Grid g, const double *px, const double *py, const double *pz,
                           const double *h, int64_t n, float4 *rel) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const double x = px[j], y = py[j], z = pz[j];
    const int cx = cell_coord(x, g.lo[0], g.inv_cell, g.nc[0]);
    const int cy = cell_coord(y, g.lo[1], g.inv_cell, g.nc[1]);
    const int cz = cell_coord(z, g.lo[2], g.inv_cell, g.nc[2]);
    const double cut = g.support * h[j];
    float4 r;
    r.x = (float)(x - (g.lo[0] + (double)cx * g.cell));
    r.y = g.dim > 1 ? (float)(y - (g.lo[1] + (double)cy * g.cell)) : 0.0f;
    r.z = g.dim > 2 ? (float)(z - (g.lo[2] + (double)cz * g.cell)) : 0.0f;
    r.w = (float)__dmul_rn(cut, cut);
    rel[j] = r;
  }
}

// 1 / sqrt(r2) in FP64: FP32 seed refined by two Newton steps
// y <- y (3/2 - r2/2 y^2) (quadratic convergence from ~1e-7 to the FP64
// rounding level), which costs fewer FP64 operations than an IEEE square
// root followed by a division.
__device__ __forceinline__ double rsqrt_fp64(double r2) {
  double y = (double)rsqrtf((float)r2);
  const double hr2 = 0.5 * r2;
  y = y * (1.5 - hr2 * y * y);
  y = y * (1.5 - hr2 * y * y);
  return y;
}

// Bitonic sort of one 64-bit key per lane, ascending across the warp.
__device__ __forceinline__ uint64_t warp_sort_u64(uint64_t v) {
  int lane = threadIdx.x & 31;
  for (int k = 2; k <= 32; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      uint64_t o = __shfl_xor_sync(0xffffffffu, v, j);
      bool up = ((lane & k) == 0);
      bool lower = ((lane & j) == 0);
      uint64_t mn = v < o ? v : o, mx = v < o ? o : v;
      v = (lower == up) ? mn : mx;
    }
  }
  return v;
}

// Cell lookup of the neighbour kernels: first slot and particle count of a key.
struct DenseCells {  // tables over every key
  const int64_t *start;
  const unsigned *count;
  __device__ __forceinline__ void find(uint64_t k, int64_t &beg, int64_t &cnt) const {
    beg = start[k];
    cnt = count[k];
  }
};
struct HashCells {  // occupied cells only, open addressing with linear probing
  const unsigned long long *hkey;  // [mask + 1], kEmptyCell where free
  const int64_t *hcell;            // cell of each used entry
  const int64_t *cstart;           // [ncells + 1] first slot of each cell
  uint64_t mask;
  __device__ __forceinline__ void find(uint64_t k, int64_t &beg, int64_t &cnt) const {
    beg = 0;
    cnt = 0;
    uint64_t h = cell_hash(k) & mask;
    // the table is at most half full, so a free entry ends every probe sequence
    for (uint64_t probe = 0; probe <= mask; ++probe) {
      const unsigned long long t = hkey[h];
      if (t == k) {
        const int64_t c = hcell[h];
        beg = cstart[c];
        cnt = cstart[c + 1] - beg;
        return;
      }
      if (t == kEmptyCell) return;
      h = (h + 1) & mask;
    }
  }
};

// Pair weight F_ij = W'_ij / r (two-h average) of neighbour j of i, in FP64.
__device__ __forceinline__ double pair_weight(int kern, double xi, double yi, double zi,
                                              double ihi, double cwi, int64_t j,
                                              const double *px, const double *py,
                                              const double *pz, const double *ih,
                                              const double *cw) {
  const double r2 = exact_r2(xi, yi, zi, px[j], py[j], pz[j]);
  const double ir = rsqrt_fp64(r2), r = r2 * ir;
  const double ihj = ih[j], cwj = cw[j];
  const double qi = r * ihi;
  const double dwi = cwi * (kern == SPH_RT_WENDLAND_C4 ? wendland_dw(qi) : spline_dw(qi));
  // equal smoothing lengths (the common case): the same expression, computed once
  double dwj = dwi;
  if (ihj != ihi || cwj != cwi) {
    const double qj = r * ihj;
    dwj = cwj * (kern == SPH_RT_WENDLAND_C4 ? wendland_dw(qj) : spline_dw(qj));
  }
  return 0.5 * (dwi + dwj) * ir;
}

// One warp per interior particle.  FILL: the hits of each 32-candidate batch
// (a few of 27 candidates per cell) are appended, in discovery order, to a
// per-warp buffer, and their FP64 pair weights are computed 32 at a time:
// an FP64 warp instruction costs the same with 1 or 32 active lanes, so
// computing the weights per batch would cost ~27 batches of FP64 work per
// particle instead of ~4.
constexpr int kHitBuf = 64;  // pending hits per warp (< 32 carried + 32 new)

template <bool FILL, typename Cells>
__global__ void neighbor_kernel(Grid g, const double *px, const double *py, const double *pz,
                                const double *h, const float4 *rel, Cells cells,
                                int64_t n_int, int64_t *count,
                                const int64_t *rowptr, int32_t *cols, double *F,
                                const double *ih, const double *cw) {
  __shared__ int32_t hitbuf[kWarpsPerBlock][FILL ? kHitBuf : 1];
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  int32_t *hb = hitbuf[threadIdx.x >> 5];
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int ncells = g.dim == 3 ? 27 : (g.dim == 2 ? 9 : 3);
  const float cellf = (float)g.cell;
  const float band = kNbrBand * cellf * cellf;
  for (int64_t i = warp; i < n_int; i += nwarps) {
    const double xi = px[i], yi = py[i], zi = pz[i], hi = h[i];
    const float4 ri = rel[i];
    int c[3] = {cell_coord(xi, g.lo[0], g.inv_cell, g.nc[0]),
                cell_coord(yi, g.lo[1], g.inv_cell, g.nc[1]),
                cell_coord(zi, g.lo[2], g.inv_cell, g.nc[2])};
    // lane k < ncells: the k-th cell around i; sorted by Morton key with the
    // lane (hence the offset) in the low 5 bits
    uint64_t mykey = ~0ull;
    if (lane < ncells) {
      int o[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
      bool ok = true;
      int cc[3];
      for (int d = 0; d < 3; ++d) {
        cc[d] = d < g.dim ? c[d] + o[d] : 0;
        if (d < g.dim && (cc[d] < 0 || cc[d] >= g.nc[d])) ok = false;
      }
      if (ok) mykey = (morton(g, cc[0], cc[1], cc[2]) << 5) | (uint64_t)lane;
    }
    const uint64_t sorted = warp_sort_u64(mykey);
    const int64_t out = FILL ? rowptr[i] : 0;
    const double ihi = FILL ? ih[i] : 0.0, cwi = FILL ? cw[i] : 0.0;
    int64_t total = 0;  // hits found (warp-uniform)
    int64_t done = 0;   // hits written (FILL)
    int pending = 0;    // hits in the buffer (FILL, warp-uniform)
    for (int pass = 0; pass < 2; ++pass) {  // interior cells, then ghost cells
      for (int k = 0; k < ncells; ++k) {
        const uint64_t v = __shfl_sync(0xffffffffu, sorted, k);
        if (v == ~0ull) break;
        const int ol = (int)(v & 31ull);
        const uint64_t kk = (v >> 5) | (pass ? (1ull << g.ghost_shift) : 0ull);
        // -o cell per axis (axes beyond dim stay 0)
        const float ox = -(float)(ol % 3 - 1) * cellf;
        const float oy = g.dim > 1 ? -(float)((ol / 3) % 3 - 1) * cellf : 0.0f;
        const float oz = g.dim > 2 ? -(float)(ol / 9 - 1) * cellf : 0.0f;
        int64_t beg, cnt;
        cells.find(kk, beg, cnt);
        for (int64_t base = 0; base < cnt; base += 32) {
          const int64_t j = beg + base + lane;
          bool hit = false;
          if (base + lane < cnt && j != i) {
            const float4 rj = rel[j];
            const float dx = (ri.x - rj.x) + ox;
            const float dy = (ri.y - rj.y) + oy;
            const float dz = (ri.z - rj.z) + oz;
            const float r2f = dx * dx + dy * dy + dz * dz;
            const float c2f = fmaxf(ri.w, rj.w);
            if (r2f < c2f - band) {
              hit = true;
            } else if (!(r2f > c2f + band)) {  // within the band: the exact test
              const double cut = g.support * fmax(hi, h[j]);
              hit = exact_r2(xi, yi, zi, px[j], py[j], pz[j]) < __dmul_rn(cut, cut);
            }
          }
          const unsigned m = __ballot_sync(0xffffffffu, hit);
          total += __popc(m);
          if (FILL) {
            if (hit) hb[pending + __popc(m & lt)] = (int32_t)j;
            pending += __popc(m);
            __syncwarp();
            if (pending >= 32) {  // 32 weights with every lane active
              const int32_t jj = hb[lane];
              cols[out + done + lane] = jj;
              F[out + done + lane] = pair_weight(g.kernel, xi, yi, zi, ihi, cwi, jj, px, py, pz, ih, cw);
              const int rest = pending - 32;
              const int32_t carry = lane < rest ? hb[32 + lane] : 0;
              __syncwarp();
              if (lane < rest) hb[lane] = carry;
              __syncwarp();
              pending = rest;
              done += 32;
            }
          }
        }
      }
    }
    if (FILL && pending > 0) {
      if (lane < pending) {
        const int32_t jj = hb[lane];
        cols[out + done + lane] = jj;
        F[out + done + lane] = pair_weight(g.kernel, xi, yi, zi, ihi, cwi, jj, px, py, pz, ih, cw);
      }
      __syncwarp();
    }
    if (!FILL && lane == 0) count[i] = total;
  }
}

// --------------------------------------------------------------------------
// Operator sparsity from the neighbour lists: interior columns and copy-ghost
// columns (moved to the copied particle; a copy of the row itself drops out)
// form B; Dirichlet ghosts form the boundary-coupling list.
// --------------------------------------------------------------------------
// One warp per row: the lanes take 32 consecutive entries at a time, so the
// list reads and the compacted writes are coalesced; ballots keep the entries
// in list order.
__global__ void op_count_kernel(const int64_t *nbr_ptr, const int32_t *nbr_col,
                                const int32_t *kind, const int32_t *copysrc, int64_t n_int,
                                int64_t *mat_cnt, int64_t *gh_cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n_int; i += nwarps) {
    int64_t m = 0, g = 0;
    const int64_t beg = nbr_ptr[i], end = nbr_ptr[i + 1];
    for (int64_t k0 = beg; k0 < end; k0 += 32) {
      const int64_t k = k0 + lane;
      bool isg = false, ism = false;
      if (k < end) {
        const int32_t j = nbr_col[k];
        const int32_t kj = kind[j];
        isg = kj == SPH_RT_DIRICHLET;
        ism = !isg && (kj == SPH_RT_INTERIOR || copysrc[j] != i);
      }
      g += __popc(__ballot_sync(0xffffffffu, isg));
      m += __popc(__ballot_sync(0xffffffffu, ism));
    }
    if (lane == 0) {
      mat_cnt[i] = m;
      gh_cnt[i] = g;
    }
  }
}

__global__ void op_fill_kernel(const int64_t *nbr_ptr, const int32_t *nbr_col, const double *nbr_F,
                               const int32_t *kind, const int32_t *copysrc, const double *V,
                               int64_t n_int, const int64_t *mat_ptr, int32_t *mat_col,
                               double *mat_G, const int64_t *gh_ptr, int32_t *gh_slot,
                               double *gh_W) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n_int; i += nwarps) {
    int64_t m = mat_ptr[i], g = gh_ptr[i];
    const double Vi = V[i];
    const int64_t beg = nbr_ptr[i], end = nbr_ptr[i + 1];
    for (int64_t k0 = beg; k0 < end; k0 += 32) {
      const int64_t k = k0 + lane;
      bool isg = false, ism = false;
      int32_t col = 0;
      double val = 0.0;
      if (k < end) {
        const int32_t j = nbr_col[k];
        const int32_t kj = kind[j];
        const double Fk = nbr_F[k];
        if (kj == SPH_RT_DIRICHLET) {
          isg = true;
          col = j;
          val = V[j] * Fk;
        } else {
          col = kj == SPH_RT_INTERIOR ? j : copysrc[j];
          if (col != i) {  // a copy of the row itself drops out
            ism = true;
            val = (Vi * V[j]) * Fk;
          }
        }
      }
      const unsigned bg = __ballot_sync(0xffffffffu, isg);
      const unsigned bm = __ballot_sync(0xffffffffu, ism);
      if (isg) {
        const int64_t at = g + __popc(bg & lt);
        gh_slot[at] = col;
        gh_W[at] = val;
      }
      if (ism) {
        const int64_t at = m + __popc(bm & lt);
        mat_col[at] = col;
        mat_G[at] = val;
      }
      g += __popc(bg);
      m += __popc(bm);
    }
  }
}

// --------------------------------------------------------------------------
// Host driver
// --------------------------------------------------------------------------
static int grid1(const sph_rt *s, int64_t n) {
  int64_t g = ceil_div(n > 0 ? n : 1, kBlock);
  int64_t cap = (int64_t)s->num_sms * 8;
  return (int)(g < cap ? g : cap);
}

// Build permutation, slot-order particle data, neighbour lists and operator
// sparsity from caller-order device arrays.
sph_rt_status build_particles(sph_rt *s, int64_t n, const double *pos_c, const double *mass_c,
                              const double *rho_c, const double *h_c, const double *sig0_c,
                              const int32_t *kind_c, const int64_t *copy_of_c,
                              const double *e0_c, const double *E0_c, int64_t n_int) {
  const int dim = s->dim;
  cudaStream_t st = s->stream;
  s->n = n;
  s->n_int = n_int;
  // caller-order SoA positions for the key pass
  double *cx = dalloc<double>(s, n), *cy = dalloc<double>(s, n), *cz = dalloc<double>(s, n);
  double *hc = dalloc<double>(s, n);
  double *bbox = dalloc<double>(s, 8);
  s->partials = dalloc<double>(s, 8 * kMaxRedBlocks);
  s->sc = dalloc<Scalars>(s, 1);
  if (!cx || !cy || !cz || !hc || !bbox || !s->partials || !s->sc) return SPH_RT_ENOMEM;
  SPH_CUDA(s, cudaMemsetAsync(s->sc, 0, sizeof(Scalars), st));
  caller_pos_to_soa<<<grid1(s, n), kBlock, 0, st>>>(pos_c, dim, n, cx, cy, cz);
  SPH_LAUNCHED(s);
  SPH_CUDA(s, cudaMemcpyAsync(hc, h_c, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  int gb = grid1(s, n);
  if (gb > kMaxRedBlocks) gb = kMaxRedBlocks;
  bbox_kernel<<<gb, kBlock, 0, st>>>(cx, cy, cz, hc, n, s->partials, &s->sc->counter, bbox);
  SPH_LAUNCHED(s);
  double hb[8];
  SPH_CUDA(s, cudaMemcpyAsync(hb, bbox, sizeof(double) * 7, cudaMemcpyDeviceToHost, st));
  SPH_CUDA(s, cudaStreamSynchronize(st));

  Grid g;
  g.dim = dim;
  g.kernel = s->cfg.kernel;
  g.support = s->cfg.kernel == SPH_RT_WENDLAND_C4 ? 1.0 : 2.0;
  double cell = g.support * hb[6] * (1.0 + 1e-9);
  g.cell = cell;
  g.inv_cell = 1.0 / cell;
  int maxnc = 1;
  for (int d = 0; d < 3; ++d) {
    g.lo[d] = hb[d];
    const double ncd = d < dim ? floor((hb[3 + d] - hb[d]) / cell) + 1.0 : 1.0;
    if (!(ncd <= (double)(1 << 29)))
      return set_error(s, SPH_RT_EINVAL,
                       "particle extent is too large relative to the support (more than 2^29 "
                       "cells along an axis)");
    const int nc = (int)ncd;
    g.nc[d] = nc;
    maxnc = nc > maxnc ? nc : maxnc;
  }
  int bits = 0;
  while ((1 << bits) < maxnc) ++bits;
  const int keybits = bits * dim;
  // dense key table up to 2^27 keys (2^26 cells), else the sorted-key list
  const bool fits_dense = keybits + 1 <= 27;
  const bool dense = s->cfg.cell_list == SPH_RT_CELLS_DENSE ||
                     (s->cfg.cell_list == SPH_RT_CELLS_AUTO && fits_dense);
  if (dense && !fits_dense)
    return set_error(s, SPH_RT_EINVAL,
                     "particle extent is too large relative to the support for the dense cell "
                     "table (more than 2^26 cells); use the sorted cell list");
  if (keybits > 58)
    return set_error(s, SPH_RT_EINVAL,
                     "particle extent is too large relative to the support (more than 2^58 "
                     "cells)");
  g.ghost_shift = keybits;
  const int64_t nkeys = dense ? (int64_t)1 << (keybits + 1) : 0;

  // dense table
  uint32_t *key = nullptr;
  unsigned *cnt = nullptr, *cur = nullptr;
  int64_t *cnt64 = nullptr, *start = nullptr;
  // sorted keys
  uint64_t *k64[2] = {nullptr, nullptr}, *cell_key = nullptr;
  int64_t *v64[2] = {nullptr, nullptr}, *rhist = nullptr, *head = nullptr, *cidx = nullptr;
  int64_t *cell_start = nullptr, *hcell = nullptr;
  unsigned long long *hkey = nullptr;
  HashCells hcells{};
  s->slot2caller = dalloc<int64_t>(s, n);
  s->caller2slot = dalloc<int64_t>(s, n);
  if (!s->slot2caller || !s->caller2slot) return SPH_RT_ENOMEM;
  sph_rt_status rc;
  if (dense) {
    key = dalloc<uint32_t>(s, n);
    cnt = dalloc<unsigned>(s, nkeys);
    cur = dalloc<unsigned>(s, nkeys);
    cnt64 = dalloc<int64_t>(s, nkeys);
    start = dalloc<int64_t>(s, nkeys + 1);
    if (!key || !cnt || !cur || !cnt64 || !start) return SPH_RT_ENOMEM;
    SPH_CUDA(s, cudaMemsetAsync(cnt, 0, sizeof(unsigned) * nkeys, st));
    SPH_CUDA(s, cudaMemsetAsync(cur, 0, sizeof(unsigned) * nkeys, st));
    key_kernel<<<grid1(s, n), kBlock, 0, st>>>(g, cx, cy, cz, kind_c, n, key, cnt);
    SPH_LAUNCHED(s);
    u32_to_i64<<<grid1(s, nkeys), kBlock, 0, st>>>(cnt, nkeys, cnt64);
    SPH_LAUNCHED(s);
    if ((rc = exclusive_scan(s, cnt64, nkeys, start))) return rc;
    scatter_kernel<<<grid1(s, n), kBlock, 0, st>>>(key, n, start, cur, s->slot2caller);
    SPH_LAUNCHED(s);
    segment_sort_kernel<<<grid1(s, nkeys), kBlock, 0, st>>>(start, cnt, nkeys, s->slot2caller);
    SPH_LAUNCHED(s);
  } else {
    const int64_t nb = ceil_div(n, (int64_t)kRadixTile);
    for (int a = 0; a < 2; ++a) {
      k64[a] = dalloc<uint64_t>(s, n);
      v64[a] = dalloc<int64_t>(s, n);
    }
    rhist = dalloc<int64_t>(s, 256 * nb + 1);
    int64_t *roff = dalloc<int64_t>(s, 256 * nb + 1);
    if (!k64[0] || !k64[1] || !v64[0] || !v64[1] || !rhist || !roff) return SPH_RT_ENOMEM;
    key64_kernel<<<grid1(s, n), kBlock, 0, st>>>(g, cx, cy, cz, kind_c, n, k64[0], v64[0]);
    SPH_LAUNCHED(s);
    int at = 0;
    for (int shift = 0; shift < keybits + 1; shift += 8, at ^= 1) {
      radix_hist_kernel<<<(unsigned)nb, kBlock, 0, st>>>(k64[at], n, shift, nb, rhist);
      SPH_LAUNCHED(s);
      if ((rc = exclusive_scan(s, rhist, 256 * nb, roff))) return rc;
      radix_scatter_kernel<<<(unsigned)nb, kBlock, 0, st>>>(k64[at], v64[at], n, shift, nb, roff,
                                                          k64[at ^ 1], v64[at ^ 1]);
      SPH_LAUNCHED(s);
    }
    dfree(s, roff);
    SPH_CUDA(s, cudaMemcpyAsync(s->slot2caller, v64[at], sizeof(int64_t) * n,
                                cudaMemcpyDeviceToDevice, st));
    // occupied cells: runs of equal keys
    head = dalloc<int64_t>(s, n);
    cidx = dalloc<int64_t>(s, n + 1);
    if (!head || !cidx) return SPH_RT_ENOMEM;
    cell_head_kernel<<<grid1(s, n), kBlock, 0, st>>>(k64[at], n, head);
    SPH_LAUNCHED(s);
    if ((rc = exclusive_scan(s, head, n, cidx))) return rc;
    int64_t ncells = 0;
    SPH_CUDA(s, cudaMemcpyAsync(&ncells, cidx + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SPH_CUDA(s, cudaStreamSynchronize(st));
    cell_key = dalloc<uint64_t>(s, ncells);
    cell_start = dalloc<int64_t>(s, ncells + 1);
    uint64_t hsize = 2;
    while (hsize < 2 * (uint64_t)ncells) hsize <<= 1;  // at most half full
    hkey = dalloc<unsigned long long>(s, hsize);
    hcell = dalloc<int64_t>(s, hsize);
    if (!cell_key || !cell_start || !hkey || !hcell) return SPH_RT_ENOMEM;
    cell_fill_kernel<<<grid1(s, n), kBlock, 0, st>>>(k64[at], n, head, cidx, cell_key, cell_start);
    SPH_LAUNCHED(s);
    SPH_CUDA(s, cudaMemcpyAsync(cell_start + ncells, &n, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    SPH_CUDA(s, cudaMemsetAsync(hkey, 0xff, sizeof(unsigned long long) * hsize, st));
    cell_hash_insert_kernel<<<grid1(s, ncells), kBlock, 0, st>>>(cell_key, ncells, hsize - 1, hkey,
                                                                hcell);
    SPH_LAUNCHED(s);
    hcells = HashCells{hkey, hcell, cell_start, hsize - 1};
  }
  invert_perm<<<grid1(s, n), kBlock, 0, st>>>(s->slot2caller, n, s->caller2slot);
  SPH_LAUNCHED(s);

  // slot-order particle data
  s->px = dalloc<double>(s, n);
  s->py = dalloc<double>(s, n);
  s->pz = dalloc<double>(s, n);
  s->mass = dalloc<double>(s, n);
  s->rho = dalloc<double>(s, n);
  s->h = dalloc<double>(s, n);
  s->sigma0 = dalloc<double>(s, n);
  s->V = dalloc<double>(s, n);
  s->invV = dalloc<double>(s, n);
  s->kind = dalloc<int32_t>(s, n);
  s->copysrc = dalloc<int32_t>(s, n);
  s->e = dalloc<double>(s, n);
  s->E = dalloc<double>(s, n);
  if (!s->px || !s->py || !s->pz || !s->mass || !s->rho || !s->h || !s->sigma0 || !s->V ||
      !s->invV || !s->kind || !s->copysrc || !s->e || !s->E)
    return SPH_RT_ENOMEM;
  int gg = grid1(s, n);
  gather_pos_kernel<<<gg, kBlock, 0, st>>>(pos_c, dim, s->slot2caller, n, s->px, s->py, s->pz);
  SPH_LAUNCHED(s);
  gather_kernel<double><<<gg, kBlock, 0, st>>>(mass_c, s->slot2caller, n, s->mass);
  SPH_LAUNCHED(s);
  gather_kernel<double><<<gg, kBlock, 0, st>>>(rho_c, s->slot2caller, n, s->rho);
  SPH_LAUNCHED(s);
  gather_kernel<double><<<gg, kBlock, 0, st>>>(h_c, s->slot2caller, n, s->h);
  SPH_LAUNCHED(s);
  gather_kernel<double><<<gg, kBlock, 0, st>>>(sig0_c, s->slot2caller, n, s->sigma0);
  SPH_LAUNCHED(s);
  gather_kernel<int32_t><<<gg, kBlock, 0, st>>>(kind_c, s->slot2caller, n, s->kind);
  SPH_LAUNCHED(s);
  gather_kernel<double><<<gg, kBlock, 0, st>>>(e0_c, s->slot2caller, n, s->e);
  SPH_LAUNCHED(s);
  gather_kernel<double><<<gg, kBlock, 0, st>>>(E0_c, s->slot2caller, n, s->E);
  SPH_LAUNCHED(s);
  copysrc_kernel<<<gg, kBlock, 0, st>>>(copy_of_c, s->kind, s->slot2caller, s->caller2slot, n,
                                        s->copysrc);
  SPH_LAUNCHED(s);
  volume_kernel<<<gg, kBlock, 0, st>>>(s->mass, s->rho, n, s->V, s->invV);
  SPH_LAUNCHED(s);

  // neighbour lists
  int64_t *nc = dalloc<int64_t>(s, n_int);
  s->nbr_ptr = dalloc<int64_t>(s, n_int + 1);
  if (!nc || !s->nbr_ptr) return SPH_RT_ENOMEM;
  int64_t warps = n_int;
  int gw = (int)ceil_div(warps, kWarpsPerBlock);
  int gcap = s->num_sms * 8;
  if (gw > gcap) gw = gcap;
  float4 *rel = dalloc<float4>(s, n);
  if (!rel) return SPH_RT_ENOMEM;
  rel_kernel<<<grid1(s, n), kBlock, 0, st>>>(g, s->px, s->py, s->pz, s->h, n, rel);
  SPH_LAUNCHED(s);
  if (dense)
    neighbor_kernel<false, DenseCells><<<gw, kBlock, 0, st>>>(
        g, s->px, s->py, s->pz, s->h, rel, DenseCells{start, cnt}, n_int, nc, nullptr, nullptr,
        nullptr, nullptr, nullptr);
  else
    neighbor_kernel<false, HashCells><<<gw, kBlock, 0, st>>>(g, s->px, s->py, s->pz, s->h, rel,
                                                             hcells, n_int, nc, nullptr, nullptr,
                                                             nullptr, nullptr, nullptr);
  SPH_LAUNCHED(s);
  rc = exclusive_scan(s, nc, n_int, s->nbr_ptr);
  if (rc) return rc;
  int64_t nnz = 0;
  SPH_CUDA(s, cudaMemcpyAsync(&nnz, s->nbr_ptr + n_int, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SPH_CUDA(s, cudaStreamSynchronize(st));
  s->nnz_nbr = nnz;
  s->nbr_col = dalloc<int32_t>(s, nnz);
  s->nbr_F = dalloc<double>(s, nnz);
  if (!s->nbr_col || !s->nbr_F) return SPH_RT_ENOMEM;
  double *ih = dalloc<double>(s, n), *cw = dalloc<double>(s, n);
  if (!ih || !cw) return SPH_RT_ENOMEM;
  kernel_coef_kernel<<<grid1(s, n), kBlock, 0, st>>>(n, dim, s->cfg.kernel, s->h, ih, cw);
  SPH_LAUNCHED(s);
  if (dense)
    neighbor_kernel<true, DenseCells><<<gw, kBlock, 0, st>>>(
        g, s->px, s->py, s->pz, s->h, rel, DenseCells{start, cnt}, n_int, nullptr, s->nbr_ptr,
        s->nbr_col, s->nbr_F, ih, cw);
  else
    neighbor_kernel<true, HashCells><<<gw, kBlock, 0, st>>>(g, s->px, s->py, s->pz, s->h, rel,
                                                            hcells, n_int, nullptr, s->nbr_ptr,
                                                            s->nbr_col, s->nbr_F, ih, cw);
  SPH_LAUNCHED(s);

  // operator sparsity
  int64_t *mc = dalloc<int64_t>(s, n_int), *gc = dalloc<int64_t>(s, n_int);
  s->mat_ptr = dalloc<int64_t>(s, n_int + 1);
  s->gh_ptr = dalloc<int64_t>(s, n_int + 1);
  if (!mc || !gc || !s->mat_ptr || !s->gh_ptr) return SPH_RT_ENOMEM;
  int gi = (int)ceil_div(n_int, kWarpsPerBlock);  // a warp per row
  if (gi > s->num_sms * 8) gi = s->num_sms * 8;
  op_count_kernel<<<gi, kBlock, 0, st>>>(s->nbr_ptr, s->nbr_col, s->kind, s->copysrc, n_int, mc, gc);
  SPH_LAUNCHED(s);
  if ((rc = exclusive_scan(s, mc, n_int, s->mat_ptr))) return rc;
  if ((rc = exclusive_scan(s, gc, n_int, s->gh_ptr))) return rc;
  int64_t sizes[2];
  SPH_CUDA(s, cudaMemcpyAsync(&sizes[0], s->mat_ptr + n_int, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SPH_CUDA(s, cudaMemcpyAsync(&sizes[1], s->gh_ptr + n_int, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SPH_CUDA(s, cudaStreamSynchronize(st));
  s->nnz_mat = sizes[0];
  s->nnz_gh = sizes[1];
  s->mat_col = dalloc<int32_t>(s, s->nnz_mat);
  s->mat_G = dalloc<double>(s, s->nnz_mat);
  s->mat_val = dalloc<double>(s, s->nnz_mat);
  s->gh_slot = dalloc<int32_t>(s, s->nnz_gh);
  s->gh_W = dalloc<double>(s, s->nnz_gh);
  if (!s->mat_col || !s->mat_G || !s->mat_val || !s->gh_slot || !s->gh_W) return SPH_RT_ENOMEM;
  op_fill_kernel<<<gi, kBlock, 0, st>>>(s->nbr_ptr, s->nbr_col, s->nbr_F, s->kind, s->copysrc,
                                        s->V, n_int, s->mat_ptr, s->mat_col, s->mat_G, s->gh_ptr,
                                        s->gh_slot, s->gh_W);
  SPH_LAUNCHED(s);
  SPH_CUDA(s, cudaStreamSynchronize(st));
  // set-up scratch back to the free list
  void *scratch[] = {cx, cy, cz, hc, bbox, key, cnt, cur, cnt64, start, nc, mc, gc, ih, cw, rel,
                     k64[0], k64[1], v64[0], v64[1], rhist, head, cidx, cell_key, cell_start,
                     hkey, hcell};
  for (void *p : scratch) dfree(s, p);
  return SPH_RT_OK;
}

// --------------------------------------------------------------------------
// Validation of caller arrays that are already on the device (the checks of
// the host path): error bits in flags[0], interior count in flags[1].
// --------------------------------------------------------------------------
__global__ void validate_kernel(int64_t n, int dim, const double *pos, const double *mass,
                                const double *rho, const double *h, const double *sigma0,
                                const int32_t *kind, const int64_t *copy_of, const double *e0,
                                const double *E0, unsigned long long *flags) {
  unsigned long long bad = 0, ni = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int d = 0; d < dim; ++d)
      if (!isfinite(pos[i * dim + d])) bad |= 1ull;
    if (!(isfinite(mass[i]) && mass[i] > 0) || !(isfinite(rho[i]) && rho[i] > 0) ||
        !(isfinite(h[i]) && h[i] > 0))
      bad |= 2ull;
    if (!isfinite(sigma0[i]) || sigma0[i] < 0) bad |= 4ull;
    if (!isfinite(e0[i]) || !isfinite(E0[i])) bad |= 8ull;
    int32_t k = kind[i];
    if (k < 0 || k > 2) bad |= 16ull;
    if (k == SPH_RT_INTERIOR) ++ni;
    if (k == SPH_RT_COPY) {
      if (!copy_of) {
        bad |= 32ull;
      } else {
        int64_t c = copy_of[i];
        if (c < 0 || c >= n || kind[c] != SPH_RT_INTERIOR) bad |= 32ull;
      }
    }
  }
  if (bad) atomicOr(&flags[0], bad);
  if (ni) atomicAdd(&flags[1], ni);
}

sph_rt_status validate_device_particles(sph_rt *s, int64_t n, const double *pos,
                                        const double *mass, const double *rho, const double *h,
                                        const double *sigma0, const int32_t *kind,
                                        const int64_t *copy_of, const double *e0,
                                        const double *E0, int64_t *n_int_out) {
  unsigned long long *flags = nullptr;
  SPH_CUDA(s, cudaMalloc(&flags, 2 * sizeof(unsigned long long)));
  cudaMemsetAsync(flags, 0, 2 * sizeof(unsigned long long), s->stream);
  validate_kernel<<<grid1(s, n), kBlock, 0, s->stream>>>(n, s->dim, pos, mass, rho, h, sigma0,
                                                         kind, copy_of, e0, E0, flags);
  s->launches++;
  unsigned long long hf[2] = {0, 0};
  cudaError_t e1 = cudaGetLastError();
  cudaError_t e2 = cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s->stream);
  cudaError_t e3 = cudaStreamSynchronize(s->stream);
  cudaFree(flags);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    cuda_ok(s, e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3), "validate_kernel");
    return SPH_RT_EDEVICE;
  }
  static const char *what[] = {"non-finite position", "mass, rho and h must be finite and positive",
                               "sigma0 must be finite and >= 0", "non-finite initial energy",
                               "kind out of range", "copy_of must name an interior particle"};
  for (int b = 0; b < 6; ++b)
    if (hf[0] & (1ull << b)) return set_error(s, SPH_RT_EINVAL, what[b]);
  if (hf[1] == 0) return set_error(s, SPH_RT_EINVAL, "no interior particle");
  *n_int_out = (int64_t)hf[1];
  return SPH_RT_OK;
}

}  // namespace sphrt
