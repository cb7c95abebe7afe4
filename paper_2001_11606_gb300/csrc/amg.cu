// amg.cu -- aggregation algebraic multigrid preconditioner (row a5 of the hot
// path) and its V-cycle (inside row a6).
//
// The paper preconditions GMRES with hypre's BoomerAMG, set up once at the
// start of each step and reused in every outer iteration (Sec. 3.2).  This is
// a GPU-native aggregation AMG on the symmetric operator B = V A:
//
//   strength   j is a strong neighbour of i if |B_ij| >= theta sqrt(B_ii B_jj)
//   aggregates Luby-style maximal independent set of the strength graph with
//              fixed hashed priorities (roots), every other node joins the
//              root it is most strongly coupled to; rows without strong
//              neighbours stay unaggregated (left to the smoother)
//   transfer   piecewise-constant prolongation P (tentative), R = P^T
//   Galerkin   B_c = P^T B P: each coarse entry is the sum of the fine entries
//              that map to it, summed in a fixed order (deterministic)
//   smoother   Chebyshev on D^{-1} B with the interval [lmax/8, lmax],
//              lmax from Gershgorin; the coarsest level gets a Chebyshev solve
//              over its whole Gershgorin interval
//
// The V-cycle uses the same polynomial before and after the coarse
// correction, so it is a symmetric positive-definite preconditioner for CG.
//
// Everything runs on the device.  Aggregates and the coarse sparsity are built
// from the first step's operator and kept (config.amg_rebuild = 1 rebuilds
// them every step); the Galerkin values are recomputed every step.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace sphrt {

sph_rt_status exclusive_scan(sph_rt *s, const int64_t *in, int64_t n, int64_t *out);
template <typename MT, typename VT>
sph_rt_status cheb_apply(sph_rt *s, const CsrView<MT> &A, const VT *r, VT *z, VT *d, VT *tmp,
                         int degree, const ChebCoef *cf, bool zero_guess, const Scalars *sc,
                         bool first_step_done = false);
sph_rt_status launch_cheb_slots(sph_rt *s, int first, const double *gersh_dev,
                                const std::vector<int> &mode, const std::vector<int> &degree);

constexpr int kUndecided = 1, kRoot = 2, kNonroot = 0, kIsolated = 3;
constexpr int kHash = 4096;        // shared hash-table slots per coarse row
constexpr int kCoarseTarget = 512;  // stop coarsening at or below this many rows
constexpr int kMaxLevels = 12;
// Levels at or below this many stored entries (~7 MB in FP64, L2-resident)
// may run in the cluster-resident tail (which must hold at least two levels);
// the larger levels post-smooth through A P.
constexpr int64_t kTailMaxNnz = 600000;
static_assert(1 + kMaxLevels <= kChebSlots, "one Chebyshev slot per AMG level");

}  // namespace sphrt

// Source indices of Galerkin sums over a level's entries (k < nnz for an
// off-diagonal entry, nnz + i for a diagonal): 32 bits while nnz + n fits
// (below 2^31 - 1, or unless config.index64), else 64 bits.  Exactly one of
// the two is set.
struct SrcList {
  int32_t *i32 = nullptr;
  int64_t *i64 = nullptr;
};

struct SphLevel {
  int64_t n = 0, nnz = 0;
  // operator (level 0 borrows the fine operator; others own theirs)
  int64_t *ptr = nullptr;
  int32_t *col = nullptr;
  double *val = nullptr, *diag = nullptr, *invdiag = nullptr;
  float *val32 = nullptr, *diag32 = nullptr, *invdiag32 = nullptr;
  // transfer to the next level
  int32_t *agg = nullptr;       // [n] coarse row of each row, -1 if unaggregated
  int64_t *agg_ptr = nullptr;   // [nc+1] members of each coarse row
  int32_t *agg_mem = nullptr;
  int64_t *seg_ptr = nullptr;   // [nnz_c + nc + 1] Galerkin contributions per coarse target
  SrcList seg_src;              // source: k < nnz (off-diagonal entry) or nnz + i (diagonal)
  // vectors of the V-cycle
  double *r = nullptr, *z = nullptr, *res = nullptr, *d = nullptr, *t = nullptr;
  float *r32 = nullptr, *z32 = nullptr, *res32 = nullptr, *d32 = nullptr, *t32 = nullptr;
  int W = 32, U = 4;
  // finest level only: A P (P = this level's aggregation), by fine row
  int64_t nnz_ap = 0;
  int64_t *ap_ptr = nullptr;    // [n + 1]
  int32_t *ap_col = nullptr;    // [nnz_ap] aggregate (next-level row)
  int64_t *ap_seg_ptr = nullptr;  // [nnz_ap + 1] sources of each A P entry
  SrcList ap_seg_src;             // source: k < nnz (off-diagonal entry) or nnz + i (diagonal)
  int64_t *apg_ptr = nullptr;     // [nnz_c + nc + 1] next level's Galerkin sums over A P entries
  int32_t *apg_src = nullptr;     // (P^T (A P): each A P entry (i, K) adds to (agg[i], K))
  double *ap_val = nullptr;     // [nnz_ap]
  float *ap_val32 = nullptr;
  // finest level, mixed form with the V-cycle's CG product (fine_post_smooth = 0):
  // the CG's FP32 search direction p, its product q = B p and w = B z
  float *p32 = nullptr, *q32 = nullptr, *w32 = nullptr;
  std::vector<void *> owned;
};

namespace sphrt {

// Level buffers come from the handle's caching allocator and go back to it
// when the hierarchy is released (after a stream synchronisation).
static void *lvl_alloc(sph_rt *s, SphLevel *L, size_t bytes) {
  void *p = dalloc_bytes(s, bytes > 0 ? bytes : 16);
  if (p) L->owned.push_back(p);
  return p;
}
template <typename T>
static T *lalloc(sph_rt *s, SphLevel *L, size_t count) {
  return static_cast<T *>(lvl_alloc(s, L, sizeof(T) * (count > 0 ? count : 1)));
}
// scratch buffer of one set-up phase
template <typename T>
static T *scratch(sph_rt *s, size_t count) {
  return static_cast<T *>(dalloc_bytes(s, sizeof(T) * (count > 0 ? count : 1)));
}

void amg_release(sph_rt *s) {
  if (!s->levels.empty() && s->cuda_ready) cudaStreamSynchronize(s->stream);
  for (SphLevel *L : s->levels) {
    for (void *p : L->owned) dfree(s, p);
    delete L;
  }
  s->levels.clear();
  s->amg_ready = false;
}

static int gcap(const sph_rt *s, int64_t n, int per_block) {
  int64_t g = ceil_div(n > 0 ? n : 1, per_block);
  int64_t cap = (int64_t)s->num_sms * 8;
  if (cap > kMaxRedBlocks) cap = kMaxRedBlocks;
  return (int)(g < cap ? g : cap);
}

__device__ __forceinline__ uint32_t hash_u32(uint32_t x) {  // integer mixer (Wang-style)
  x = (x ^ 61u) ^ (x >> 16);
  x *= 9u;
  x ^= x >> 4;
  x *= 0x27d4eb2du;
  x ^= x >> 15;
  return x;
}
// priority order: larger hash wins, ties by larger index
__device__ __forceinline__ bool beats(uint32_t i, uint32_t j) {
  uint32_t hi = hash_u32(i), hj = hash_u32(j);
  return hi > hj || (hi == hj && i > j);
}

// ---------------------------------------------------------------------------
// strength and aggregation
// ---------------------------------------------------------------------------
// A warp per row: the row's entries 32 at a time (coalesced), the count of
// strong entries by ballot.
__global__ void strength_kernel(int64_t n, const int64_t *ptr, const int32_t *col,
                                const double *val, const double *diag, double theta2,
                                uint8_t *strong, int *state) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    int cnt = 0;
    const double di = diag[i];
    const int64_t e = ptr[i + 1];
    for (int64_t k0 = ptr[i]; k0 < e; k0 += 32) {
      const int64_t k = k0 + lane;
      bool st = false;
      if (k < e) {
        const int32_t j = col[k];
        // |B_ij| >= theta sqrt(B_ii B_jj), squared: no FP64 square root per entry
        st = j != i && val[k] * val[k] >= theta2 * (di * diag[j]);
        strong[k] = st;
      }
      cnt += __popc(__ballot_sync(0xffffffffu, st));
    }
    if (lane == 0) state[i] = cnt > 0 ? kUndecided : kIsolated;
  }
}

// The MIS passes and the assignment with a warp per row: the row's entries
// 32 at a time (coalesced), decisions by ballot, the assignment's strongest
// root by a warp arg-max under the same order (largest |B_ij|, then smallest
// j; the columns of a row are distinct, so the choice is unique).
__global__ void mis_select_kernel(int64_t n, const int64_t *ptr, const int32_t *col,
                                  const uint8_t *strong, const int *state, uint8_t *cand) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    uint8_t c = 0;
    if (state[i] == kUndecided) {
      c = 1;
      const int64_t e = ptr[i + 1];
      for (int64_t k0 = ptr[i]; k0 < e; k0 += 32) {
        const int64_t k = k0 + lane;
        bool block = false;
        if (k < e && strong[k]) {
          const int32_t j = col[k];
          const int sj = state[j];
          block = sj == kRoot || (sj == kUndecided && beats((uint32_t)j, (uint32_t)i));
        }
        if (__ballot_sync(0xffffffffu, block)) {
          c = 0;
          break;
        }
      }
    }
    if (lane == 0) cand[i] = c;
  }
}

__global__ void mis_apply_kernel(int64_t n, const uint8_t *cand, int *state) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (cand[i]) state[i] = kRoot;
}

__global__ void mis_mark_kernel(int64_t n, const int64_t *ptr, const int32_t *col,
                                const uint8_t *strong, int *state, unsigned *undecided) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned left = 0;
  for (int64_t i = warp; i < n; i += nwarps) {
    if (state[i] != kUndecided) continue;  // warp-uniform
    bool nr = false;
    const int64_t e = ptr[i + 1];
    for (int64_t k0 = ptr[i]; k0 < e && !nr; k0 += 32) {
      const int64_t k = k0 + lane;
      const bool hit = k < e && strong[k] && state[col[k]] == kRoot;
      nr = __ballot_sync(0xffffffffu, hit) != 0;
    }
    if (lane == 0) {
      if (nr) state[i] = kNonroot;
      else ++left;
    }
  }
  if (left) atomicAdd(undecided, left);
}

__global__ void root_flag_kernel(int64_t n, const int *state, int64_t *flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = state[i] == kRoot ? 1 : 0;
}

__global__ void assign_kernel(int64_t n, const int64_t *ptr, const int32_t *col, const double *val,
                              const uint8_t *strong, const int *state, const int64_t *root_id,
                              int32_t *agg, unsigned *members) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const int st = state[i];
    int32_t a = -1;
    if (st == kRoot) {
      a = (int32_t)root_id[i];
    } else if (st == kNonroot) {
      double best = -1.0;
      int32_t bj = -1;
      const int64_t e = ptr[i + 1];
      for (int64_t k = ptr[i] + lane; k < e; k += 32) {
        const int32_t j = col[k];
        if (!strong[k] || state[j] != kRoot) continue;
        const double v = fabs(val[k]);
        if (v > best || (v == best && j < bj)) {
          best = v;
          bj = j;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int32_t oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (oj >= 0 && (bj < 0 || ov > best || (ov == best && oj < bj))) {
          best = ov;
          bj = oj;
        }
      }
      a = bj >= 0 ? (int32_t)root_id[bj] : -1;
    }
    if (lane == 0) {
      agg[i] = a;
      if (a >= 0) atomicAdd(&members[a], 1u);
    }
  }
}

// counting-sort scatter + per-segment insertion sort (shared by the member
// lists and the Galerkin contribution lists): orders each segment by value
// S: the item index type (int32_t, or int64_t for more than 2^31 - 1 items)
template <typename S>
__global__ void bucket_scatter_kernel(int64_t n, const int32_t *bucket, const int64_t *start,
                                      unsigned *cursor, S *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t b = bucket[i];
    if (b < 0) continue;
    int64_t at = start[b] + atomicAdd(&cursor[b], 1u);
    out[at] = (S)i;
  }
}
// Buckets of up to kSmallBucket items are insertion-sorted by one thread
// (bucket_sort_kernel); larger ones, where a quadratic sort in one thread
// would dominate the set-up, by a warp (bucket_rank_kernel).
constexpr int kSmallBucket = 32;
// largest bucket the warp sort stages in shared memory (32 KB a block)
template <typename S>
constexpr int rank_bucket() { return 4096 / (int)sizeof(S); }
template <typename S>
__device__ __forceinline__ void insertion_sort(S *a, int64_t c) {
  for (int64_t t = 1; t < c; ++t) {
    S v = a[t];
    int64_t u = t - 1;
    while (u >= 0 && a[u] > v) {
      a[u + 1] = a[u];
      --u;
    }
    a[u + 1] = v;
  }
}
// A thread per small bucket, sorted in the thread's slice of shared memory
// (one read and one write of the bucket in global memory); 64-bit items, for
// the rare levels past 2^31 sources, are sorted in place.
template <typename S>
__global__ void __launch_bounds__(kBlock) bucket_sort_kernel(int64_t nb, const int64_t *start,
                                                             S *out) {
  __shared__ int32_t stage[kSmallBucket][kBlock];  // item q of thread t at [q][t]
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s0 = start[b], c = start[b + 1] - s0;
    if (c < 2 || c > kSmallBucket) continue;
    if (sizeof(S) != sizeof(int32_t)) {
      insertion_sort(out + s0, c);
      continue;
    }
    for (int q = 0; q < (int)c; ++q) stage[q][threadIdx.x] = (int32_t)out[s0 + q];
    for (int t = 1; t < (int)c; ++t) {
      const int32_t v = stage[t][threadIdx.x];
      int u = t - 1;
      while (u >= 0 && stage[u][threadIdx.x] > v) {
        stage[u + 1][threadIdx.x] = stage[u][threadIdx.x];
        --u;
      }
      stage[u + 1][threadIdx.x] = v;
    }
    for (int q = 0; q < (int)c; ++q) out[s0 + q] = stage[q][threadIdx.x];
  }
}
// A warp takes 32 consecutive buckets and sorts each larger one in turn: the
// items (distinct indices) are staged in shared memory and each is written at
// its rank, the number of smaller items.  Buckets beyond rank_bucket items
// (not met by the aggregation levels, whose sources per target are a few
// hundred at most) fall back to one thread.
template <typename S>
__global__ void bucket_rank_kernel(int64_t nb, const int64_t *start, S *out) {
  constexpr int kRankBucket = rank_bucket<S>();
  __shared__ S stage[kWarpsPerBlock][kRankBucket];
  S *sm = stage[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t b0 = warp * 32; b0 < nb; b0 += nwarps * 32) {
    const int64_t b = b0 + lane;
    const int64_t c = b < nb ? start[b + 1] - start[b] : 0;
    unsigned m = __ballot_sync(0xffffffffu, c > kSmallBucket);
    while (m) {
      const int t = __ffs(m) - 1;
      m &= m - 1;
      const int64_t bb = b0 + t;
      const int64_t s0 = start[bb], cc = start[bb + 1] - s0;
      if (cc > kRankBucket) {
        if (lane == 0) insertion_sort(out + s0, cc);
        __syncwarp();
        continue;
      }
      for (int64_t k = lane; k < cc; k += 32) sm[k] = out[s0 + k];
      __syncwarp();
      for (int64_t k = lane; k < cc; k += 32) {
        const S v = sm[k];
        int rank = 0;
        for (int q = 0; q < (int)cc; ++q) rank += sm[q] < v;
        out[s0 + rank] = v;
      }
      __syncwarp();
    }
  }
}

__global__ void u32_to_i64_kernel(int64_t n, const unsigned *in, int64_t *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

// ---------------------------------------------------------------------------
// coarse sparsity: one block per coarse row, shared-memory hash of the coarse
// columns reached from the members' rows, then sorted.
// ---------------------------------------------------------------------------
template <bool FILL>
__global__ void coarse_struct_kernel(int64_t nc, const int64_t *agg_ptr, const int32_t *agg_mem,
                                     const int64_t *ptr, const int32_t *col, const int32_t *agg,
                                     int64_t *ccount, const int64_t *cptr, int32_t *ccol,
                                     int32_t *tgt, int64_t nnz_c, int32_t *tgt_diag,
                                     int *overflow) {
  __shared__ int32_t table[kHash];
  __shared__ int32_t keys[kHash / 2];
  __shared__ int nkeys;
  for (int64_t I = blockIdx.x; I < nc; I += gridDim.x) {
    for (int t = threadIdx.x; t < kHash; t += blockDim.x) table[t] = 0x7fffffff;
    if (threadIdx.x == 0) nkeys = 0;
    __syncthreads();
    const int64_t m0 = agg_ptr[I], m1 = agg_ptr[I + 1];
    // insert
    for (int64_t m = m0; m < m1; ++m) {
      int32_t i = agg_mem[m];
      for (int64_t k = ptr[i] + threadIdx.x; k < ptr[i + 1]; k += blockDim.x) {
        int32_t J = agg[col[k]];
        if (J < 0 || J == (int32_t)I) continue;
        uint32_t hsh = hash_u32((uint32_t)J) & (kHash - 1);
        for (int probe = 0; probe < kHash; ++probe) {
          int32_t prev = atomicCAS(&table[hsh], 0x7fffffff, J);
          if (prev == 0x7fffffff) {
            atomicAdd(&nkeys, 1);
            break;
          }
          if (prev == J) break;
          hsh = (hsh + 1) & (kHash - 1);
        }
      }
    }
    __syncthreads();
    int cnt = nkeys;
    if (cnt > kHash / 2) {  // too wide for the table's load factor: give up on this level
      if (threadIdx.x == 0) atomicExch(overflow, 1);
      __syncthreads();
      continue;
    }
    // compact the keys (any order), pad to a power of two and sort ascending
    __shared__ int ncomp;
    if (threadIdx.x == 0) ncomp = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < kHash; t += blockDim.x) {
      int32_t v = table[t];
      if (v != 0x7fffffff) keys[atomicAdd(&ncomp, 1)] = v;
    }
    int P2 = 1;
    while (P2 < cnt) P2 <<= 1;
    __syncthreads();
    for (int t = cnt + threadIdx.x; t < P2; t += blockDim.x) keys[t] = 0x7fffffff;
    __syncthreads();
    for (int k = 2; k <= P2; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < P2; t += blockDim.x) {
          int u = t ^ j;
          if (u > t) {
            int32_t a = keys[t], b = keys[u];
            bool up = (t & k) == 0;
            if ((a > b) == up) {
              keys[t] = b;
              keys[u] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    if (!FILL) {
      if (threadIdx.x == 0) ccount[I] = cnt;
    } else {
      const int64_t base = cptr[I];
      for (int t = threadIdx.x; t < cnt; t += blockDim.x) ccol[base + t] = keys[t];
      for (int64_t m = m0; m < m1; ++m) {
        int32_t i = agg_mem[m];
        if (threadIdx.x == 0) tgt_diag[i] = (int32_t)(nnz_c + I);
        for (int64_t k = ptr[i] + threadIdx.x; k < ptr[i + 1]; k += blockDim.x) {
          int32_t J = agg[col[k]];
          int32_t tg = -1;
          if (J == (int32_t)I) {
            tg = (int32_t)(nnz_c + I);
          } else if (J >= 0) {
            int lo = 0, hi = cnt;  // lower_bound
            while (lo < hi) {
              int mid = (lo + hi) >> 1;
              if (keys[mid] < J) lo = mid + 1;
              else hi = mid;
            }
            tg = (int32_t)(base + lo);
          }
          tgt[k] = tg;
        }
      }
    }
    __syncthreads();
  }
}

// targets of the fine diagonal entries of unaggregated rows stay -1
__global__ void fill_i32_kernel(int64_t n, int32_t v, int32_t *a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

__global__ void target_count_kernel(int64_t nsrc, const int32_t *tgt, unsigned *cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nsrc;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t t = tgt[i];
    if (t >= 0) atomicAdd(&cnt[t], 1u);
  }
}

// Galerkin values: thread per coarse target, fixed-order sum of its sources
// (8 source indices loaded before their gathers, so the gathers overlap).  A
// warp adds as many slots of a batch as its longest segment has left (most
// A P targets have 3-4 sources): the additions a lane skips would add +0.0,
// and a sum that starts at +0.0 is unchanged by them, so the result is that of
// adding all 8 slots.
// T: the hierarchy's value type (FP32 in the mixed form: its sums are formed
// from the FP32 fine values directly).
// S: the source index type (SrcList).
template <typename T, typename S>
__global__ void galerkin_kernel(int64_t nnz_c, int64_t nc, const int64_t *seg_ptr,
                                const S *seg_src, int64_t nnz_f, const T *val_f,
                                const T *diag_f, T *val_c, T *diag_c, T *invdiag_c) {
  constexpr int G = 8;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz_c + nc;
       t += (int64_t)gridDim.x * blockDim.x) {
    const unsigned mask = __activemask();
    T acc = T(0);
    const int64_t u1 = seg_ptr[t + 1];
    for (int64_t u = seg_ptr[t];; u += G) {
      const int64_t left = u1 - u;
      const int m = __reduce_max_sync(mask, left <= 0 ? 0 : (left < G ? (int)left : G));
      if (m == 0) break;  // uniform over the lanes of `mask`
      S src[G];
#pragma unroll
      for (int g = 0; g < G; ++g) src[g] = u + g < u1 ? __ldg(seg_src + u + g) : S(-1);
      T v[G];
#pragma unroll
      for (int g = 0; g < G; ++g)
        v[g] = src[g] < 0 ? T(0) : (src[g] < nnz_f ? __ldg(val_f + src[g]) : __ldg(diag_f + (src[g] - nnz_f)));
#pragma unroll 1
      for (int g = 0; g < m; ++g) {
        acc += v[0];  // sources in order; a shorter segment's padding adds +0.0
#pragma unroll
        for (int q = 0; q + 1 < G; ++q) v[q] = v[q + 1];
      }
    }
    if (t < nnz_c) {
      val_c[t] = acc;
    } else {
      diag_c[t - nnz_c] = acc;
      invdiag_c[t - nnz_c] = T(1) / acc;
    }
  }
}

// Gershgorin bound of D^{-1} A for a level: max_i sum_j |A_ij| / A_ii
template <typename T>
__global__ void gersh_kernel(int64_t n, const int64_t *ptr, const T *val, const T *diag,
                             double *partials, unsigned *counter, double *out) {
  double g = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double sacc = 0.0;
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) sacc += fabs((double)val[k]);
    g = fmax(g, sacc / (double)diag[i]);
  }
  __shared__ double sh[32];
  g = block_max(g, sh);
  double part[1] = {g}, o[1];
  const bool mx[1] = {true};
  if (last_block_combine<1>(part, partials, counter, o, mx) && threadIdx.x == 0) *out = o[0];
}

template <typename S, typename D>
__global__ void convert_kernel(int64_t n, const S *in, D *out) {
  pdl_wait();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (D)in[i];
}

// ---------------------------------------------------------------------------
// V-cycle kernels
// ---------------------------------------------------------------------------
// PRE: load the row operands before the row sums (coarse levels) or after
// them (finest level), as in cheb_step_body.
template <int W, int U, typename MT, typename VT, bool PRE>
__device__ __forceinline__ void resid_level_body(const CsrView<MT> &A, const VT *r, const VT *z,
                                                 VT *res, const Scalars *sc, int *wflag) {
  pdl_wait();
  if (sc && sc->done) {
    mark_work(wflag, 0);
    return;
  }
  mark_work(wflag, 1);
  const int own = tile_own_row<W>(threadIdx.x & 31);
  int64_t r0, r1;
  warp_rows<W>(A.n, r0, r1);
  for (int64_t base = r0; base < r1; base += 32) {
    const int rows = (int)(r1 - base < 32 ? r1 - base : 32);
    const int64_t i = base + own;
    const bool active = own < rows;
    VT ri = VT(0), dg = VT(0), zi = VT(0);
    auto operands = [&]() {
      ri = r[i];
      dg = (VT)A.diag[i];
      zi = z[i];
    };
    if (PRE && active) operands();
    const VT s = tile_row_sums<W, U, MT, VT>(base, rows, A.ptr, A.col, A.val, z);
    if (active) {
      if (!PRE) operands();
      res[i] = ri - fmadd(dg, zi, s);
    }
  }
}
// one body, two names: finest level vs coarse levels in profiles
template <int W, int U, typename MT, typename VT>
__global__ void __launch_bounds__(kBlock, kCoarseMinBlocks) resid_level_kernel(CsrView<MT> A, const VT *r, const VT *z, VT *res,
                                   const Scalars *sc, int *wflag) {
  resid_level_body<W, U, MT, VT, true>(A, r, z, res, sc, wflag);
}
template <int W, int U, typename MT, typename VT>
__global__ void __launch_bounds__(kBlock, sweep_min_blocks(U)) fine_resid_level_kernel(CsrView<MT> A, const VT *r, const VT *z, VT *res,
                                        const Scalars *sc, int *wflag) {
  resid_level_body<W, U, MT, VT, false>(A, r, z, res, sc, wflag);
}

// Sum of res over the members [m0, m1) of an aggregate, in member order.
// Aggregates have ~6 members: 8 member indices are loaded before their
// gathers, so an aggregate costs two dependent round trips instead of two per
// member.
template <typename VT>
__device__ __forceinline__ VT aggregate_sum(int64_t m0, int64_t m1, const int32_t *agg_mem,
                                            const VT *res) {
  constexpr int G = 8;
  VT acc = 0;
  for (int64_t m = m0; m < m1; m += G) {
    int32_t j[G];
#pragma unroll
    for (int g = 0; g < G; ++g) j[g] = m + g < m1 ? agg_mem[m + g] : -1;
    VT v[G];
#pragma unroll
    for (int g = 0; g < G; ++g) v[g] = j[g] >= 0 ? res[j[g]] : VT(0);
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (j[g] >= 0) acc += v[g];
  }
  return acc;
}

template <typename VT>
__global__ void restrict_kernel(int64_t nc, const int64_t *agg_ptr, const int32_t *agg_mem,
                                const VT *res, VT *rc, const Scalars *sc) {
  pdl_wait();
  if (sc && sc->done) return;
  for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < nc;
       I += (int64_t)gridDim.x * blockDim.x) {
    const VT acc = aggregate_sum(agg_ptr[I], agg_ptr[I + 1], agg_mem, res);
    rc[I] = acc;
  }
}

// Restriction fused with the next level's zero-guess smoother start
// (cheb_init_zero_kernel's arithmetic): rc = P^T res; d_c = z_c = D_c^{-1} rc / theta_c.
template <typename MT, typename VT>
__global__ void restrict_init_kernel(int64_t nc, const int64_t *agg_ptr, const int32_t *agg_mem,
                                     const VT *res, VT *rc, const MT *invdiag_c,
                                     const ChebCoef *cf_c, VT *d_c, VT *z_c, const Scalars *sc) {
  pdl_wait();
  if (sc && sc->done) return;
  const double inv_theta = cf_c->inv_theta;
  for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < nc;
       I += (int64_t)gridDim.x * blockDim.x) {
    const VT acc = aggregate_sum(agg_ptr[I], agg_ptr[I + 1], agg_mem, res);
    rc[I] = acc;
    VT di = (VT)(inv_theta * (double)invdiag_c[I] * (double)acc);
    d_c[I] = di;
    z_c[I] = di;
  }
}

template <typename VT>
__global__ void prolong_kernel(int64_t n, const int32_t *agg, const VT *zc, VT *z,
                               const Scalars *sc) {
  pdl_wait();
  if (sc && sc->done) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = agg[i];
    if (a >= 0) z[i] += zc[a];
  }
}

// Coarsest level: the whole Chebyshev solve (zero guess, `degree` steps over
// [lo, hi]) in ONE block with the level's operator AND vectors staged in
// shared memory, so every step is a few shared-memory passes instead of a
// separate launch.  Used when the level fits (coarse_smem_bytes <= 200 KiB).
__host__ inline size_t coarse_smem_bytes(int64_t n, int64_t nnz, size_t mt, size_t vt) {
  size_t b = (size_t)nnz * (mt + 4) + (size_t)(n + 1) * 4 + (size_t)n * (2 * mt + 4 * vt);
  return (b + 15) & ~(size_t)15;
}
constexpr size_t kCoarseSmemMax = 200 * 1024;

// Body of the coarsest-level solve for one block (blockDim.x threads, the
// shared-memory buffer of coarse_smem_bytes(n, nnz, sizeof(VT), sizeof(VT)));
// also run by one block of the cluster-resident V-cycle tail.  MT / GT: type
// of the level's operator / vectors in global memory; VT: the type the solve
// is staged and computed in (the operator is converted when it is staged).
template <typename MT, typename VT, typename GT = VT>
__device__ void coarse_cheb_body(const CsrView<MT> &A, const GT *r_g, GT *z_g, const ChebCoef *cf,
                                 int degree, unsigned char *smem_raw) {
  const int n = (int)A.n, nnz = (int)A.nnz;
  // layout: values, diag, invdiag | r, z0, z1, d (all VT) | cols, ptr (int32)
  VT *val = reinterpret_cast<VT *>(smem_raw);
  VT *dg = val + nnz, *idg = dg + n;
  VT *r = reinterpret_cast<VT *>(idg + n);
  VT *zb0 = r + n, *zb1 = zb0 + n, *d = zb1 + n;
  int *col = reinterpret_cast<int *>(d + n);
  int *ptr = col + nnz;
  const int64_t base = A.ptr[0];
  const double inv_theta = cf->inv_theta;
  // the step coefficients, staged once: a global load per step would put an
  // L2 round trip on the critical path of every step
  __shared__ VT cs1[kChebMaxDeg], cs2[kChebMaxDeg];
  for (int k = threadIdx.x; k < degree && k < kChebMaxDeg; k += blockDim.x) {
    cs1[k] = (VT)cf->c1[k];
    cs2[k] = (VT)cf->c2[k];
  }
  for (int k = threadIdx.x; k < nnz; k += blockDim.x) {
    val[k] = (VT)A.val[base + k];
    col[k] = A.col[base + k];
  }
  for (int i = threadIdx.x; i <= n; i += blockDim.x) ptr[i] = (int)(A.ptr[i] - base);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    dg[i] = (VT)A.diag[i];
    idg[i] = (VT)A.invdiag[i];
    VT ri = (VT)r_g[i];
    r[i] = ri;
    VT di = (VT)(inv_theta * (double)A.invdiag[i] * (double)ri);
    d[i] = di;
    zb0[i] = di;
  }
  __syncthreads();
  VT *zin = zb0, *zout = zb1;
  for (int k = 1; k < degree; ++k) {
    const VT c1 = cs1[k], c2 = cs2[k];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {  // thread per row: no shuffles
      // 8 column / value loads, then 8 gathers in flight, summed in entry order
      VT s = 0;
      const int e = ptr[i + 1];
      for (int kk = ptr[i]; kk < e; kk += 8) {
        int cc[8];
        VT vv[8], zz[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          cc[u] = kk + u < e ? col[kk + u] : -1;
          vv[u] = kk + u < e ? val[kk + u] : VT(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) zz[u] = cc[u] >= 0 ? zin[cc[u]] : VT(0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (cc[u] >= 0) s = fmadd(vv[u], zz[u], s);
      }
      VT res = r[i] - fmadd((VT)dg[i], zin[i], s);
      VT di = fmadd(c1, d[i], (c2 * (VT)idg[i]) * res);
      d[i] = di;
      zout[i] = zin[i] + di;
    }
    __syncthreads();
    VT *t = zin;
    zin = zout;
    zout = t;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) z_g[i] = (GT)zin[i];
}

template <typename MT, typename VT, typename GT>
__global__ void __launch_bounds__(1024) coarse_cheb_kernel(CsrView<MT> A, const GT *r_g, GT *z_g,
                                                           const ChebCoef *cf, int degree,
                                                           const Scalars *sc) {
  pdl_wait();
  if (sc && sc->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  coarse_cheb_body<MT, VT, GT>(A, r_g, z_g, cf, degree, smem_raw);
}

// ---------------------------------------------------------------------------
// A P of the finest level.  After the coarse correction e_c, the first
// post-smoothing step needs r - A (z_pre + P e_c) = res - (A P) e_c, where
// res = r - A z_pre is the residual already formed before the restriction.
// A P has one entry per (fine row, distinct aggregate among the row's own
// and its columns' aggregates) -- about a sixth of A's entries -- so that
// step reads A P instead of A (and absorbs the prolongation).  Its entries
// are kept in first-occurrence order along the row (own aggregate first).
// ---------------------------------------------------------------------------
// structure, pass 1 (per fine row, one thread): distinct aggregates written
// uncompacted at tmp[ptr[i] + i ..], relative positions in ap_map / ap_dmap
__global__ void ap_structure_kernel(int64_t n, const int64_t *ptr, const int32_t *col,
                                    const int32_t *agg, int32_t *tmp, int64_t *cnt,
                                    int32_t *ap_map, int32_t *ap_dmap) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t *keys = tmp + ptr[i] + i;
    int32_t m = 0;
    const int32_t a0 = agg[i];
    if (a0 >= 0) keys[m++] = a0;
    ap_dmap[i] = a0 >= 0 ? 0 : -1;
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
      const int32_t K = agg[col[k]];
      int32_t pos = -1;
      if (K >= 0) {
        for (int32_t q = 0; q < m; ++q)
          if (keys[q] == K) {
            pos = q;
            break;
          }
        if (pos < 0) {
          pos = m;
          keys[m++] = K;
        }
      }
      ap_map[k] = pos;
    }
    cnt[i] = m;
  }
}
// The same pass with a warp per row: the row's entries are read 32 at a time
// (coalesced), equal aggregates within a batch are grouped with match_any, and
// a batch's new aggregates are appended in lane order after the keys of the
// earlier batches, which the warp keeps in shared memory -- so keys, positions
// and counts are exactly those of ap_structure_kernel.  A row with more than
// kApWarpKeys distinct aggregates sets *overflow; the caller then runs
// ap_structure_kernel instead.
constexpr int kApWarpKeys = 128;
__global__ void ap_structure_warp_kernel(int64_t n, const int64_t *ptr, const int32_t *col,
                                         const int32_t *agg, int32_t *tmp, int64_t *cnt,
                                         int32_t *ap_map, int32_t *ap_dmap, int *overflow) {
  __shared__ int32_t keys_sh[kWarpsPerBlock][kApWarpKeys];
  int32_t *ks = keys_sh[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const int32_t a0 = agg[i];
    int m = 0;  // keys so far (warp-uniform)
    if (a0 >= 0) {
      if (lane == 0) ks[0] = a0;
      m = 1;
    }
    if (lane == 0) ap_dmap[i] = a0 >= 0 ? 0 : -1;
    __syncwarp();
    bool over = false;
    const int64_t b = ptr[i], e = ptr[i + 1];
    for (int64_t k0 = b; k0 < e; k0 += 32) {
      const int64_t k = k0 + lane;
      const bool valid = k < e;
      const int32_t K = valid ? agg[col[k]] : -1;
      int pos = -1;
      if (K >= 0)
        for (int q = 0; q < m; ++q)
          if (ks[q] == K) {
            pos = q;
            break;
          }
      // first lane of each group of equal new aggregates appends it
      const unsigned peers = __match_any_sync(0xffffffffu, K);
      const int leader = __ffs(peers) - 1;
      const bool fresh = K >= 0 && pos < 0;
      const bool adds = fresh && lane == leader;
      const unsigned newmask = __ballot_sync(0xffffffffu, adds);
      int mine = adds ? m + __popc(newmask & lt) : -1;
      if (adds && mine < kApWarpKeys) ks[mine] = K;
      mine = __shfl_sync(0xffffffffu, mine, leader);
      if (fresh) pos = mine;
      m += __popc(newmask);
      if (m > kApWarpKeys) {  // warp-uniform; the keys past the list were not kept
        over = true;
        break;
      }
      __syncwarp();
      if (valid) ap_map[k] = pos;
    }
    if (over) {
      if (lane == 0) *overflow = 1;
      continue;
    }
    int32_t *keys = tmp + b + i;
    for (int q = lane; q < m; q += 32) keys[q] = ks[q];
    if (lane == 0) cnt[i] = m;
    __syncwarp();
  }
}
// pass 2: compact the keys and make the positions absolute
__global__ void ap_compact_kernel(int64_t n, const int64_t *ptr, const int32_t *tmp,
                                  const int64_t *ap_ptr, int32_t *ap_col, int32_t *ap_map,
                                  int32_t *ap_dmap) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = ap_ptr[i];
    const int32_t *keys = tmp + ptr[i] + i;
    for (int64_t q = 0; q < ap_ptr[i + 1] - b; ++q) ap_col[b + q] = keys[q];
    if (ap_dmap[i] >= 0) ap_dmap[i] = (int32_t)b + ap_dmap[i];
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k)
      if (ap_map[k] >= 0) ap_map[k] = (int32_t)b + ap_map[k];
  }
}
// The values (every step) are fixed-order sums of each entry's sources, the
// same gather-sum as the Galerkin product (galerkin_kernel).  The next
// level's operator P^T A P = P^T (A P) is then summed from the A P entries
// (about a sixth as many sources as A's entries): entry (i, K) of A P adds to
// coarse entry (agg[i], K), the diagonal when K = agg[i].
__global__ void ap_galerkin_target_kernel(int64_t n, const int64_t *ap_ptr, const int32_t *ap_col,
                                          const int32_t *agg, int64_t nnz_c, const int64_t *cptr,
                                          const int32_t *ccol, int32_t *tgt, int *missing) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t I = agg[i];
    for (int64_t q = ap_ptr[i]; q < ap_ptr[i + 1]; ++q) {
      const int32_t K = ap_col[q];
      int64_t t = -1;
      if (I >= 0) {
        if (K == I) {
          t = nnz_c + I;
        } else {  // binary search in the sorted coarse row I
          int64_t lo = cptr[I], hi = cptr[I + 1];
          while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            if (ccol[mid] < K) lo = mid + 1; else hi = mid;
          }
          if (lo < cptr[I + 1] && ccol[lo] == K) t = lo;
          else *missing = 1;
        }
      }
      tgt[q] = (int32_t)t;
    }
  }
}

// First post-smoothing step of a level with the prolongation folded in:
// z = z_pre + P e_c, res2 = res - (A P) e_c (= r - A z), d = c2 D^{-1} res2
// (step 0 from a nonzero guess), z_out = z + d.  z_out may be z_pre.
// DOT (finest level, smoother degree 1, where this is the V-cycle's last
// sweep): also the preconditioned inner product of DotFuse over the new z.
template <int W, int U, typename MT, typename VT, bool PRE, bool DOT>
__device__ __forceinline__ void post_ap_body(int64_t n, const int64_t *ap_ptr,
                                             const int32_t *ap_col, const MT *ap_val,
                                             const int32_t *agg, const VT *ec, const VT *z_pre,
                                             const VT *res, const MT *invdiag, const ChebCoef *cf,
                                             VT *d, VT *z_out, const Scalars *sc, int *wflag,
                                             const DotFuse &df) {
  pdl_wait();
  if (sc && sc->done) {
    mark_work(wflag, 0);
    return;
  }
  mark_work(wflag, 1);
  const VT c2 = (VT)cf->inv_theta;
  const int own = tile_own_row<W>(threadIdx.x & 31);
  int64_t r0, r1;
  warp_rows<W>(n, r0, r1);
  double da = 0.0, db = 0.0;  // (r, z) and (r, z_old) partials (DOT)
  for (int64_t base = r0; base < r1; base += 32) {
    const int rows = (int)(r1 - base < 32 ? r1 - base : 32);
    const int64_t i = base + own;
    const bool active = own < rows;
    VT zp = VT(0), rs = VT(0), idg = VT(0), pe = VT(0);
    auto operands = [&]() {
      zp = z_pre[i];
      rs = res[i];
      idg = (VT)invdiag[i];
      const int32_t a = agg[i];
      pe = a >= 0 ? ec[a] : VT(0);
    };
    if (PRE && active) operands();
    const VT s = tile_row_sums<W, U, MT, VT>(base, rows, ap_ptr, ap_col, ap_val, ec);
    if (active) {
      if (!PRE) operands();
      const VT zi = zp + pe;
      const VT di = (c2 * idg) * (rs - s);
      const VT zo = zi + di;
      d[i] = di;
      z_out[i] = zo;
      if (DOT) {
        const double ri = df.r[i], zn = (double)zo;
        if (df.flex) {
          if (!df.first) db += ri * df.z64[i];
          df.z64[i] = zn;
        }
        da += ri * zn;
      }
    }
  }
  if (DOT) {
    __shared__ double sh[32];
    da = block_sum(da, sh);
    __syncthreads();
    db = block_sum(db, sh);
    double part[2] = {da, db}, out[2];
    const bool mx[2] = {false, false};
    if (last_block_combine<2>(part, df.partials, &df.sc->counter, out, mx) && threadIdx.x == 0) {
      Scalars *w = df.sc;
      if (!df.first) w->beta = (df.flex ? out[0] - out[1] : out[0]) / w->rho;
      w->rho = out[0];
    }
  }
}
// the same sweep under two names: finest level / coarser levels in profiles
template <int W, int U, typename MT, typename VT>
__global__ void __launch_bounds__(kBlock, sweep_min_blocks(U))
    fine_post_ap_kernel(int64_t n, const int64_t *ap_ptr, const int32_t *ap_col,
                        const MT *ap_val, const int32_t *agg, const VT *ec, const VT *z_pre,
                        const VT *res, const MT *invdiag, const ChebCoef *cf, VT *d, VT *z_out,
                        const Scalars *sc, int *wflag) {
  post_ap_body<W, U, MT, VT, false, false>(n, ap_ptr, ap_col, ap_val, agg, ec, z_pre, res,
                                           invdiag, cf, d, z_out, sc, wflag, DotFuse{});
}
template <int W, int U, typename MT, typename VT>
__global__ void __launch_bounds__(kBlock, sweep_min_blocks(U))
    fine_post_ap_dot_kernel(int64_t n, const int64_t *ap_ptr, const int32_t *ap_col,
                            const MT *ap_val, const int32_t *agg, const VT *ec, const VT *z_pre,
                            const VT *res, const MT *invdiag, const ChebCoef *cf, VT *d,
                            VT *z_out, const Scalars *sc, int *wflag, const DotFuse df) {
  post_ap_body<W, U, MT, VT, false, true>(n, ap_ptr, ap_col, ap_val, agg, ec, z_pre, res, invdiag,
                                          cf, d, z_out, sc, wflag, df);
}
template <int W, int U, typename MT, typename VT>
__global__ void __launch_bounds__(kBlock, kCoarseMinBlocks)
    post_ap_kernel(int64_t n, const int64_t *ap_ptr, const int32_t *ap_col, const MT *ap_val,
                   const int32_t *agg, const VT *ec, const VT *z_pre, const VT *res,
                   const MT *invdiag, const ChebCoef *cf, VT *d, VT *z_out, const Scalars *sc,
                   int *wflag) {
  post_ap_body<W, U, MT, VT, true, false>(n, ap_ptr, ap_col, ap_val, agg, ec, z_pre, res, invdiag,
                                          cf, d, z_out, sc, wflag, DotFuse{});
}

// ---------------------------------------------------------------------------
// The finest level without post-smoothing, for the CG whose product comes from
// the V-cycle (config.fine_post_smooth = 0).  With the zero-guess smoother
// start z_pre = c0 D^{-1} r, the residual res = r - B z_pre (the V-cycle's
// first sweep) and the coarse correction e_c, the preconditioned residual is
// z = z_pre + P e_c, and
//   B z = B z_pre + (B P) e_c = (r - res) + (res - res2) = r - res2,
// res2 = res - (A P) e_c -- the A P sweep gives B z without a sweep of B.  The
// CG then needs no product sweep of its own: q = B p = B z + beta q_old.
// The sweep also forms the iteration's inner products, so alpha and beta are
// known when it ends (one reduction per iteration):
//   a = (r, z), b = (r, z_old), c = (z, B z), d = (z, q_old), e = (p_old, B z)
//   beta = (a - b) / rho_old     (flexible, Polak-Ribiere: the V-cycle without
//                                 post-smoothing is not symmetric)
//   (p, q) = (z + beta p_old, B z + beta q_old) = c + beta (d + e) + beta^2 (p_old, q_old)
//   alpha = a / (p, q)
// first = 1 (the first iteration of a solve): p = z, beta = 0, (p, q) = c.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fcg_scalars(const double (&o)[5], int first, Scalars *sc) {
  const double a = o[0];
  double beta = 0.0, pq = o[2];
  if (!first) {
    beta = (a - o[1]) / sc->rho;
    pq = o[2] + beta * (o[3] + o[4]) + beta * beta * sc->pq;
  }
  sc->beta = beta;
  sc->rho = a;
  sc->pq = pq;
  sc->pfirst = first;
  if (!(pq > 0.0) || !(pq < 1e308) || !(a == a)) {  // loss of definiteness or NaN
    sc->breakdown = 1;
    sc->done = 1;
  } else {
    sc->alpha = a / pq;
  }
}

// Row epilogue shared by the two forms of the last sweep: z and B z of row i
// and the five inner-product partials.
template <typename VT>
__device__ __forceinline__ void fcg_row(int64_t i, VT zn, VT wn, const VT *r, VT *z, VT *w,
                                        const VT *p, const VT *q, int first, double (&acc)[5]) {
  const double ri = (double)r[i], zd = (double)zn, wd = (double)wn;
  acc[0] += ri * zd;
  acc[2] += zd * wd;
  if (!first) {
    acc[1] += ri * (double)z[i];
    acc[3] += zd * (double)q[i];
    acc[4] += (double)p[i] * wd;
  }
  z[i] = zn;
  w[i] = wn;
}

template <typename VT>
__device__ __forceinline__ void fcg_reduce(double (&acc)[5], int first, Scalars *sc,
                                           double *partials) {
  __shared__ double sh[32];
  for (int k = 0; k < 5; ++k) {
    acc[k] = block_sum(acc[k], sh);
    __syncthreads();
  }
  double out[5];
  const bool mx[5] = {false, false, false, false, false};
  if (last_block_combine<5>(acc, partials, &sc->counter, out, mx) && threadIdx.x == 0)
    fcg_scalars(out, first, sc);
}

// The A P sweep: res2 = res - (A P) e_c, z = z_pre + P e_c, B z = r - res2.
// (five FP64 partials on top of the row tile: compiled for the resident blocks
// per SM at which the register file holds them without spilling -- 4 with FP32
// vectors (64 registers), 3 with FP64 ones (72))
template <typename VT>
__host__ __device__ constexpr int fcg_min_blocks() {
  return sizeof(VT) == sizeof(float) ? 4 : 3;
}
template <int W, int U, typename MT, typename VT>
__global__ void __launch_bounds__(kBlock, fcg_min_blocks<VT>())
    fine_ap_cg_kernel(int64_t n, const int64_t *ap_ptr, const int32_t *ap_col, const MT *ap_val,
                      const int32_t *agg, const VT *ec, const VT *z_pre, const VT *res,
                      const VT *r, VT *z, VT *w, const VT *p, const VT *q, int first, Scalars *sc,
                      double *partials, int *wflag) {
  pdl_wait();
  if (sc->done) {
    mark_work(wflag, 0);
    return;
  }
  mark_work(wflag, 1);
  const int own = tile_own_row<W>(threadIdx.x & 31);
  int64_t r0, r1;
  warp_rows<W>(n, r0, r1);
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t base = r0; base < r1; base += 32) {
    const int rows = (int)(r1 - base < 32 ? r1 - base : 32);
    const int64_t i = base + own;
    const VT s = tile_row_sums<W, U, MT, VT>(base, rows, ap_ptr, ap_col, ap_val, ec);
    if (own < rows) {
      const int32_t a = agg[i];
      const VT pe = a >= 0 ? ec[a] : VT(0);
      const VT zn = z_pre[i] + pe;
      const VT res2 = res[i] - s;
      fcg_row<VT>(i, zn, r[i] - res2, r, z, w, p, q, first, acc);
    }
  }
  fcg_reduce<VT>(acc, first, sc, partials);
}

// Without A P (operators below the A P threshold): z = z_pre + P e_c into t,
// then B z by a sweep of B.
template <typename VT>
__global__ void fcg_prolong_kernel(int64_t n, const int32_t *agg, const VT *ec, const VT *z_pre,
                                   VT *t, const Scalars *sc) {
  pdl_wait();
  if (sc->done) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = agg[i];
    t[i] = z_pre[i] + (a >= 0 ? ec[a] : VT(0));
  }
}
template <int W, int U, typename MT, typename VT>
__global__ void __launch_bounds__(kBlock, fcg_min_blocks<VT>())
    fcg_spmv_dot_kernel(CsrView<MT> A, const VT *t, const VT *r, VT *z, VT *w, const VT *p,
                        const VT *q, int first, Scalars *sc, double *partials, int *wflag) {
  pdl_wait();
  if (sc->done) {
    mark_work(wflag, 0);
    return;
  }
  mark_work(wflag, 1);
  const int own = tile_own_row<W>(threadIdx.x & 31);
  int64_t r0, r1;
  warp_rows<W>(A.n, r0, r1);
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t base = r0; base < r1; base += 32) {
    const int rows = (int)(r1 - base < 32 ? r1 - base : 32);
    const int64_t i = base + own;
    const VT s = tile_row_sums<W, U, MT, VT>(base, rows, A.ptr, A.col, A.val, t);
    if (own < rows) {
      const VT ti = t[i];
      fcg_row<VT>(i, ti, fmadd((VT)A.diag[i], ti, s), r, z, w, p, q, first, acc);
    }
  }
  fcg_reduce<VT>(acc, first, sc, partials);
}

// ---------------------------------------------------------------------------
// Cluster-resident V-cycle tail: the levels from `tail_level` down (small
// operators that live in L2) run as ONE launch of one thread-block cluster.
// Phases that depend on other rows are separated by cluster barriers instead
// of kernel boundaries, so a small level costs a few barrier round trips
// instead of several launches.  Rows of a level are split into contiguous
// ranges, one per block; every phase repeats the arithmetic of the per-level
// kernels exactly (same W-lane row sums, same update expressions, same
// restriction order), so the result is bitwise that of the launched V-cycle.
// Vectors written inside the launch are read with L2 (.cg) loads.  All
// control flow is uniform over the cluster: every block passes every barrier.
// ---------------------------------------------------------------------------
template <typename T>
struct TailLevel {
  CsrView<T> A;
  const int32_t *agg;      // [n] row of the next level (-1: unaggregated)
  const int64_t *agg_ptr;  // [n_next + 1] members of each next-level row
  const int32_t *agg_mem;
  T *r, *z, *res, *d, *t;
  const ChebCoef *cf;
  int deg;
};
template <typename T>
struct TailParams {
  int nlev;        // levels in the tail; the last one is the coarsest
  int coarse_smem; // 1: the coarsest solve runs in block 0 from shared memory
  int coarse_fp32; // 1: that solve is staged and computed in FP32
  TailLevel<T> L[kMaxLevels];
};

template <int W, typename MT, typename VT>
__device__ __forceinline__ VT row_dot_cg(int64_t beg, int64_t end, const int32_t *__restrict__ col,
                                         const MT *__restrict__ val, const VT *x, int sub) {
  constexpr int U = 4;
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
      if (c[u] >= 0) s = fmadd((VT)v[u], __ldcg(x + c[u]), s);
  }
  return s;
}

// f(i, s) for the rows [r0, r1) of this block, s = sum_j A_ij x_j (off-diagonal)
template <int W, typename T, typename F>
__device__ __forceinline__ void tail_rows(const CsrView<T> &A, const T *x, int64_t r0, int64_t r1,
                                          F &&f) {
  const int sub = threadIdx.x % W;
  const int64_t grp = threadIdx.x / W, ngrp = blockDim.x / W;
  for (int64_t wb = r0 + warp_first_group<W>(grp); wb < r1; wb += ngrp) {
    const int64_t i = wb + group_in_warp<W>(grp);
    const bool active = i < r1;
    T s = active ? row_dot_cg<W, T, T>(__ldg(A.ptr + i), __ldg(A.ptr + i + 1), A.col, A.val, x,
                                       sub)
                 : T(0);
    s = row_reduce<W>(s);
    if (active && sub == 0) f(i, s);
  }
}
template <typename T, typename F>
__device__ __forceinline__ void tail_rows_w(const CsrView<T> &A, const T *x, int64_t r0,
                                            int64_t r1, F &&f) {
  if (A.W <= 4)
    tail_rows<4>(A, x, r0, r1, f);
  else
    tail_rows<8>(A, x, r0, r1, f);
}

// Chebyshev step k of a level (cheb_step_kernel's arithmetic) on this block's rows
template <typename T>
__device__ __forceinline__ void tail_cheb_step(const TailLevel<T> &L, const T *zin, T *zout,
                                               int k, int64_t r0, int64_t r1) {
  const double c1 = k > 0 ? L.cf->c1[k] : 0.0, c2 = k > 0 ? L.cf->c2[k] : L.cf->inv_theta;
  const T vc1 = (T)c1, vc2 = (T)c2;
  tail_rows_w(L.A, zin, r0, r1, [&](int64_t i, T s) {
    T zi = __ldcg(zin + i);
    T res = __ldcg(L.r + i) - fmadd((T)L.A.diag[i], zi, s);
    T di = (vc2 * (T)L.A.invdiag[i]) * res;
    if (k > 0) di = fmadd(vc1, __ldcg(L.d + i), di);
    L.d[i] = di;
    zout[i] = zi + di;
  });
}

template <typename T>
__global__ void __launch_bounds__(1024, 1) vcycle_tail_kernel(const __grid_constant__ TailParams<T> P,
                                                              const Scalars *sc) {
  if (sc && sc->done) return;  // uniform: nothing in this launch writes `done`
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int64_t cb = cl.block_rank(), nb = cl.num_blocks();
  auto lo = [&](int64_t n) { return n * cb / nb; };
  auto hi = [&](int64_t n) { return n * (cb + 1) / nb; };
  // Chebyshev from a zero guess over `deg` steps, result in z (cheb_apply's ping-pong)
  auto cheb_zero = [&](const TailLevel<T> &L, int deg) {
    T *bufs[2] = {L.z, L.t};
    const int w0 = (deg - 1) % 2;
    const int64_t r0 = lo(L.A.n), r1 = hi(L.A.n);
    const double inv_theta = L.cf->inv_theta;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      T di = (T)(inv_theta * (double)L.A.invdiag[i] * (double)__ldcg(L.r + i));
      L.d[i] = di;
      bufs[w0][i] = di;
    }
    cl.sync();
    int at = w0;
    for (int k = 1; k < deg; ++k) {
      tail_cheb_step(L, bufs[at], bufs[at ^ 1], k, r0, r1);
      cl.sync();
      at ^= 1;
    }
  };
  const int last = P.nlev - 1;
  // down: pre-smoothing, residual, restriction
  for (int l = 0; l < last; ++l) {
    const TailLevel<T> &L = P.L[l];
    const TailLevel<T> &C = P.L[l + 1];
    cheb_zero(L, L.deg);
    const int64_t r0 = lo(L.A.n), r1 = hi(L.A.n);
    tail_rows_w(L.A, L.z, r0, r1, [&](int64_t i, T s) {
      L.res[i] = __ldcg(L.r + i) - fmadd((T)L.A.diag[i], __ldcg(L.z + i), s);
    });
    cl.sync();
    for (int64_t I = lo(C.A.n) + threadIdx.x; I < hi(C.A.n); I += blockDim.x) {
      T acc = 0;
      for (int64_t m = L.agg_ptr[I]; m < L.agg_ptr[I + 1]; ++m) acc += __ldcg(L.res + L.agg_mem[m]);
      C.r[I] = acc;
    }
    cl.sync();
  }
  // coarsest level
  {
    const TailLevel<T> &L = P.L[last];
    if (P.coarse_smem) {
      if (cb == 0) {
        if (P.coarse_fp32)
          coarse_cheb_body<T, float, T>(L.A, L.r, L.z, L.cf, L.deg, smem_raw);
        else
          coarse_cheb_body<T, T, T>(L.A, L.r, L.z, L.cf, L.deg, smem_raw);
      }
      cl.sync();
    } else {
      cheb_zero(L, L.deg);
    }
  }
  // up: prolongation, post-smoothing from the corrected guess
  for (int l = last - 1; l >= 0; --l) {
    const TailLevel<T> &L = P.L[l];
    const TailLevel<T> &C = P.L[l + 1];
    const int64_t r0 = lo(L.A.n), r1 = hi(L.A.n);
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      int32_t a = L.agg[i];
      if (a >= 0) L.z[i] = __ldcg(L.z + i) + __ldcg(C.z + a);
    }
    cl.sync();
    T *bufs[2] = {L.z, L.t};
    const int w0 = (L.deg - 1) % 2;
    if (w0 == 0) {  // the guess is read from bufs[1]
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) L.t[i] = __ldcg(L.z + i);
      cl.sync();
    }
    tail_cheb_step(L, bufs[w0 ^ 1], bufs[w0], 0, r0, r1);
    cl.sync();
    int at = w0;
    for (int k = 1; k < L.deg; ++k) {
      tail_cheb_step(L, bufs[at], bufs[at ^ 1], k, r0, r1);
      cl.sync();
      at ^= 1;
    }
  }
}

// ---------------------------------------------------------------------------
// host: structure
// ---------------------------------------------------------------------------
CsrView<double> fine_view(const sph_rt *s);


// bucket sort of ids by bucket[i] into (start, out); nb buckets
template <typename S>
static sph_rt_status bucket_sort(sph_rt *s, SphLevel *owner, int64_t nitems,
                                 const int32_t *bucket, int64_t nb, int64_t **start_out,
                                 S **out_out, int64_t *total_out) {
  unsigned *cnt = scratch<unsigned>(s, nb + 1), *cur = scratch<unsigned>(s, nb + 1);
  int64_t *cnt64 = scratch<int64_t>(s, nb + 1);
  if (!cnt || !cur || !cnt64) return SPH_RT_ENOMEM;
  int64_t *start = lalloc<int64_t>(s, owner, nb + 1);
  if (!start) return SPH_RT_ENOMEM;
  SPH_CUDA(s, cudaMemsetAsync(cnt, 0, sizeof(unsigned) * (nb + 1), s->stream));
  SPH_CUDA(s, cudaMemsetAsync(cur, 0, sizeof(unsigned) * (nb + 1), s->stream));
  target_count_kernel<<<gcap(s, nitems, kBlock), kBlock, 0, s->stream>>>(nitems, bucket, cnt);
  SPH_LAUNCHED(s);
  u32_to_i64_kernel<<<gcap(s, nb, kBlock), kBlock, 0, s->stream>>>(nb, cnt, cnt64);
  SPH_LAUNCHED(s);
  sph_rt_status rc = exclusive_scan(s, cnt64, nb, start);
  if (rc) return rc;
  int64_t total = 0;
  SPH_CUDA(s, cudaMemcpyAsync(&total, start + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s->stream));
  SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  S *out = lalloc<S>(s, owner, total);
  if (!out) return SPH_RT_ENOMEM;
  bucket_scatter_kernel<S><<<gcap(s, nitems, kBlock), kBlock, 0, s->stream>>>(nitems, bucket,
                                                                             start, cur, out);
  SPH_LAUNCHED(s);
  bucket_sort_kernel<S><<<gcap(s, nb, kBlock), kBlock, 0, s->stream>>>(nb, start, out);
  SPH_LAUNCHED(s);
  bucket_rank_kernel<S><<<gcap(s, ceil_div(nb, 32), kWarpsPerBlock), kBlock, 0, s->stream>>>(
      nb, start, out);
  SPH_LAUNCHED(s);
  SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  dfree(s, cnt);
  dfree(s, cur);
  dfree(s, cnt64);
  *start_out = start;
  *out_out = out;
  if (total_out) *total_out = total;
  return SPH_RT_OK;
}

// Galerkin source lists over nitems = nnz + n sources: 64-bit indices when
// they do not fit 32 bits (or config.index64), else 32-bit.
static sph_rt_status source_sort(sph_rt *s, SphLevel *owner, int64_t nitems,
                                 const int32_t *bucket, int64_t nb, int64_t **start_out,
                                 SrcList *out) {
  *out = SrcList{};
  if (s->cfg.index64 || nitems >= ((int64_t)1 << 31) - 1)
    return bucket_sort<int64_t>(s, owner, nitems, bucket, nb, start_out, &out->i64, nullptr);
  return bucket_sort<int32_t>(s, owner, nitems, bucket, nb, start_out, &out->i32, nullptr);
}

template <typename T>
static sph_rt_status launch_galerkin(sph_rt *s, int64_t nnz_c, int64_t nc, const int64_t *seg_ptr,
                            const SrcList &src, int64_t nnz_f, const T *val_f, const T *diag_f,
                            T *val_c, T *diag_c, T *invdiag_c) {
  const int g = gcap(s, nnz_c + nc, kBlock);
  if (src.i64)
    galerkin_kernel<T, int64_t><<<g, kBlock, 0, s->stream>>>(nnz_c, nc, seg_ptr, src.i64, nnz_f,
                                                             val_f, diag_f, val_c, diag_c,
                                                             invdiag_c);
  else
    galerkin_kernel<T, int32_t><<<g, kBlock, 0, s->stream>>>(nnz_c, nc, seg_ptr, src.i32, nnz_f,
                                                             val_f, diag_f, val_c, diag_c,
                                                             invdiag_c);
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

// Aggregate level L and build the next level's sparsity plus the Galerkin
// contribution lists.  Returns the new level in *next (nullptr: stop).
static sph_rt_status coarsen(sph_rt *s, SphLevel *L, SphLevel **next) {
  *next = nullptr;
  const int64_t n = L->n, nnz = L->nnz;
  cudaStream_t st = s->stream;
  uint8_t *strong = scratch<uint8_t>(s, nnz), *cand = scratch<uint8_t>(s, n);
  int *state = scratch<int>(s, n);
  int64_t *flag = scratch<int64_t>(s, n), *root_id = scratch<int64_t>(s, n + 1);
  unsigned *undec = scratch<unsigned>(s, 1), *members = nullptr;
  if (!strong || !cand || !state || !flag || !root_id || !undec) return SPH_RT_ENOMEM;
  auto cleanup = [&]() {
    cudaStreamSynchronize(s->stream);
    dfree(s, strong);
    dfree(s, cand);
    dfree(s, state);
    dfree(s, flag);
    dfree(s, root_id);
    dfree(s, undec);
    if (members) dfree(s, members);
  };
  const int g = gcap(s, n, kBlock);
  const int gw = gcap(s, n, kWarpsPerBlock);  // a warp per row
  strength_kernel<<<gw, kBlock, 0, st>>>(n, L->ptr, L->col, L->val, L->diag,
                                        s->cfg.amg_theta * s->cfg.amg_theta,
                                        strong, state);
  SPH_LAUNCHED(s);
  for (int round = 0; round < 200; ++round) {
    mis_select_kernel<<<gw, kBlock, 0, st>>>(n, L->ptr, L->col, strong, state, cand);
    SPH_LAUNCHED(s);
    mis_apply_kernel<<<g, kBlock, 0, st>>>(n, cand, state);
    SPH_LAUNCHED(s);
    SPH_CUDA(s, cudaMemsetAsync(undec, 0, sizeof(unsigned), st));
    mis_mark_kernel<<<gw, kBlock, 0, st>>>(n, L->ptr, L->col, strong, state, undec);
    SPH_LAUNCHED(s);
    unsigned left = 0;
    SPH_CUDA(s, cudaMemcpyAsync(&left, undec, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    SPH_CUDA(s, cudaStreamSynchronize(st));
    if (left == 0) break;
  }
  root_flag_kernel<<<g, kBlock, 0, st>>>(n, state, flag);
  SPH_LAUNCHED(s);
  sph_rt_status rc = exclusive_scan(s, flag, n, root_id);
  if (rc) return cleanup(), rc;
  int64_t nc = 0;
  SPH_CUDA(s, cudaMemcpyAsync(&nc, root_id + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SPH_CUDA(s, cudaStreamSynchronize(st));
  if (nc == 0 || nc * 10 > n * 9) {  // nothing to coarsen, or coarsening too slow
    cleanup();
    return SPH_RT_OK;
  }
  members = scratch<unsigned>(s, nc);
  if (!members) return cleanup(), SPH_RT_ENOMEM;
  SPH_CUDA(s, cudaMemsetAsync(members, 0, sizeof(unsigned) * nc, st));
  L->agg = lalloc<int32_t>(s, L, n);
  if (!L->agg) return cleanup(), SPH_RT_ENOMEM;
  assign_kernel<<<gw, kBlock, 0, st>>>(n, L->ptr, L->col, L->val, strong, state, root_id, L->agg,
                                      members);
  SPH_LAUNCHED(s);
  cleanup();
  members = nullptr;
  // member lists of the coarse rows
  int64_t tot = 0;
  if ((rc = bucket_sort<int32_t>(s, L, n, L->agg, nc, &L->agg_ptr, &L->agg_mem, &tot))) return rc;

  SphLevel *C = new SphLevel();
  C->n = nc;
  // coarse sparsity: count, scan, fill (+ Galerkin targets of every fine entry)
  int64_t *ccount = lalloc<int64_t>(s, C, nc);
  C->ptr = lalloc<int64_t>(s, C, nc + 1);
  int *overflow = scratch<int>(s, 1);
  if (!ccount || !C->ptr || !overflow) return SPH_RT_ENOMEM;
  SPH_CUDA(s, cudaMemsetAsync(overflow, 0, sizeof(int), st));
  int gb = (int)std::min<int64_t>(nc, (int64_t)s->num_sms * 16);
  coarse_struct_kernel<false><<<gb, kBlock, 0, st>>>(nc, L->agg_ptr, L->agg_mem, L->ptr, L->col,
                                                     L->agg, ccount, nullptr, nullptr, nullptr, 0,
                                                     nullptr, overflow);
  SPH_LAUNCHED(s);
  int ovf = 0;
  SPH_CUDA(s, cudaMemcpyAsync(&ovf, overflow, sizeof(int), cudaMemcpyDeviceToHost, st));
  SPH_CUDA(s, cudaStreamSynchronize(st));
  if (ovf) {
    dfree(s, overflow);
    for (void *p : C->owned) dfree(s, p);
    delete C;
    return SPH_RT_OK;  // stop coarsening here
  }
  if ((rc = exclusive_scan(s, ccount, nc, C->ptr))) return rc;
  SPH_CUDA(s, cudaMemcpyAsync(&C->nnz, C->ptr + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SPH_CUDA(s, cudaStreamSynchronize(st));
  C->col = lalloc<int32_t>(s, C, C->nnz);
  int32_t *tgt = scratch<int32_t>(s, nnz + n);  // off-diagonal entries, then diagonals
  if (!C->col || !tgt) return SPH_RT_ENOMEM;
  fill_i32_kernel<<<gcap(s, nnz + n, kBlock), kBlock, 0, st>>>(nnz + n, -1, tgt);
  SPH_LAUNCHED(s);
  coarse_struct_kernel<true><<<gb, kBlock, 0, st>>>(nc, L->agg_ptr, L->agg_mem, L->ptr, L->col,
                                                    L->agg, nullptr, C->ptr, C->col, tgt, C->nnz,
                                                    tgt + nnz, overflow);
  SPH_LAUNCHED(s);
  // Galerkin contribution lists per coarse target (nnz_c off-diagonal + nc diagonal)
  rc = source_sort(s, L, nnz + n, tgt, C->nnz + nc, &L->seg_ptr, &L->seg_src);
  SPH_CUDA(s, cudaStreamSynchronize(st));
  dfree(s, tgt);
  dfree(s, overflow);
  if (rc) return rc;
  // coarse values and vectors
  C->val = lalloc<double>(s, C, C->nnz);
  C->diag = lalloc<double>(s, C, nc);
  C->invdiag = lalloc<double>(s, C, nc);
  C->r = lalloc<double>(s, C, nc);
  C->z = lalloc<double>(s, C, nc);
  C->res = lalloc<double>(s, C, nc);
  C->d = lalloc<double>(s, C, nc);
  C->t = lalloc<double>(s, C, nc);
  if (!C->val || !C->diag || !C->invdiag || !C->r || !C->z || !C->res || !C->d || !C->t)
    return SPH_RT_ENOMEM;
  {
    RowShape sh = shape_for_mean(nc ? (double)C->nnz / (double)nc : 0.0);
    C->W = sh.W;
    C->U = sh.U;
  }
  *next = C;
  return SPH_RT_OK;
}

static sph_rt_status level_vectors_fine(sph_rt *s, SphLevel *L) {
  L->res = lalloc<double>(s, L, L->n);
  L->d = lalloc<double>(s, L, L->n);
  L->t = lalloc<double>(s, L, L->n);
  if (!L->res || !L->d || !L->t) return SPH_RT_ENOMEM;
  (void)s;
  return SPH_RT_OK;
}

// structure of A P on the finest level (see ap_structure_kernel)
static sph_rt_status build_ap(sph_rt *s, size_t l) {
  SphLevel *L = s->levels[l];
  const int64_t n = L->n;
  int32_t *tmp = scratch<int32_t>(s, (size_t)(L->nnz + n));
  int64_t *cnt = scratch<int64_t>(s, (size_t)n + 1);
  // target A P entry of each source: off-diagonal entries, then the diagonals
  int32_t *map = scratch<int32_t>(s, (size_t)(L->nnz + n));
  L->ap_ptr = lalloc<int64_t>(s, L, n + 1);
  if (!tmp || !cnt || !map || !L->ap_ptr) return SPH_RT_ENOMEM;
  int32_t *dmap = map + L->nnz;
  int *ovf = scratch<int>(s, 1);
  if (!ovf) return SPH_RT_ENOMEM;
  SPH_CUDA(s, cudaMemsetAsync(ovf, 0, sizeof(int), s->stream));
  ap_structure_warp_kernel<<<gcap(s, n, kWarpsPerBlock), kBlock, 0, s->stream>>>(
      n, L->ptr, L->col, L->agg, tmp, cnt, map, dmap, ovf);
  SPH_LAUNCHED(s);
  int h_ovf = 0;
  SPH_CUDA(s, cudaMemcpyAsync(&h_ovf, ovf, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  dfree(s, ovf);
  if (h_ovf) {  // a row with more distinct aggregates than the warp keeps: one thread a row
    ap_structure_kernel<<<gcap(s, n, kBlock), kBlock, 0, s->stream>>>(n, L->ptr, L->col, L->agg,
                                                                      tmp, cnt, map, dmap);
    SPH_LAUNCHED(s);
  }
  sph_rt_status rc = exclusive_scan(s, cnt, n, L->ap_ptr);
  if (rc) return rc;
  int64_t total = 0;
  SPH_CUDA(s, cudaMemcpyAsync(&total, L->ap_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost,
                              s->stream));
  SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  if (total >= ((int64_t)1 << 31)) return set_error(s, SPH_RT_EINVAL, "A P too large");
  L->nnz_ap = total;
  L->ap_col = lalloc<int32_t>(s, L, (size_t)total);
  L->ap_val = lalloc<double>(s, L, (size_t)total);
  if (!L->ap_col || !L->ap_val) return SPH_RT_ENOMEM;
  if (s->cfg.precision == SPH_RT_MIXED && !(L->ap_val32 = lalloc<float>(s, L, (size_t)total)))
    return SPH_RT_ENOMEM;
  ap_compact_kernel<<<gcap(s, n, kBlock), kBlock, 0, s->stream>>>(n, L->ptr, tmp, L->ap_ptr,
                                                                  L->ap_col, map, dmap);
  SPH_LAUNCHED(s);
  // sources of each A P entry in increasing source order
  if ((rc = source_sort(s, L, L->nnz + n, map, total, &L->ap_seg_ptr, &L->ap_seg_src)))
    return rc;
  // next level's Galerkin sources: the A P entries of its members' rows
  SphLevel *C = s->levels[l + 1];
  int32_t *tgt = scratch<int32_t>(s, (size_t)total);
  int *missing = scratch<int>(s, 1);
  if (!tgt || !missing) return SPH_RT_ENOMEM;
  SPH_CUDA(s, cudaMemsetAsync(missing, 0, sizeof(int), s->stream));
  ap_galerkin_target_kernel<<<gcap(s, n, kBlock), kBlock, 0, s->stream>>>(
      n, L->ap_ptr, L->ap_col, L->agg, C->nnz, C->ptr, C->col, tgt, missing);
  SPH_LAUNCHED(s);
  if ((rc = bucket_sort<int32_t>(s, L, total, tgt, C->nnz + C->n, &L->apg_ptr, &L->apg_src,
                                 nullptr)))
    return rc;
  int miss = 0;
  SPH_CUDA(s, cudaMemcpyAsync(&miss, missing, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  dfree(s, tgt);
  dfree(s, missing);
  if (miss) return set_error(s, SPH_RT_EDEVICE, "A P entry outside the coarse sparsity");
  SPH_CUDA(s, cudaStreamSynchronize(s->stream));
  dfree(s, tmp);
  dfree(s, cnt);
  dfree(s, map);
  return SPH_RT_OK;
}

static sph_rt_status build_structure(sph_rt *s) {
  amg_release(s);
  SphLevel *L0 = new SphLevel();
  CsrView<double> A = fine_view(s);
  L0->n = A.n;
  L0->nnz = A.nnz;
  L0->ptr = const_cast<int64_t *>(A.ptr);
  L0->col = const_cast<int32_t *>(A.col);
  L0->val = const_cast<double *>(A.val);
  L0->diag = const_cast<double *>(A.diag);
  L0->invdiag = const_cast<double *>(A.invdiag);
  L0->W = A.W;
  L0->U = A.U;
  s->levels.push_back(L0);
  sph_rt_status rc = level_vectors_fine(s, L0);
  if (rc) return rc;
  SphLevel *L = L0;
  while ((int)s->levels.size() < kMaxLevels && L->n > kCoarseTarget) {
    // the strength test needs this level's values
    if (L != L0) {
      // values are produced by the numeric pass below; build them now
    }
    SphLevel *C = nullptr;
    if ((rc = coarsen(s, L, &C))) return rc;
    if (!C) break;
    s->levels.push_back(C);
    // numeric Galerkin product for C so that the next strength test can run
    if ((rc = launch_galerkin<double>(s, C->nnz, C->n, L->seg_ptr, L->seg_src, L->nnz, L->val,
                                      L->diag, C->val, C->diag, C->invdiag)))
      return rc;
    L = C;
  }
  s->amg_ready = true;
  return SPH_RT_OK;
}

// numeric set-up of every level from the current fine operator
// Bytes per value the coarsest-level solve is staged and computed in: FP32
// when config.coarse_fp32 (also in the FP64 form), else the level's type.
template <typename T>
static size_t coarse_solve_bytes(const sph_rt *s) {
  return s->cfg.coarse_fp32 ? sizeof(float) : sizeof(T);
}

// Chebyshev degree of the coarsest-level solve.  Each step is a dependent pass
// through one SM (~2 us for a few hundred rows); 6 steps gave the same Krylov
// counts as 12 on the 64^3 and 128^3 manufactured problems.
static int coarse_degree(const sph_rt *s, const SphLevel *L) {
  return L->n <= kCoarseTarget * 4 ? 6 : 3 * s->cfg.cheb_degree;
}

template <typename T>
struct LevelVecs;
template <>
struct LevelVecs<double> {
  static CsrView<double> view(SphLevel *L) {
    CsrView<double> A;
    A.n = L->n;
    A.ptr = L->ptr;
    A.col = L->col;
    A.val = L->val;
    A.diag = L->diag;
    A.invdiag = L->invdiag;
    A.nnz = L->nnz;
    A.W = L->W;
    A.U = L->U;
    return A;
  }
  static double *r(SphLevel *L) { return L->r; }
  static double *z(SphLevel *L) { return L->z; }
  static double *res(SphLevel *L) { return L->res; }
  static double *d(SphLevel *L) { return L->d; }
  static double *t(SphLevel *L) { return L->t; }
  static const double *ap(SphLevel *L) { return L->ap_val; }
};
template <>
struct LevelVecs<float> {
  static CsrView<float> view(SphLevel *L) {
    CsrView<float> A;
    A.n = L->n;
    A.ptr = L->ptr;
    A.col = L->col;
    A.val = L->val32;
    A.diag = L->diag32;
    A.invdiag = L->invdiag32;
    A.nnz = L->nnz;
    A.W = L->W;
    A.U = L->U;
    return A;
  }
  static float *r(SphLevel *L) { return L->r32; }
  static float *z(SphLevel *L) { return L->z32; }
  static float *res(SphLevel *L) { return L->res32; }
  static float *d(SphLevel *L) { return L->d32; }
  static float *t(SphLevel *L) { return L->t32; }
  static const float *ap(SphLevel *L) { return L->ap_val32; }
};


// FP32 storage of every level of the mixed form (level 0 borrows the FP32
// copy the assembly writes).
static sph_rt_status level_fp32(sph_rt *s, size_t l) {
  SphLevel *L = s->levels[l];
  if (L->r32) return SPH_RT_OK;
  if (l == 0) {
    L->val32 = s->mat_val32;
    L->diag32 = s->diag32;
    L->invdiag32 = s->invdiag32;
  } else {
    L->val32 = lalloc<float>(s, L, L->nnz);
    L->diag32 = lalloc<float>(s, L, L->n);
    L->invdiag32 = lalloc<float>(s, L, L->n);
  }
  L->r32 = lalloc<float>(s, L, L->n);
  L->z32 = lalloc<float>(s, L, L->n);
  L->res32 = lalloc<float>(s, L, L->n);
  L->d32 = lalloc<float>(s, L, L->n);
  L->t32 = lalloc<float>(s, L, L->n);
  if (!L->val32 || !L->diag32 || !L->invdiag32 || !L->r32 || !L->z32 || !L->res32 || !L->d32 ||
      !L->t32)
    return SPH_RT_ENOMEM;
  return SPH_RT_OK;
}

// Galerkin values of every level from the current fine operator, in the
// hierarchy's type T: FP64, or FP32 in the mixed form, where the sums are
// formed from the FP32 fine copy directly.
template <typename T>
static sph_rt_status galerkin_levels(sph_rt *s) {
  using LV = LevelVecs<T>;
  for (size_t l = 0; l + 1 < s->levels.size(); ++l) {
    SphLevel *L = s->levels[l], *C = s->levels[l + 1];
    const CsrView<T> Lv = LV::view(L), Cv = LV::view(C);
    if (L->ap_ptr) {  // A P of this level (its values are final: level l is done)
      sph_rt_status rc = launch_galerkin<T>(s, L->nnz_ap, 0, L->ap_seg_ptr, L->ap_seg_src,
                                            L->nnz, Lv.val, Lv.diag, const_cast<T *>(LV::ap(L)),
                                            nullptr, nullptr);
      if (rc) return rc;
    }
    T *cval = const_cast<T *>(Cv.val), *cdiag = const_cast<T *>(Cv.diag),
      *cinv = const_cast<T *>(Cv.invdiag);
    // P^T (A P): its sources are A P entries (fewer than 2^31)
    sph_rt_status rc =
        L->apg_ptr ? launch_galerkin<T>(s, C->nnz, C->n, L->apg_ptr, SrcList{L->apg_src, nullptr},
                                        L->nnz_ap, LV::ap(L), nullptr, cval, cdiag, cinv)
                   : launch_galerkin<T>(s, C->nnz, C->n, L->seg_ptr, L->seg_src, L->nnz, Lv.val,
                                        Lv.diag, cval, cdiag, cinv);
    if (rc) return rc;
  }
  // Gershgorin bounds of every level, turned into Chebyshev coefficients on
  // the device (slot 1 + l): no host read
  if (!s->amg_gersh) s->amg_gersh = dalloc<double>(s, kMaxLevels);
  double *dg = s->amg_gersh;
  if (!dg) return SPH_RT_ENOMEM;
  for (size_t l = 0; l < s->levels.size(); ++l) {
    SphLevel *L = s->levels[l];
    if (l == 0) {
      // the finest level's bound was reduced by the assembly of this step
      SPH_CUDA(s, cudaMemcpyAsync(dg, s->gersh, sizeof(double), cudaMemcpyDeviceToDevice,
                                  s->stream));
      continue;
    }
    const CsrView<T> Lv = LV::view(L);
    gersh_kernel<T><<<gcap(s, L->n, kBlock), kBlock, 0, s->stream>>>(
        L->n, L->ptr, Lv.val, Lv.diag, s->partials, &s->sc->counter, dg + l);
    SPH_LAUNCHED(s);
  }
  return SPH_RT_OK;
}

bool fcg_active(const sph_rt *s);
sph_rt_status fcg_vectors(sph_rt *s, FcgVecs *v);

static sph_rt_status numeric(sph_rt *s) {
  sph_rt_status rc;
  const bool mixed = s->cfg.precision == SPH_RT_MIXED;
  if (mixed) {
    for (size_t l = 0; l < s->levels.size(); ++l)
      if ((rc = level_fp32(s, l))) return rc;
    SphLevel *L0 = s->levels[0];
    if (L0->ap_ptr && !L0->ap_val32 && !(L0->ap_val32 = lalloc<float>(s, L0, L0->nnz_ap)))
      return SPH_RT_ENOMEM;
    if ((rc = galerkin_levels<float>(s))) return rc;
  } else {
    if ((rc = galerkin_levels<double>(s))) return rc;
  }
  std::vector<int> mode(s->levels.size()), degree(s->levels.size());
  for (size_t l = 0; l < s->levels.size(); ++l) {
    const bool coarsest = l + 1 == s->levels.size();
    mode[l] = coarsest ? 2 : 1;
    degree[l] = coarsest ? coarse_degree(s, s->levels[l]) : s->cfg.cheb_degree;
  }
  if ((rc = launch_cheb_slots(s, 1, s->amg_gersh, mode, degree))) return rc;
  // FP32 CG vectors of the V-cycle-product CG, allocated here (not while a
  // loop graph is being captured)
  if (mixed && fcg_active(s)) {
    FcgVecs v;
    if ((rc = fcg_vectors(s, &v))) return rc;
  }
  return SPH_RT_OK;
}

template <typename T>
static void tail_setup(sph_rt *s);

sph_rt_status amg_setup(sph_rt *s) {
  sph_rt_status rc;
  if (!s->amg_ready || s->cfg.amg_rebuild) {
    if ((rc = build_structure(s))) return rc;
    if (s->cfg.precision == SPH_RT_MIXED)
      tail_setup<float>(s);
    else
      tail_setup<double>(s);
    // A P of the levels larger than the tail threshold: the smaller ones
    // post-smooth the same way with or without the cluster tail, so both give
    // bitwise the same V-cycle
    for (size_t l = 0; l + 1 < s->levels.size() && s->levels[l]->nnz > kTailMaxNnz; ++l)
      if ((rc = build_ap(s, l))) return rc;
  }
  return numeric(s);
}

// ---------------------------------------------------------------------------
// V-cycle
// ---------------------------------------------------------------------------
template <typename T>
static sph_rt_status launch_tail(sph_rt *s, size_t l0, const T *r, T *z, const Scalars *sc) {
  using LV = LevelVecs<T>;
  TailParams<T> P;
  memset(&P, 0, sizeof P);
  P.nlev = (int)(s->levels.size() - l0);
  for (int m = 0; m < P.nlev; ++m) {
    SphLevel *L = s->levels[l0 + m];
    TailLevel<T> &t = P.L[m];
    t.A = LV::view(L);
    t.agg = L->agg;
    t.agg_ptr = L->agg_ptr;
    t.agg_mem = L->agg_mem;
    t.r = m == 0 ? const_cast<T *>(r) : LV::r(L);
    t.z = m == 0 ? z : LV::z(L);
    t.res = LV::res(L);
    t.d = LV::d(L);
    t.t = LV::t(L);
    t.cf = s->cheb_slots + 1 + l0 + m;
    t.deg = m + 1 == P.nlev ? coarse_degree(s, L) : s->cfg.cheb_degree;
  }
  SphLevel *Lc = s->levels.back();
  const size_t cs = coarse_solve_bytes<T>(s);
  const size_t smem = coarse_smem_bytes(Lc->n, Lc->nnz, cs, cs);
  P.coarse_smem = 1;  // tail_setup only enables the tail when the coarsest level fits
  P.coarse_fp32 = cs == sizeof(float) && sizeof(T) == sizeof(double);
  cudaLaunchConfig_t lc;
  memset(&lc, 0, sizeof lc);
  lc.gridDim = dim3((unsigned)s->tail_cluster);
  lc.blockDim = dim3(1024);
  lc.dynamicSmemBytes = smem;
  lc.stream = s->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)s->tail_cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  SPH_CUDA(s, cudaLaunchKernelEx(&lc, vcycle_tail_kernel<T>, P, sc));
  SPH_LAUNCHED(s);
  return SPH_RT_OK;
}

// Decide where the cluster tail starts (0 = no tail) and its cluster size:
// 16 blocks where the device can co-schedule them, else 8.
template <typename T>
static void tail_setup(sph_rt *s) {
  s->tail_level = 0;
  s->tail_cluster = 0;
  const int nl = (int)s->levels.size();
  if (nl < 3 || !s->cfg.amg_tail) return;
  int l0 = nl;
  while (l0 > 1 && s->levels[l0 - 1]->nnz <= kTailMaxNnz) --l0;
  if (nl - l0 < 2) return;
  SphLevel *Lc = s->levels.back();
  const size_t cs = coarse_solve_bytes<T>(s);
  const size_t smem = coarse_smem_bytes(Lc->n, Lc->nnz, cs, cs);
  if (smem > kCoarseSmemMax) return;
  auto kern = vcycle_tail_kernel<T>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kCoarseSmemMax) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaGetLastError();
  for (int cl : {16, 8}) {
    cudaLaunchConfig_t lc;
    memset(&lc, 0, sizeof lc);
    lc.gridDim = dim3((unsigned)cl);
    lc.blockDim = dim3(1024);
    lc.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &lc) == cudaSuccess && clusters >= 1) {
      s->tail_level = l0;
      s->tail_cluster = cl;
      return;
    }
    cudaGetLastError();
  }
}

template <typename T>
static sph_rt_status vcycle(sph_rt *s, size_t l, const T *r, T *z, const Scalars *sc,
                            bool init_done = false, const DotFuse *df = nullptr,
                            bool *dot_done = nullptr) {
  using LV = LevelVecs<T>;
  if (s->tail_level > 0 && l == (size_t)s->tail_level) return launch_tail<T>(s, l, r, z, sc);
  SphLevel *L = s->levels[l];
  CsrView<T> A = LV::view(L);
  const int deg = s->cfg.cheb_degree;
  sph_rt_status rc;
  if (l + 1 == s->levels.size()) {
    // coarsest level: Chebyshev solve over the whole Gershgorin interval
    const int cdeg = coarse_degree(s, L);
    const ChebCoef *cf = s->cheb_slots + 1 + l;
    const size_t cs = coarse_solve_bytes<T>(s);
    const size_t smem = coarse_smem_bytes(L->n, L->nnz, cs, cs);
    if (l > 0 && smem <= kCoarseSmemMax) {
      // opt in to more than 48 KiB of dynamic shared memory (once per handle and variant)
      const bool f32 = cs == sizeof(float) && sizeof(T) == sizeof(double);
      const int bit = f32 ? 4 : (sizeof(T) == 8 ? 1 : 2);
      if (!(s->coarse_smem_optin & bit)) {
        if (f32)
          SPH_CUDA(s, cudaFuncSetAttribute(coarse_cheb_kernel<T, float, T>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kCoarseSmemMax));
        else
          SPH_CUDA(s, cudaFuncSetAttribute(coarse_cheb_kernel<T, T, T>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kCoarseSmemMax));
        s->coarse_smem_optin |= bit;
      }
      if (f32)
        pdl_launch(s, coarse_cheb_kernel<T, float, T>, 1, 1024, smem, A, r, z, cf, cdeg, sc);
      else
        pdl_launch(s, coarse_cheb_kernel<T, T, T>, 1, 1024, smem, A, r, z, cf, cdeg, sc);
      SPH_LAUNCHED(s);
      return SPH_RT_OK;
    }
    return cheb_apply<T, T>(s, A, r, z, LV::d(L), LV::t(L), cdeg, cf, true, sc);
  }
  const ChebCoef *cf = s->cheb_slots + 1 + l;
  // zero-guess pre-smoothing (its first write was made by the restriction above
  // when init_done)
  if ((rc = cheb_apply<T, T>(s, A, r, z, LV::d(L), LV::t(L), deg, cf, true, sc, init_done)))
    return rc;
  const int gw = l == 0 ? row_grid(s->num_sms, L->n, A.W, A.U)
                        : row_grid_blocks(s->num_sms, L->n, A.W, kCoarseMinBlocks);
  T *res = LV::res(L);
  // fine-level residual sweeps are timed with the other fine SpMV-class kernels;
  // per row: rowptr, diag, r, z, res
  int *wf = l == 0 ? timing_begin(s) : nullptr;
  if (l == 0)
    SPH_DISPATCH_SHAPE(A.W, A.U,
                       (pdl_launch(s, fine_resid_level_kernel<W, U, T, T>, gw, kBlock, 0,
                           A, r, z, res, sc, wf)));
  else
    SPH_DISPATCH_SHAPE(A.W, A.U,
                       (pdl_launch(s, resid_level_kernel<W, U, T, T>, gw, kBlock, 0, A, r, z, res,
                                                                                      sc, wf)));
  SPH_LAUNCHED(s);
  if (l == 0)
    timing_end(s, (4.0 + sizeof(T)) * (double)A.nnz + (8.0 + 4.0 * sizeof(T)) * (double)A.n,
               kTimedResid);
  SphLevel *C = s->levels[l + 1];
  // a launched, non-coarsest next level takes its smoother start from the restriction
  const bool fuse = l + 2 < s->levels.size() &&
                    !(s->tail_level > 0 && l + 1 == (size_t)s->tail_level);
  if (fuse) {
    const int wc = (deg - 1) % 2;  // cheb_apply's first write goes to bufs[wc]
    T *zc_first = wc == 0 ? LV::z(C) : LV::t(C);
    pdl_launch(s, restrict_init_kernel<T, T>, gcap(s, C->n, kBlock), kBlock, 0,
        C->n, L->agg_ptr, L->agg_mem, res, LV::r(C), LV::view(C).invdiag,
        s->cheb_slots + 1 + (l + 1), LV::d(C), zc_first, sc);
  } else {
    pdl_launch(s, restrict_kernel<T>, gcap(s, C->n, kBlock), kBlock, 0,
        C->n, L->agg_ptr, L->agg_mem, res, LV::r(C), sc);
  }
  SPH_LAUNCHED(s);
  if ((rc = vcycle<T>(s, l + 1, LV::r(C), LV::z(C), sc, fuse))) return rc;
  if (L->ap_ptr && LV::ap(L)) {
    // prolongation and the first post-smoothing step in one sweep of A P
    T *bufs[2] = {z, LV::t(L)};
    const int w0 = (deg - 1) % 2;
    const RowShape sh = shape_for_mean(L->n ? (double)L->nnz_ap / (double)L->n : 0.0);
    const int gp = l == 0 ? row_grid(s->num_sms, L->n, sh.W, sh.U)
                          : row_grid_blocks(s->num_sms, L->n, sh.W, kCoarseMinBlocks);
    int *wf = l == 0 ? timing_begin(s) : nullptr;
    // with degree 1 this sweep is the V-cycle's last: the inner product rides along
    const bool dot = l == 0 && df && dot_done && deg == 1;
    if (dot) {
      SPH_DISPATCH_SHAPE(sh.W, sh.U,
                         (pdl_launch(s, fine_post_ap_dot_kernel<W, U, T, T>, gp, kBlock, 0,
                             L->n, L->ap_ptr, L->ap_col, LV::ap(L), L->agg, LV::z(C), z, res,
                             A.invdiag, cf, LV::d(L), bufs[w0], sc, wf, *df)));
      *dot_done = true;
    } else if (l == 0)
      SPH_DISPATCH_SHAPE(sh.W, sh.U,
                         (pdl_launch(s, fine_post_ap_kernel<W, U, T, T>, gp, kBlock, 0,
                             L->n, L->ap_ptr, L->ap_col, LV::ap(L), L->agg, LV::z(C), z, res,
                             A.invdiag, cf, LV::d(L), bufs[w0], sc, wf)));
    else
      SPH_DISPATCH_SHAPE(sh.W, sh.U,
                         (pdl_launch(s, post_ap_kernel<W, U, T, T>, gp, kBlock, 0,
                             L->n, L->ap_ptr, L->ap_col, LV::ap(L), L->agg, LV::z(C), z, res,
                             A.invdiag, cf, LV::d(L), bufs[w0], sc, nullptr)));
    SPH_LAUNCHED(s);
    // A P entry: column + value; per row: ap_ptr, agg, the coarse entry of P e_c,
    // z_pre, res, 1/diag, d, z_out; with the inner product also r (and, flexible,
    // the FP64 z read and written)
    if (l == 0)
      timing_end(s,
                 (4.0 + sizeof(T)) * (double)L->nnz_ap +
                     (12.0 + 6.0 * sizeof(T) + (dot ? (df->flex ? 24.0 : 8.0) : 0.0)) *
                         (double)L->n,
                 kTimedPost);
    return cheb_apply<T, T>(s, A, r, z, LV::d(L), LV::t(L), deg, cf, false, sc, true);
  }
  pdl_launch(s, prolong_kernel<T>, gcap(s, L->n, kBlock), kBlock, 0, L->n, L->agg, LV::z(C), z, sc);
  SPH_LAUNCHED(s);
  return cheb_apply<T, T>(s, A, r, z, LV::d(L), LV::t(L), deg, cf, false, sc);
}

// Mixed form without the last conversion: r is rounded to FP32 and the FP32
// V-cycle leaves z in levels[0]->z32 (amg_z32), for a caller that widens it
// itself (the fused flexible-CG inner product).  init_done: r32 and the finest
// level's smoother start were written by the CG update.
sph_rt_status amg_apply_to32(sph_rt *s, const double *r, const Scalars *sc, bool init_done,
                             const DotFuse *df, bool *dot_done) {
  if (s->levels.empty()) return set_error(s, SPH_RT_ESTATE, "AMG hierarchy not set up");
  SphLevel *L0 = s->levels[0];
  if (!init_done) {
    pdl_launch(s, convert_kernel<double, float>, gcap(s, L0->n, kBlock), kBlock, 0, L0->n, r,
                                                                                    L0->r32);
    SPH_LAUNCHED(s);
  }
  return vcycle<float>(s, 0, L0->r32, L0->z32, sc, init_done, df, dot_done);
}
const float *amg_z32(const sph_rt *s) { return s->levels.empty() ? nullptr : s->levels[0]->z32; }

// The finest level's zero-guess smoother start for the CG update to write
// (FineInit): in FP64 into the preconditioner output z (or the ping-pong
// buffer the start goes to), in FP32 into the level's FP32 vectors together
// with the narrowed residual.  False where the V-cycle takes no such start
// (a single level: the finest level is then the coarsest).
bool amg_fine_init(sph_rt *s, FineInit<double> *f64, FineInit<float> *f32) {
  if (s->levels.size() < 2) return false;
  SphLevel *L0 = s->levels[0];
  const int w0 = (s->cfg.cheb_degree - 1) % 2;  // cheb_apply's first write: bufs[w0]
  const ChebCoef *cf = s->cheb_slots + 1;
  if (s->cfg.precision == SPH_RT_MIXED) {
    *f32 = {L0->r32, L0->invdiag32, cf, L0->d32, w0 == 0 ? L0->z32 : L0->t32};
  } else {
    *f64 = {nullptr, L0->invdiag, cf, L0->d, w0 == 0 ? s->z : L0->t};
  }
  return true;
}

sph_rt_status amg_apply(sph_rt *s, const double *r, double *z, const Scalars *sc, bool init_done,
                        const DotFuse *df, bool *dot_done) {
  if (s->levels.empty()) return set_error(s, SPH_RT_ESTATE, "AMG hierarchy not set up");
  if (s->cfg.precision == SPH_RT_MIXED) {
    SphLevel *L0 = s->levels[0];
    if (!init_done) {
      pdl_launch(s, convert_kernel<double, float>, gcap(s, L0->n, kBlock), kBlock, 0, L0->n, r,
                                                                                      L0->r32);
      SPH_LAUNCHED(s);
    }
    sph_rt_status rc = vcycle<float>(s, 0, L0->r32, L0->z32, sc, init_done);
    if (rc) return rc;
    pdl_launch(s, convert_kernel<float, double>, gcap(s, L0->n, kBlock), kBlock, 0, L0->n, L0->z32, z);
    SPH_LAUNCHED(s);
    return SPH_RT_OK;
  }
  return vcycle<double>(s, 0, r, z, sc, init_done, df, dot_done);
}

// ---------------------------------------------------------------------------
// The V-cycle of the CG with the V-cycle's product (fine_post_smooth = 0), in
// the precision T of the hierarchy: from r and the smoother start z_pre (in
// the finest level's d, written by the CG update or the residual kernel), the
// finest-level residual sweep, the coarse V-cycle (symmetric, as always) and
// the last sweep that forms z, w = B z and the CG scalars (see
// fine_ap_cg_kernel).  The vectors are those of FcgVecs.
// ---------------------------------------------------------------------------
bool fcg_active(const sph_rt *s) {
  return s->cfg.fine_post_smooth == 0 && s->cfg.precond == SPH_RT_PRECOND_AMG &&
         s->levels.size() >= 2;
}

sph_rt_status fcg_vectors(sph_rt *s, FcgVecs *v) {
  SphLevel *L0 = s->levels[0];
  if (s->cfg.precision == SPH_RT_MIXED) {
    if (!L0->p32) {
      L0->p32 = lalloc<float>(s, L0, L0->n);
      L0->q32 = lalloc<float>(s, L0, L0->n);
      L0->w32 = lalloc<float>(s, L0, L0->n);
      if (!L0->p32 || !L0->q32 || !L0->w32) return SPH_RT_ENOMEM;
    }
    v->f32 = {L0->r32, L0->z32, L0->w32, L0->p32, L0->q32, L0->d32, L0->invdiag32};
  } else {
    v->f64 = {s->r, s->z, s->w, s->p, s->q, L0->d, L0->invdiag};
  }
  v->cf = s->cheb_slots + 1;
  return SPH_RT_OK;
}

template <typename T>
static sph_rt_status fcg_cycle_t(sph_rt *s, const FcgSet<T> &v, int first) {
  using LV = LevelVecs<T>;
  SphLevel *L = s->levels[0];
  CsrView<T> A = LV::view(L);
  const Scalars *sc = s->sc;
  T *res = LV::res(L);
  const int gw = row_grid(s->num_sms, L->n, A.W, A.U);
  int *wf = timing_begin(s);
  SPH_DISPATCH_SHAPE(A.W, A.U,
                     (pdl_launch(s, fine_resid_level_kernel<W, U, T, T>, gw, kBlock, 0, A, v.r,
                                 v.zpre, res, sc, wf)));
  SPH_LAUNCHED(s);
  timing_end(s, (4.0 + sizeof(T)) * (double)A.nnz + (8.0 + 4.0 * sizeof(T)) * (double)A.n,
             kTimedResid);
  SphLevel *C = s->levels[1];
  const int deg = s->cfg.cheb_degree;
  const bool fuse = s->levels.size() > 2 && !(s->tail_level > 0 && s->tail_level == 1);
  if (fuse) {
    const int wc = (deg - 1) % 2;
    T *zc_first = wc == 0 ? LV::z(C) : LV::t(C);
    pdl_launch(s, restrict_init_kernel<T, T>, gcap(s, C->n, kBlock), kBlock, 0, C->n, L->agg_ptr,
               L->agg_mem, (const T *)res, LV::r(C), LV::view(C).invdiag, s->cheb_slots + 2,
               LV::d(C), zc_first, sc);
  } else {
    pdl_launch(s, restrict_kernel<T>, gcap(s, C->n, kBlock), kBlock, 0, C->n, L->agg_ptr,
               L->agg_mem, (const T *)res, LV::r(C), sc);
  }
  SPH_LAUNCHED(s);
  sph_rt_status rc = vcycle<T>(s, 1, LV::r(C), LV::z(C), sc, fuse);
  if (rc) return rc;
  if (L->ap_ptr && LV::ap(L)) {
    const RowShape sh = shape_for_mean(L->n ? (double)L->nnz_ap / (double)L->n : 0.0);
    const int gp = row_grid_blocks(s->num_sms, L->n, sh.W, fcg_min_blocks<T>());
    wf = timing_begin(s);
    SPH_DISPATCH_SHAPE(sh.W, sh.U,
                       (pdl_launch(s, fine_ap_cg_kernel<W, U, T, T>, gp, kBlock, 0, L->n,
                                   L->ap_ptr, L->ap_col, LV::ap(L), L->agg, (const T *)LV::z(C),
                                   (const T *)v.zpre, (const T *)res, (const T *)v.r, v.z, v.w,
                                   (const T *)v.p, (const T *)v.q, first, s->sc, s->partials,
                                   wf)));
    SPH_LAUNCHED(s);
    // A P entry: column + value; per row: ap_ptr, agg, P e_c, z_pre, res, r, z r/w, w,
    // p, q
    timing_end(s, (4.0 + sizeof(T)) * (double)L->nnz_ap + (12.0 + 10.0 * sizeof(T)) * (double)L->n,
               kTimedPost);
    return SPH_RT_OK;
  }
  T *t = LV::t(L);
  pdl_launch(s, fcg_prolong_kernel<T>, gcap(s, L->n, kBlock), kBlock, 0, L->n,
             (const int32_t *)L->agg, (const T *)LV::z(C), (const T *)v.zpre, t, sc);
  SPH_LAUNCHED(s);
  wf = timing_begin(s);
  const int gd = row_grid_blocks(s->num_sms, L->n, A.W, fcg_min_blocks<T>());
  SPH_DISPATCH_SHAPE(A.W, A.U,
                     (pdl_launch(s, fcg_spmv_dot_kernel<W, U, T, T>, gd, kBlock, 0, A,
                                 (const T *)t, (const T *)v.r, v.z, v.w, (const T *)v.p,
                                 (const T *)v.q, first, s->sc, s->partials, wf)));
  SPH_LAUNCHED(s);
  timing_end(s, (4.0 + sizeof(T)) * (double)A.nnz + (8.0 + 9.0 * sizeof(T)) * (double)A.n,
             kTimedSpmvPQ);
  return SPH_RT_OK;
}

sph_rt_status fcg_cycle(sph_rt *s, const FcgVecs &v, int first) {
  if (s->cfg.precision == SPH_RT_MIXED) return fcg_cycle_t<float>(s, v.f32, first);
  return fcg_cycle_t<double>(s, v.f64, first);
}

// Launch-relevant layout of the hierarchy (sizes, shapes and every buffer the
// V-cycle touches), appended to the signature of a captured loop graph.
void amg_signature(const sph_rt *s, std::vector<uint64_t> &sig) {
  sig.push_back(s->levels.size());
  sig.push_back((uint64_t)s->tail_level);
  sig.push_back((uint64_t)s->tail_cluster);
  for (const SphLevel *L : s->levels) {
    const uint64_t v[] = {(uint64_t)L->n,
                          (uint64_t)L->nnz,
                          (uint64_t)L->W,
                          (uint64_t)L->U,
                          (uint64_t)(uintptr_t)L->ptr,
                          (uint64_t)(uintptr_t)L->col,
                          (uint64_t)(uintptr_t)L->val,
                          (uint64_t)(uintptr_t)L->diag,
                          (uint64_t)(uintptr_t)L->invdiag,
                          (uint64_t)(uintptr_t)L->val32,
                          (uint64_t)(uintptr_t)L->diag32,
                          (uint64_t)(uintptr_t)L->invdiag32,
                          (uint64_t)(uintptr_t)L->agg,
                          (uint64_t)(uintptr_t)L->agg_ptr,
                          (uint64_t)(uintptr_t)L->agg_mem,
                          (uint64_t)(uintptr_t)L->r,
                          (uint64_t)(uintptr_t)L->z,
                          (uint64_t)(uintptr_t)L->res,
                          (uint64_t)(uintptr_t)L->d,
                          (uint64_t)(uintptr_t)L->t,
                          (uint64_t)(uintptr_t)L->r32,
                          (uint64_t)(uintptr_t)L->z32,
                          (uint64_t)(uintptr_t)L->res32,
                          (uint64_t)(uintptr_t)L->d32,
                          (uint64_t)(uintptr_t)L->t32,
                          (uint64_t)(uintptr_t)L->ap_ptr,
                          (uint64_t)(uintptr_t)L->ap_col,
                          (uint64_t)(uintptr_t)L->ap_val,
                          (uint64_t)(uintptr_t)L->ap_val32};
    sig.insert(sig.end(), v, v + sizeof v / sizeof v[0]);
  }
}

// number of levels and rows/nnz per level (for diagnostics)
int amg_levels(const sph_rt *s, int64_t *rows, int64_t *nnz, int maxl) {
  int k = 0;
  for (SphLevel *L : s->levels) {
    if (k >= maxl) break;
    rows[k] = L->n;
    nnz[k] = L->nnz;
    ++k;
  }
  return k;
}

}  // namespace sphrt
