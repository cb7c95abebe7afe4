// noalloc.cu -- interior energy totals with scratch in static device memory.
//
// For callers that cannot let the library allocate (see sph_rt_noalloc.h):
// the partial sums of the blocks and the arrival counter of the deterministic
// last-block reduction live in a file-scope __device__ array instead of a
// cudaMalloc'ed buffer.  In host code the array's name is only a stand-in for
// the symbol, so its device address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernel.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/sph_rt_noalloc.h"
#include "common.cuh"

namespace sphrt {
void set_thread_error(const std::string &msg);  // message for sph_rt_last_error(NULL)
}

namespace {

constexpr int kNaBlock = 256;
constexpr int kNaItems = 32;                            // particles per thread
constexpr int64_t kNaPerBlock = (int64_t)kNaBlock * kNaItems;  // 8192
constexpr int kNaMaxBlocks = 4096;
static_assert(kNaPerBlock * kNaMaxBlocks == SPH_RT_NOALLOC_MAX_N, "size bound");

// Two partial sums per block, then the arrival counter (64 KiB + 256 B).  Like
// every __device__ variable without an initialiser the array is zero when the
// module is loaded, so the counter starts at zero; each call's last block
// resets it for the next call.
constexpr int kNaCounterSlot = 2 * kNaMaxBlocks;
static __device__ __align__(256) double g_noalloc_scratch[2 * kNaMaxBlocks + 32];

__global__ void totals_noalloc_kernel(int64_t n, const int32_t *kind, const double *mass,
                                      const double *rho, const double *e, const double *E,
                                      double *scratch, double *out) {
  double a = 0.0, b = 0.0;
  const int64_t base = (int64_t)blockIdx.x * kNaPerBlock + threadIdx.x;
  for (int k = 0; k < kNaItems; ++k) {
    const int64_t i = base + (int64_t)k * kNaBlock;
    if (i < n && kind[i] == SPH_RT_INTERIOR) {
      a += mass[i] * e[i];
      b += mass[i] / rho[i] * E[i];
    }
  }
  __shared__ double sh[32];
  a = sphrt::block_sum(a, sh);
  __syncthreads();
  b = sphrt::block_sum(b, sh);
  unsigned *counter = reinterpret_cast<unsigned *>(scratch + kNaCounterSlot);
  double part[2] = {a, b}, res[2];
  const bool mx[2] = {false, false};
  // the last block to arrive combines the partials in block order and resets
  // the counter, so the array is ready for the next call
  if (sphrt::last_block_combine<2>(part, scratch, counter, res, mx) && threadIdx.x == 0) {
    out[0] = res[0];
    out[1] = res[1];
  }
}

std::mutex g_mu;
constexpr int kMaxDevices = 64;
double *g_addr[kMaxDevices] = {nullptr};  // device address of the scratch, per device

}  // namespace

extern "C" sph_rt_status sph_rt_energy_totals_noalloc(int64_t n_total, const int32_t *kind,
                                                      const double *mass, const double *rho,
                                                      const double *e, const double *E,
                                                      double *totals, void *stream) {
  if (n_total < 1 || n_total > SPH_RT_NOALLOC_MAX_N) {
    sphrt::set_thread_error("n_total must be in [1, " + std::to_string(SPH_RT_NOALLOC_MAX_N) +
                            "] for the fixed scratch of sph_rt_energy_totals_noalloc");
    return SPH_RT_EINVAL;
  }
  if (!kind || !mass || !rho || !e || !E || !totals) {
    sphrt::set_thread_error("sph_rt_energy_totals_noalloc: NULL array");
    return SPH_RT_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    sphrt::set_thread_error("sph_rt_energy_totals_noalloc: no usable current CUDA device");
    return SPH_RT_EDEVICE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      // set-up, once per device, with that device current
      void *p = nullptr;
      cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (err != cudaSuccess) {
        cudaGetLastError();
        sphrt::set_thread_error(std::string("cudaGetSymbolAddress failed: ") +
                                cudaGetErrorString(err));
        return SPH_RT_EDEVICE;
      }
      g_addr[dev] = static_cast<double *>(p);
    }
    scratch = g_addr[dev];
  }
  const unsigned blocks = (unsigned)((n_total + kNaPerBlock - 1) / kNaPerBlock);
  totals_noalloc_kernel<<<blocks, kNaBlock, 0, st>>>(n_total, kind, mass, rho, e, E, scratch,
                                                     totals);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    sphrt::set_thread_error(std::string("kernel launch failed: ") + cudaGetErrorString(err));
    return SPH_RT_EDEVICE;
  }
  return SPH_RT_OK;
}
