/*
 * sph_rt_noalloc.h -- an entry point of libsphrt that allocates no memory.
 *
 * Not part of the paper's method: the paper has no counterpart.  It exists
 * for callers that cannot let this library allocate device memory while they
 * run it -- a host application whose framework owns the whole device through
 * its own caching allocator (a second allocator would fragment it or be
 * refused), code inside a real-time or timed region where cudaMalloc and
 * cudaFree are forbidden because they synchronise the device, or a process
 * that has handed all free device memory to its own arena.  Such callers keep
 * their particle data in memory they already own and can still ask for the
 * interior energy totals that sph_rt_get_energies reports.
 */
#ifndef SPH_RT_NOALLOC_H
#define SPH_RT_NOALLOC_H

#include <stdint.h>

#include "sph_rt.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Largest n_total accepted: the scratch holds partial sums of at most 4096
 * thread blocks of 8192 particles each. */
#define SPH_RT_NOALLOC_MAX_N ((int64_t)4096 * 8192)

/*
 * Interior energy totals without allocating: totals[0] = sum_i m_i e_i and
 * totals[1] = sum_i (m_i / rho_i) E_i over the particles with kind == 0, the
 * same quantities as the totals of sph_rt_get_energies (summed in a different
 * order, so they agree to rounding).
 *
 * All array arguments are DEVICE pointers of the current CUDA device, in any
 * particle order, length n_total; totals is a device pointer to two doubles,
 * written when the kernel completes on `stream` (a cudaStream_t, NULL = the
 * legacy default stream).  The call only enqueues work; it does not wait.
 *
 * Scratch: a fixed 64 KiB array in the library's static device memory (every
 * GPU that loads the library holds it until the process exits), not a
 * cudaMalloc.  It is zero when the library's device code is loaded, and each
 * call leaves its arrival counter at zero for the next one.  The first call on
 * a device does a set-up step: it looks up that array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it; make that
 * first call before any stream capture.  Every call on a device shares the one
 * array, so calls whose kernels overlap on the GPU (different streams, or
 * concurrent host threads) race and give wrong totals: serialise them.
 *
 * Returns EINVAL for n_total < 1, n_total > SPH_RT_NOALLOC_MAX_N or a NULL
 * pointer (the reason is in sph_rt_last_error(NULL) on the calling thread),
 * EDEVICE for a CUDA error.  Calls no cudaMalloc, cudaFree or allocating
 * library routine.
 */
sph_rt_status sph_rt_energy_totals_noalloc(int64_t n_total, const int32_t *kind,
                                           const double *mass, const double *rho,
                                           const double *e, const double *E, double *totals,
                                           void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SPH_RT_NOALLOC_H */
