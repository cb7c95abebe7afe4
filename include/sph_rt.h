/*
 * sph_rt.h -- C ABI of the GB300 implicit SPH thermal-radiative-transfer step.
 *
 * The library advances the grey two-temperature equations of Bassett, Owen &
 * Brunner (arXiv:2001.11606) -- material energy e and radiation energy E of
 * SPH particles coupled by emission and absorption, radiation transported by
 * flux-limited diffusion -- with backward Euler in time and the paper's
 * nonlinear-elimination (inexact Newton) iteration (Alg. 1).  Space is
 * discretised with the SPH Brookshaw second derivative (Sec. 2.3-2.4).
 *
 * Conventions for every call:
 *  - Arrays are owned by the caller and only read or written during the call.
 *    Unless a name ends in `_device`, pointers are HOST pointers.  `_device`
 *    variants take pointers into device memory of the handle's device; they
 *    are read on the handle's stream (stream-ordered, no host sync needed by
 *    the caller beyond normal stream semantics).
 *  - Particle arrays are in the CALLER'S order, length n_total (interior and
 *    ghost particles together); positions are row-major [n_total][dim].
 *  - The handle (sph_rt*) is owned by the library; a stream passed in the
 *    configuration is borrowed, never destroyed.
 *  - One handle is used by one host thread at a time.
 *  - Errors are negative sph_rt_status codes; sph_rt_last_error() gives a
 *    message.  Input validation happens on the host before any device work,
 *    so an invalid call leaves the handle unchanged.  A step that does not
 *    converge returns SPH_RT_ENOTCONV and leaves the state at t^{n-1}.
 *  - All arithmetic of the FP64 path is IEEE double on the device; FMA
 *    contraction is disabled where results are compared bit for bit
 *    (neighbour distances).
 */
#ifndef SPH_RT_H
#define SPH_RT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_rt sph_rt; /* opaque handle */

typedef enum {
  SPH_RT_OK = 0,
  SPH_RT_EINVAL = -1,   /* invalid argument (checked on the host) */
  SPH_RT_ENOMEM = -2,   /* device allocation failed */
  SPH_RT_ENOTCONV = -3, /* outer or Krylov iteration limit reached; state unchanged */
  SPH_RT_EDEVICE = -4,  /* CUDA error; message has the CUDA error string */
  SPH_RT_ESTATE = -5    /* call out of order (e.g. step before set_particles) */
} sph_rt_status;

enum { SPH_RT_INTERIOR = 0, SPH_RT_DIRICHLET = 1, SPH_RT_COPY = 2 };
enum { SPH_RT_LIMITER_NONE = 0, SPH_RT_LIMITER_LEVERMORE = 1, SPH_RT_LIMITER_LARSEN = 2 };
enum { SPH_RT_PRECOND_JACOBI = 0, SPH_RT_PRECOND_CHEBYSHEV = 1, SPH_RT_PRECOND_AMG = 2 };
enum { SPH_RT_FP64 = 0, SPH_RT_MIXED = 1 };
/* SPH kernel: the M4 cubic B-spline with support 2h, or the paper's Wendland C4
 * kernel with support h (Sec. 2.4, Eq. wendlandc4; the printed polynomial in
 * every dimension, normalised to a unit volume integral, Sec. 2.3). */
enum { SPH_RT_M4_SPLINE = 0, SPH_RT_WENDLAND_C4 = 1 };
/* cell list of the neighbour search (sph_rt_config.cell_list) */
enum { SPH_RT_CELLS_AUTO = 0, SPH_RT_CELLS_DENSE = 1, SPH_RT_CELLS_SORTED = 2 };

/*
 * Problem constants and solver controls.
 * Physics (Sec. 2.1-2.2): B = a T^4, e = c_v T, sigma_a = sigma0 T^p,
 * sigma_t = sigma_a + sigma_s, D = c lambda(R) / sigma_t with
 * R = |grad E| / (sigma_t E) and lambda from
 *   none      lambda = 1/3                      (Fick's law, Eq. diffusion with 1/3)
 *   Levermore lambda = (2+R)/(6+3R+R^2)          (Sec. 2.1, Levermore limiter)
 *   Larsen    lambda = (3^k + R^k)^(-1/k)        (Sec. 2.1, Larsen limiter)
 * Tolerances (Table tab:tolerances, Eq. mat-rad-convergence):
 *   tol_outer_e / tol_outer_E  max_i |x^{l+1}-x^l| / |x^{l+1}| of the outer loop
 *   tol_inner_e                per-particle Newton |de| <= tol |e|
 *   tol_krylov                 ||b - A E||_2 <= tol ||b||_2 (unscaled rows)
 */
typedef struct {
  int32_t dim;          /* 2 or 3 (1 is accepted too) */
  int32_t kernel;       /* SPH_RT_M4_SPLINE (default) or SPH_RT_WENDLAND_C4 */
  double a, c, cv;      /* radiation constant (>= 0; 0: no emission), speed of light, specific
                           heat (both > 0) */
  int32_t limiter;      /* SPH_RT_LIMITER_* */
  double larsen_k;      /* k of the Larsen limiter (> 0) */
  double opacity_exp;   /* p in sigma = sigma0 T^p */
  double T_floor;       /* T inside sigma and R is max(T, T_floor); 0 = off */
  double sigma_s;       /* scattering opacity (constant, >= 0): sigma_t = sigma_a + sigma_s
                           sets R and D; sigma_a alone the emission and absorption */
  double tol_outer_e, tol_outer_E, tol_inner_e, tol_krylov;
  int32_t max_outer, max_inner_e, max_krylov;
  int32_t precond;      /* SPH_RT_PRECOND_* */
  int32_t precision;    /* SPH_RT_FP64 or SPH_RT_MIXED */
  int32_t cheb_degree;  /* Chebyshev smoother / preconditioner degree (1..16; default 1: on
                           GB300 each extra degree costs a fine-level FP64 sweep, and degree 1
                           gave the fastest AMG-CG at 64^3 and 128^3) */
  int32_t amg_rebuild;  /* 1: redo AMG aggregation every step; 0: keep the first step's */
  double amg_theta;     /* AMG strength threshold: j strong for i if |B_ij| >= theta sqrt(B_ii B_jj) */
  int32_t check_every;  /* Krylov iterations queued between host convergence reads */
  int32_t kernel_timing;/* 1: record CUDA events around SpMV launches (sph_rt_kernel_stats) */
  int32_t autotune;     /* 1: autotune on the first step.  The fine SpMV loads in flight (U = 4
                           or 8; never changes a result bit) on the first step of a particle
                           set (kept for later particle sets within 25 % of its rows and
                           entries), and once per handle the smoother: one timed trial step (after
                           an untimed one that captures its graph) from the same state for
                           each candidate -- with the AMG preconditioner finest-level
                           post-smoothing off (fine_post_smooth = 0, cheb_degree = 1; in the
                           mixed form with reliable_drop 1e-4 and 1e-6) or on with
                           cheb_degree 1, 2, 3; with the Chebyshev preconditioner degrees 1,
                           2, 3, 4, 6 -- keeping the fastest that converges in the handle's
                           configuration (sph_rt_get_config, sph_rt_get_solver_tuning).  The
                           state is restored after every trial.  2: the loads in flight only.
                           0 (default): as configured.  In a batch (sph_rt_batch_*), 1 tunes
                           the batched launch's shape on its first step */
  int32_t amg_tail;     /* 1: run the small AMG levels (each <= 600k stored entries) of every
                           V-cycle as one thread-block-cluster launch (bitwise the same result;
                           default 0: measured no faster than the per-level launches) */
  int32_t coarse_fp32;  /* 1: the coarsest AMG level's Chebyshev solve (<= 2,048 rows, one
                           thread block) is staged and computed in FP32, also in the FP64 form:
                           in FP64 it is bound by one SM's FP64 rate.  It is part of the
                           preconditioner only; residuals and updates stay FP64 */
  int32_t graphs;       /* 1: run each step's outer loop as one CUDA graph with conditional
                           WHILE nodes (no host round trip per iteration); ignored while
                           kernel_timing = 1, which needs per-launch events */
  int32_t pdl;          /* 1: launch the Krylov iteration's kernels with programmatic
                           dependent launch (a kernel's blocks are scheduled while its
                           predecessor drains; each waits for the predecessor's results before
                           touching them), 0: ordinary stream order.  Same results either way */
  int32_t fine_post_smooth; /* AMG preconditioner only.  1: the V-cycle smooths before and after
                           the coarse correction on every level (symmetric; the CG product
                           B p is a sweep of its own).  0: the finest level only pre-smooths;
                           its residual sweep and the A P sweep of the coarse correction then
                           give B z, so the CG (flexible: the V-cycle is not symmetric) needs
                           no product sweep -- two sweeps of the fine operator per iteration
                           instead of three, for ~1.4x the iterations.  With 0 and the mixed
                           precision the CG vectors are FP32 too, and the FP64 residual
                           replaces the recursive one (see reliable_drop).  Requires
                           cheb_degree = 1 */
  double reliable_drop; /* mixed precision with fine_post_smooth = 0: the FP64 residual
                           b - A x replaces the FP32 recursive one whenever the latter has
                           dropped by this factor since the last replacement, and before
                           convergence is accepted (the solve stops on the FP64 residual).
                           In (0, 1) */
  /* Time step choice (Sec. 3.3, Eq. energy-fractional).  With dt_target > 0 every
   * converged step reports in its stats the fractional changes
   *   eta_x = max_i |x_i^n - x_i^{n-1}| / (x_i^n + dt_target xbar^n + dt_eta_floor)
   * of x = e and x = E over the interior particles (xbar^n: volume average,
   * sum x_i V_i / sum V_i) and the proposed next step
   *   dt_next = min(dt (dt_target / eta_e)^(1/2), dt (dt_target / eta_E)^(1/2),
   *                 dt_growth dt, dt_max), at least dt_min.
   * The caller passes dt_next (or any other dt) to the next sph_rt_step. */
  double dt_target;     /* target fractional change (the paper uses 0.05); 0 = off */
  double dt_growth;     /* largest factor between consecutive steps (>= 1) */
  double dt_min, dt_max;
  double dt_eta_floor;  /* added to the denominator for states that may be zero everywhere */
  int32_t cell_list;    /* neighbour search cell list (SPH_RT_CELLS_*): AUTO (default) takes the
                           dense key table while the grid has at most 2^26 cells and the sorted
                           64-bit keys (radix sort, hash table of occupied cells; up to 2^58
                           cells) beyond; DENSE refuses larger grids with EINVAL; SORTED always
                           sorts.  Both give the same slots and neighbour lists. */
  int32_t index64;      /* 1: 64-bit source indices in the AMG set-up's Galerkin lists even where
                           32 bits suffice; 0 (default): 64 bits only for a level with 2^31 - 1
                           or more entries plus rows.  Never changes a result. */
  int32_t krylov_start; /* start of each step's first linear solve: 0 E^{n-1}, the state
                           (Alg. 1's E^{n,0}); p = 1, 2, 3 (default 3) the value at t_n of the
                           polynomial in time through E^{n-1}, ..., E^{n-1-p} (Lagrange
                           extrapolation), of lower order while fewer converged steps of the
                           same particle set are behind it.  Only the Krylov start changes:
                           the stopping test (||r|| <= tol_krylov ||b||), the outer iteration
                           and its fixed point do not.  The handle and the batched form (per
                           problem) both follow it. */
  int32_t device;       /* CUDA device ordinal */
  void *stream;         /* cudaStream_t to run on (borrowed); NULL = library-owned stream */
} sph_rt_config;

/* Per-step diagnostics (the paper's columns: outer iterations per step and
 * Krylov iterations per outer iteration, Sec. 4.3 -- the first 64 outer
 * iterations are recorded; energy balance, Sec. 2.5). */
typedef struct {
  int32_t outer_iters;
  int32_t krylov_iters_total;
  int32_t krylov_iters_per_outer[64];
  int32_t newton_iters_max;
  double energy_before, energy_after; /* sum_i m_i e_i + V_i E_i over interior particles */
  double source_energy;               /* dt sum_i V_i (Q_e + Q_E) */
  double boundary_energy;             /* dt sum_i V_i sum_{j ghost} w_ij (E_j - E_i) */
  double last_change_e, last_change_E;/* final outer-loop changes */
  double t_setup_ms, t_assembly_ms, t_amg_ms, t_krylov_ms, t_newton_ms;
  double eta_e, eta_E;                /* fractional changes of the step (config.dt_target > 0) */
  double dt_next;                     /* proposed next step (config.dt_target > 0), else 0 */
} sph_rt_stats;

/* Fill *cfg with defaults: dim 3, a = c = c_v = 1, no limiter, p = 0,
 * tolerances of Table tab:tolerances (manufactured problem row) with
 * tol_inner_e = 1e-13, AMG preconditioner (theta 0.02, Chebyshev degree 1,
 * coarsest solve in FP32), FP64, the per-step CUDA graph and programmatic
 * dependent launch on, device 0, own stream. */
void sph_rt_default_config(sph_rt_config *cfg);

/* Create a handle.  No device work happens until sph_rt_set_particles.
 * Returns EINVAL (and *out = NULL) for an out-of-range configuration; the
 * reason is then available from sph_rt_last_error(NULL) on the same thread. */
sph_rt_status sph_rt_create(const sph_rt_config *cfg, sph_rt **out);

/*
 * Set the particles (positions, masses, densities, smoothing lengths, opacity
 * prefactors, kinds) and the initial state; build the Morton-sorted cell list,
 * the neighbour lists (j != i with r^2 < (s max(h_i,h_j))^2, s = 2 for the
 * cubic B-spline and 1 for the Wendland C4 kernel, Sec. 3.1), the
 * fixed geometric weights and the operator's sparsity.  Replaces any previous
 * particle set.
 *   kind[i]    SPH_RT_INTERIOR, SPH_RT_DIRICHLET (ghost with prescribed values)
 *              or SPH_RT_COPY (ghost that copies interior particle copy_of[i])
 *   copy_of    may be NULL when there are no copy ghosts
 *   e0, E0     initial material and radiation energy (ghosts: their values)
 * EINVAL: n_total < 1, no interior particle, non-finite value, m/rho/h <= 0,
 * sigma0 < 0, kind out of range, copy_of not pointing at an interior particle.
 */
sph_rt_status sph_rt_set_particles(sph_rt *s, int64_t n_total, const double *pos,
                                   const double *mass, const double *rho, const double *h,
                                   const double *sigma0, const int32_t *kind,
                                   const int64_t *copy_of, const double *e0, const double *E0);

/* Same, with every array in device memory. */
sph_rt_status sph_rt_set_particles_device(sph_rt *s, int64_t n_total, const double *pos,
                                          const double *mass, const double *rho,
                                          const double *h, const double *sigma0,
                                          const int32_t *kind, const int64_t *copy_of,
                                          const double *e0, const double *E0);

/*
 * One backward-Euler step of size dt (Eq. ne-starting-point, Alg. 1):
 *   material data from the state at the step's start (Sec. 3.2), operator
 *   assembly, preconditioner set-up, initial material solve, then outer
 *   iterations of {diffusion solve (Eq. diffusion-solve), material solve
 *   (Eq. material-energy-solve)} until Eq. mat-rad-convergence holds.
 *   Qe, QE    sources at t^n [n_total] (ghost entries ignored); NULL = 0
 *   ghost_e, ghost_E  Dirichlet-ghost values at t^n [n_total] (other entries
 *             ignored); NULL = keep the current ghost values
 *   stats     may be NULL
 * EINVAL (state unchanged): dt not finite and positive, or a non-finite
 * source of an interior particle or ghost value of a Dirichlet ghost (checked
 * on the device before the state is touched).
 */
sph_rt_status sph_rt_step(sph_rt *s, double dt, const double *Qe, const double *QE,
                          const double *ghost_e, const double *ghost_E, sph_rt_stats *stats);

/* Same, with the four arrays in device memory. */
sph_rt_status sph_rt_step_device(sph_rt *s, double dt, const double *Qe, const double *QE,
                                 const double *ghost_e, const double *ghost_E,
                                 sph_rt_stats *stats);

/* The history of the extrapolated Krylov start (krylov_start = p > 0), for checkpoints.
 * Row j of E_hist [3][n_total] (caller order, host) is E^{n-2-j}, the radiation energy at
 * the start of the step j + 1 steps back (row 0: the last step's start), and dt_hist[j]
 * that step's dt; depth = min(p, converged steps of this particle set behind the state)
 * rows are valid, the ones the next step reads.
 * get: writes *depth (0 after sph_rt_set_particles or a step that did not converge), the
 *   valid rows (rows beyond depth and every ghost entry are 0) and dt_hist[3]; E_hist and
 *   dt_hist may be NULL.
 * set (after sph_rt_set_particles): installs depth rows (1 <= depth <= p, EINVAL
 *   otherwise; every entry finite, ghost entries ignored; dt_hist[0 .. depth-1] > 0), so a
 *   checkpoint of e, E and this history restarts bit for bit.  Both synchronise the
 *   stream. */
sph_rt_status sph_rt_get_history(sph_rt *s, int32_t *depth, double *E_hist, double *dt_hist);
/* The weights of that extrapolation (host only, no device work): w[0 .. order] with
 * sum_j w[j] E^{n-1-j} the value at t_n = t_{n-1} + dt of the polynomial of degree `order`
 * (0..3) through E^{n-1}, ..., E^{n-1-order}; dt_hist[j] = t_{n-1-j} - t_{n-2-j} (newest
 * first).  EINVAL for another order or a step that is not finite and > 0. */
sph_rt_status sph_rt_extrapolation_weights(int32_t order, double dt, const double *dt_hist,
                                           double *w);
sph_rt_status sph_rt_set_history(sph_rt *s, int32_t depth, const double *E_hist,
                                 const double *dt_hist);

/* Copy the current state out, caller order [n_total] (either may be NULL);
 * totals[0] = sum m_i e_i, totals[1] = sum V_i E_i over interior particles
 * (may be NULL). */
sph_rt_status sph_rt_get_energies(sph_rt *s, double *e, double *E, double totals[2]);

/* Same into device memory. */
sph_rt_status sph_rt_get_energies_device(sph_rt *s, double *e, double *E);

/*
 * Smoothing lengths by the initialisation iteration of Sec. 3.1: the support
 * radius of every interior particle becomes eta local particle spacings (the
 * paper uses eta = 4 with the Wendland C4 kernel).  Reading of the ASPH method
 * the paper names: each particle iterates on the kernel's zeroth moment
 * S_i(h) = sum_j W(r_ij, h) (the SPH number density, i included):
 *   h_i <- h_i (eta / s) / (h_i^d S_i(h_i))^(1/d),  at most x2 or /2 per update,
 * s = the kernel's support in units of h, until |dh_i| <= tol h_i or max_iter
 * updates.  Copy ghosts take the h of the particle they copy, Dirichlet ghosts
 * keep theirs.  Starts from the current h; then rebuilds the neighbour lists and
 * operator sparsity (as sph_rt_set_particles) with the state e, E kept.
 * *iters (may be NULL): the largest number of updates of a particle.
 * EINVAL: eta or tol not positive, max_iter < 1, or a starting h so large that
 * one support holds more than 4096 particles; ENOTCONV if the lengths keep
 * growing past six successive search grids (the particle set is unchanged).
 */
sph_rt_status sph_rt_adapt_smoothing_lengths(sph_rt *s, double eta, double tol,
                                             int32_t max_iter, int32_t *iters);

/* Current smoothing lengths, caller order [n_total] (host). */
sph_rt_status sph_rt_get_smoothing_lengths(sph_rt *s, double *h);

/*
 * Moving particles: new positions (caller order, row-major [n_total][dim]) for
 * the current particle set.  Masses, densities, smoothing lengths, opacities,
 * kinds, copy sources and the state e, E are kept; the Morton order, the
 * neighbour lists and the operator sparsity are rebuilt (rows a1-a2 re-run),
 * and the next step builds a new AMG hierarchy.  EINVAL: a non-finite position.
 */
sph_rt_status sph_rt_move_particles(sph_rt *s, const double *pos);

/* Same, with the positions in device memory. */
sph_rt_status sph_rt_move_particles_device(sph_rt *s, const double *pos);

/* Sizes after set_particles: interior count, neighbour-list nnz, operator nnz. */
sph_rt_status sph_rt_get_sizes(const sph_rt *s, int64_t *n_interior, int64_t *nnz_neighbors,
                               int64_t *nnz_operator);

/* Test hook: neighbour lists in caller IDs.  rowptr[n_total+1]; cols[nnz]
 * sorted ascending within each row; ghost rows are empty.  cols may be NULL
 * to get rowptr only. */
sph_rt_status sph_rt_get_neighbors(sph_rt *s, int64_t *rowptr, int64_t *cols);

/*
 * Test hook: the operator assembled by the last step, in caller IDs, scaled
 * back to the paper's rows (Eq. diffusion-solve): row i (interior) holds
 * A_ij for interior columns j (a copy ghost's entry under the column of the
 * particle it copies, duplicates summed by the caller if needed), diag[i] = A_ii,
 * gb[i] = Dirichlet-ghost coupling sum_j w_ij E_j.  rowptr[n_total+1];
 * cols/vals sized by nnz_operator.  Any output may be NULL.
 */
sph_rt_status sph_rt_get_operator(sph_rt *s, int64_t *rowptr, int64_t *cols, double *vals,
                                  double *diag, double *gb);

/* Test hook: material data of the last step, caller order [n_total]:
 * T, sigma, Fleck factor f, R, lambda, D.  Any may be NULL. */
sph_rt_status sph_rt_get_properties(sph_rt *s, double *T, double *sigma, double *f, double *R,
                                    double *lambda, double *D);

/* Kernel timing (config.kernel_timing = 1): number of SpMV launches on the
 * fine operator since the last reset, their summed CUDA-event time in ms, and
 * their algorithmic bytes (12 per stored nonzero + 8 per row for rowptr,
 * x and y).  reset != 0 clears the counters after reading. */
sph_rt_status sph_rt_kernel_stats(sph_rt *s, int64_t *launches, double *total_ms,
                                  double *bytes, int reset);

/* The same counters split by kernel: SPH_RT_KERNEL_SPMV_PQ (the CG product
 * fused with the p, q updates and (p, q)), SPH_RT_KERNEL_RESID (residual
 * sweeps: CG start and V-cycle fine level), SPH_RT_KERNEL_CHEB (fine-level
 * Chebyshev smoother / preconditioner sweeps), SPH_RT_KERNEL_POST (the sweep
 * of A P on the finest level with the prolongation folded in: the first
 * post-smoothing step, or with fine_post_smooth = 0 the sweep that forms z and
 * B z), SPH_RT_KERNEL_TRUE_RESID (with fine_post_smooth = 0: the FP64 residual
 * b - A x at the start of a solve and at each reliable update).  Cleared with
 * the totals. */
enum { SPH_RT_KERNEL_SPMV_PQ = 0, SPH_RT_KERNEL_RESID = 1, SPH_RT_KERNEL_CHEB = 2,
       SPH_RT_KERNEL_POST = 3, SPH_RT_KERNEL_TRUE_RESID = 4 };
sph_rt_status sph_rt_kernel_stats_kind(sph_rt *s, int32_t kind, int64_t *launches,
                                       double *total_ms, double *bytes);

/* AMG hierarchy of the last step: number of levels, and rows and stored
 * off-diagonal nonzeros per level (arrays of max_levels entries, may be NULL). */
sph_rt_status sph_rt_get_amg_info(sph_rt *s, int32_t *nlevels, int64_t *rows, int64_t *nnz,
                                  int32_t max_levels);

/* Number of this library's kernels launched since creation (all kinds; the
 * kernels a loop graph ran are counted from its device trip counters). */
int64_t sph_rt_launch_count(const sph_rt *s);

/* Device-driven outer loop (config.graphs = 1): how many times the loop graph
 * was captured (once per particle set / AMG hierarchy / dt while nothing else
 * changes) and launched (once per step).  Either pointer may be NULL. */
sph_rt_status sph_rt_loop_graph_info(const sph_rt *s, int64_t *captures, int64_t *launches);

/* The handle's configuration as it stands (the solver autotuner's choice
 * included). */
sph_rt_status sph_rt_get_config(const sph_rt *s, sph_rt_config *cfg);

/* Trials of the solver autotuner (config.autotune): *count = the number of
 * trials (0 before the first step or without autotune), the first min(cap,
 * count) copied to trials (may be NULL).  ms is the timed trial step's CUDA-
 * event time, -1 where the step did not converge. */
typedef struct {
  int32_t fine_post_smooth, cheb_degree;
  double reliable_drop, ms;
} sph_rt_tune_trial;
sph_rt_status sph_rt_get_solver_tuning(const sph_rt *s, sph_rt_tune_trial *trials, int32_t cap,
                                       int32_t *count);

/* ------------------------------------------------------------------------ */
/* Serving: a continuous-batching request loop over many independent        */
/* problems on one GPU.  This is a runtime around the calls above, not part */
/* of the paper's method (the paper runs one problem at a time).            */
/*                                                                          */
/* Every admitted request is resident on the device in its own handle and   */
/* stream; worker threads advance resident requests `steps_per_tick` steps  */
/* at a time, so the work of different requests overlaps on the GPU.  Small  */
/* requests (n_total <= fuse_max_n) that are ready together and share the   */
/* configuration, dt and step count are fused: up to fuse_max_k of them run */
/* as one sph_rt_batch (one persistent launch per step, all steps in one    */
/* CUDA-graph launch).  A fused request's result is the batched form's      */
/* result, the same as in a batch of its own.  With cfg.autotune = 1 the     */
/* first fused batch of a configuration and dt tunes its launch shape        */
/* (sph_rt_batch_autotune) and later fused batches of that key reuse it.     */
/* Queued requests are admitted in FIFO order while the device footprint of */
/* the resident ones stays within hbm_budget_bytes (an estimate until a     */
/* request is set up, its measured allocation after; the library's cache of */
/* freed device buffers, at most 8 GB per device, is outside the budget).   */
/* A request's result does not depend on the other requests (same           */
/* deterministic kernels on its own data).                                  */
/* ------------------------------------------------------------------------ */
typedef struct sph_rt_srv sph_rt_srv;
enum { SPH_RT_SRV_QUEUED = 0, SPH_RT_SRV_ADMITTED = 1, SPH_RT_SRV_RUNNING = 2,
       SPH_RT_SRV_DONE = 3, SPH_RT_SRV_FAILED = 4 };

typedef struct {
  int32_t workers;         /* host threads driving resident requests (>= 1) */
  int32_t max_resident;    /* cap on resident requests (>= 1) */
  int32_t steps_per_tick;  /* steps a worker advances a request before rotating */
  double hbm_budget_bytes; /* admission budget for resident device memory */
  int32_t device;
  int64_t fuse_max_n;      /* largest n_total run in a fused batch; 0 = never fuse */
  int32_t fuse_max_k;      /* most requests in one fused batch (>= 1) */
} sph_rt_srv_config;

typedef struct {
  int32_t queued, resident, peak_resident;
  int64_t resident_bytes, peak_bytes; /* budget accounting */
  int64_t particle_steps;             /* completed interior particle-steps */
  double t_first_submit, t_last_done; /* seconds on the server's steady clock */
  int64_t fused_requests, fused_batches; /* requests run fused, and fused batches run */
} sph_rt_srv_info_t;

/* Defaults: 8 workers, 64 resident, 1 step per tick, 120e9-byte budget,
 * device 0, fuse requests of up to 20,000 particles, 64 per batch. */
void sph_rt_srv_default_config(sph_rt_srv_config *cfg);
sph_rt_status sph_rt_srv_create(const sph_rt_srv_config *cfg, sph_rt_srv **out);

/* Queue a request: a configuration (its stream and device fields are ignored),
 * particles and initial state as for sph_rt_set_particles, constant sources
 * Qe/QE (NULL = 0; ghost values stay as given in e0/E0) and `steps` steps of
 * size dt.  All arrays are copied before the call returns.  *request_id gets
 * the request's id. */
sph_rt_status sph_rt_srv_submit(sph_rt_srv *srv, const sph_rt_config *cfg, int64_t n_total,
                                const double *pos, const double *mass, const double *rho,
                                const double *h, const double *sigma0, const int32_t *kind,
                                const int64_t *copy_of, const double *e0, const double *E0,
                                const double *Qe, const double *QE, int32_t steps, double dt,
                                int64_t *request_id);

/* State (SPH_RT_SRV_*) and times {submit, admit, done} of a request. */
sph_rt_status sph_rt_srv_poll(sph_rt_srv *srv, int64_t request_id, int32_t *state,
                              double times[3]);

/* Block until the request is done or failed; returns its status. */
sph_rt_status sph_rt_srv_wait(sph_rt_srv *srv, int64_t request_id);

/* Final state (caller order [n_total], either may be NULL), the stats of its
 * last step, and the error message of a failed request (msg may be NULL). */
sph_rt_status sph_rt_srv_result(sph_rt_srv *srv, int64_t request_id, double *e, double *E,
                                sph_rt_stats *last_stats, char *msg, int64_t msg_len);

sph_rt_status sph_rt_srv_info(sph_rt_srv *srv, sph_rt_srv_info_t *info);

/* Stop the workers (after their current tick), release every resident
 * request and the server. */
void sph_rt_srv_destroy(sph_rt_srv *srv);

/* ------------------------------------------------------------------------ */
/* Batched form: many small problems advanced by one persistent launch per  */
/* step and cluster size.  Each problem gets one thread-block cluster (1 to  */
/* 8 blocks, by its size) that runs its whole step (material data,          */
/* assembly, material solves and Chebyshev-preconditioned CG with           */
/* cluster-wide reductions, per-problem convergence); all problems share the */
/* configuration (physics, tolerances, cheb_degree).  Like serving, this is a */
/* runtime form around the paper's method, not part of the method itself.    */
/* ------------------------------------------------------------------------ */
typedef struct sph_rt_batch sph_rt_batch;

sph_rt_status sph_rt_batch_create(const sph_rt_config *cfg, sph_rt_batch **out);

/* Add a problem (host arrays as for sph_rt_set_particles; set-up runs now).
 * *index gets its position in the batch.  Problems can only be added before
 * the first step. */
sph_rt_status sph_rt_batch_add(sph_rt_batch *b, int64_t n_total, const double *pos,
                               const double *mass, const double *rho, const double *h,
                               const double *sigma0, const int32_t *kind, const int64_t *copy_of,
                               const double *e0, const double *E0, int32_t *index);

/* Several problems at once: their set-ups run on `threads` host threads (<= 0:
 * 1), each problem on its own stream, so that they overlap on the GPU.  The arrays
 * are as for sph_rt_batch_add; problem k gets index *first_index + k (may be
 * NULL).  All or none are added: on an error no problem is added, and the
 * message names the first failing problem. */
typedef struct {
  int64_t n_total;
  const double *pos, *mass, *rho, *h, *sigma0;
  const int32_t *kind;
  const int64_t *copy_of;
  const double *e0, *E0;
} sph_rt_problem;
sph_rt_status sph_rt_batch_add_many(sph_rt_batch *b, int32_t count, const sph_rt_problem *problems,
                                    int32_t threads, int32_t *first_index);

/* Constant sources of one problem (caller order, NULL = 0), used every step. */
sph_rt_status sph_rt_batch_set_sources(sph_rt_batch *b, int32_t index, const double *Qe,
                                       const double *QE);

/* One backward-Euler step of every problem in ONE kernel launch.  Per problem
 * (arrays of sph_rt_batch_size entries, any may be NULL): status (0, or -3 if
 * it did not converge -- its state is then unchanged), outer iterations,
 * Krylov iterations, and energy[4k..4k+3] = before, after, source, boundary
 * inflow.  Returns ENOTCONV if any problem did not converge. */
sph_rt_status sph_rt_batch_step(sph_rt_batch *b, double dt, int32_t *status,
                                int32_t *outer_iters, int32_t *krylov_iters, double *energy);

/* `steps` backward-Euler steps of size dt of every problem with ONE CUDA-graph
 * launch: the graph holds the `steps` launches of the batched step kernel and
 * a per-step accumulation, is captured on the first run and replayed by later
 * runs with the same dt and steps.  A problem whose step does not converge
 * keeps the state of its last converged step and skips the remaining steps.
 * Per problem (arrays of sph_rt_batch_size entries, any may be NULL): status
 * of the run (0, or -3), and outer and Krylov iterations summed over the steps
 * it ran.  Returns ENOTCONV if any problem failed.  The results equal those of
 * `steps` calls of sph_rt_batch_step. */
sph_rt_status sph_rt_batch_run(sph_rt_batch *b, double dt, int32_t steps, int32_t *status,
                               int32_t *outer_total, int32_t *krylov_total);

/* Launch shape of the batched step.  lanes_per_row W: 1, 2, 4 or 8 (a warp
 * works on 32 / W rows at a time); cheb_degree: 1..16 (1 is a Jacobi
 * preconditioner); blocks_per_sm: 1 or 2 resident blocks per SM (2 caps the
 * registers per thread at 64 so that twice as many blocks are in flight);
 * rows_per_cta: 0, or >= 64 -- a problem of n interior particles runs on a
 * thread-block cluster of C = 1, 2, 4 or 8 blocks, the smallest power of two
 * with C * rows_per_cta >= n (at most 8, and at most what the GPU can
 * co-schedule), each block owning a contiguous share of its rows; 0 gives
 * every problem one block.  W and blocks_per_sm never change a result; the
 * degree changes the Krylov path and rows_per_cta the order of the sums
 * (results then agree to the solver tolerances).  A problem's result depends
 * on its own data and the shape only, not on the other problems of the batch.
 * Until set or tuned, W follows the mean row length (4, or 8 above 160
 * entries), the degree is cfg.cheb_degree, blocks_per_sm is 2 when the batch
 * has more problems than the GPU has SMs, and rows_per_cta is 4096.  Setting
 * the shape turns off the automatic tuning of cfg.autotune.  EINVAL for a
 * value outside those sets. */
typedef struct {
  int32_t lanes_per_row, cheb_degree, blocks_per_sm, rows_per_cta;
} sph_rt_batch_shape;
sph_rt_status sph_rt_batch_set_shape(sph_rt_batch *b, const sph_rt_batch_shape *shape);
sph_rt_status sph_rt_batch_get_shape(const sph_rt_batch *b, sph_rt_batch_shape *shape);

/* Autotuner of the batched launch.  Runs one step of size dt of the whole
 * batch for each candidate shape, each from the current state, which is
 * restored after every trial (the problems do not advance), times each step
 * with CUDA events and keeps the fastest shape among those with which every
 * problem converged (the current shape if none did).  Candidates, in the
 * order of times_ms: first the 40 shapes blocks_per_sm in {1, 2} (outermost)
 * x lanes_per_row in {1, 2, 4, 8} x cheb_degree in {1, 2, 3, 4, 6}
 * (innermost) at the current rows_per_cta, then rows_per_cta in {0, 2048,
 * 4096, 8192} with the best of those.  times_ms[SPH_RT_BATCH_TUNE_CANDIDATES]
 * (may be NULL) gets each trial's time in milliseconds, -1 where some problem
 * did not converge; the chosen shape goes to *chosen (may be NULL) and stays
 * set.  With cfg.autotune = 1 the first sph_rt_batch_step or sph_rt_batch_run
 * of a batch whose shape was not set calls it with that call's dt.  The
 * choice rests on timings, so two batches of the same problems may pick
 * different shapes. */
#define SPH_RT_BATCH_TUNE_CANDIDATES 44
sph_rt_status sph_rt_batch_autotune(sph_rt_batch *b, double dt, float *times_ms,
                                    sph_rt_batch_shape *chosen);

/* State of one problem, caller order (either may be NULL). */
sph_rt_status sph_rt_batch_get_energies(sph_rt_batch *b, int32_t index, double *e, double *E);

/* Sizes of problem `index`: info[0] = particles (n_total), info[1] = interior
 * particles, info[2] = stored off-diagonal operator entries, info[3] =
 * neighbour-list entries, info[4] = blocks of the cluster it runs on with the
 * current shape (valid once the batch has stepped or been tuned: the GPU's
 * largest co-schedulable cluster is known then).  EINVAL for an index
 * outside the batch. */
sph_rt_status sph_rt_batch_problem_info(const sph_rt_batch *b, int32_t index, int64_t info[5]);

int32_t sph_rt_batch_size(const sph_rt_batch *b);
const char *sph_rt_batch_last_error(const sph_rt_batch *b);
void sph_rt_batch_destroy(sph_rt_batch *b);

/* Message of the last failed call on this handle (NULL: of the last failed
 * sph_rt_create on this thread).  Owned by the library; valid until the next
 * call on the handle. */
const char *sph_rt_last_error(const sph_rt *s);

/* Release the handle (NULL is a no-op).  Its device buffers go to a
 * library-wide cache per device (at most 8 GB; the rest back to CUDA), from
 * which later handles take before allocating, so that handles created and
 * destroyed again and again neither allocate nor synchronise the device. */
void sph_rt_destroy(sph_rt *s);

/* Return the cache's buffers of `device` to CUDA (cudaFree).  Safe at any
 * time: cached buffers belong to no handle.  EINVAL for a negative device. */
sph_rt_status sph_rt_release_cached_memory(int32_t device);

#ifdef __cplusplus
}
#endif
#endif /* SPH_RT_H */
