"""Python binding of libsphrt (include/sph_rt.h): argument marshalling only.

Every computation happens in the CUDA library.  Importing this module does not
need a GPU; loading the library does (it links the CUDA runtime), and every
call that touches the device fails loudly if the library or the GPU is missing.
There is no CPU fallback.

Function names follow the C ABI (`create`, `set_particles`, `step`,
`get_energies`, ...).  Host arrays are numpy arrays; the `*_device` variants
take raw device pointers (ints), e.g. `torch.Tensor.data_ptr()`.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ENOTCONV, EDEVICE, ESTATE = 0, -1, -2, -3, -4, -5
INTERIOR, DIRICHLET, COPY = 0, 1, 2
LIMITER_NONE, LIMITER_LEVERMORE, LIMITER_LARSEN = 0, 1, 2
PRECOND_JACOBI, PRECOND_CHEBYSHEV, PRECOND_AMG = 0, 1, 2
FP64, MIXED = 0, 1
M4_SPLINE, WENDLAND_C4 = 0, 1
CELLS_AUTO, CELLS_DENSE, CELLS_SORTED = 0, 1, 2
# candidate shapes of sph_rt_batch_autotune: a grid, outermost first, then the
# rows per CTA (SPH_RT_BATCH_TUNE_CANDIDATES = 2 x 4 x 5 + 4)
BATCH_TUNE_BLOCKS = (1, 2)
BATCH_TUNE_LANES = (1, 2, 4, 8)
BATCH_TUNE_DEGREES = (1, 2, 3, 4, 6)
BATCH_TUNE_ROWS = (0, 2048, 4096, 8192)
BATCH_TUNE_CANDIDATES = (len(BATCH_TUNE_BLOCKS) * len(BATCH_TUNE_LANES) * len(BATCH_TUNE_DEGREES)
                         + len(BATCH_TUNE_ROWS))
_NAMES = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ENOTCONV: "ENOTCONV", EDEVICE: "EDEVICE",
          ESTATE: "ESTATE"}


class Config(C.Structure):
    _fields_ = [
        ("dim", C.c_int32),
        ("kernel", C.c_int32),
        ("a", C.c_double), ("c", C.c_double), ("cv", C.c_double),
        ("limiter", C.c_int32),
        ("larsen_k", C.c_double),
        ("opacity_exp", C.c_double),
        ("T_floor", C.c_double),
        ("sigma_s", C.c_double),
        ("tol_outer_e", C.c_double), ("tol_outer_E", C.c_double),
        ("tol_inner_e", C.c_double), ("tol_krylov", C.c_double),
        ("max_outer", C.c_int32), ("max_inner_e", C.c_int32), ("max_krylov", C.c_int32),
        ("precond", C.c_int32),
        ("precision", C.c_int32),
        ("cheb_degree", C.c_int32),
        ("amg_rebuild", C.c_int32),
        ("amg_theta", C.c_double),
        ("check_every", C.c_int32),
        ("kernel_timing", C.c_int32),
        ("autotune", C.c_int32),
        ("amg_tail", C.c_int32),
        ("coarse_fp32", C.c_int32),
        ("graphs", C.c_int32),
        ("pdl", C.c_int32),
        ("fine_post_smooth", C.c_int32),
        ("reliable_drop", C.c_double),
        ("dt_target", C.c_double), ("dt_growth", C.c_double), ("dt_min", C.c_double),
        ("dt_max", C.c_double), ("dt_eta_floor", C.c_double), ("cell_list", C.c_int32),
        ("index64", C.c_int32), ("krylov_start", C.c_int32),
        ("device", C.c_int32),
        ("stream", C.c_void_p),
    ]


class TuneTrial(C.Structure):
    """sph_rt_tune_trial."""
    _fields_ = [("fine_post_smooth", C.c_int32), ("cheb_degree", C.c_int32),
                ("reliable_drop", C.c_double), ("ms", C.c_double)]


class Stats(C.Structure):
    _fields_ = [
        ("outer_iters", C.c_int32),
        ("krylov_iters_total", C.c_int32),
        ("krylov_iters_per_outer", C.c_int32 * 64),
        ("newton_iters_max", C.c_int32),
        ("energy_before", C.c_double), ("energy_after", C.c_double),
        ("source_energy", C.c_double), ("boundary_energy", C.c_double),
        ("last_change_e", C.c_double), ("last_change_E", C.c_double),
        ("t_setup_ms", C.c_double), ("t_assembly_ms", C.c_double), ("t_amg_ms", C.c_double),
        ("t_krylov_ms", C.c_double), ("t_newton_ms", C.c_double),
        ("eta_e", C.c_double), ("eta_E", C.c_double), ("dt_next", C.c_double),
    ]

    def krylov_per_outer(self):
        return list(self.krylov_iters_per_outer[: self.outer_iters])


SRV_QUEUED, SRV_ADMITTED, SRV_RUNNING, SRV_DONE, SRV_FAILED = 0, 1, 2, 3, 4


class SrvConfig(C.Structure):
    _fields_ = [("workers", C.c_int32), ("max_resident", C.c_int32),
                ("steps_per_tick", C.c_int32), ("hbm_budget_bytes", C.c_double),
                ("device", C.c_int32), ("fuse_max_n", C.c_int64), ("fuse_max_k", C.c_int32)]


class SrvInfo(C.Structure):
    _fields_ = [("queued", C.c_int32), ("resident", C.c_int32), ("peak_resident", C.c_int32),
                ("resident_bytes", C.c_int64), ("peak_bytes", C.c_int64),
                ("particle_steps", C.c_int64), ("t_first_submit", C.c_double),
                ("t_last_done", C.c_double), ("fused_requests", C.c_int64),
                ("fused_batches", C.c_int64)]


class SphRtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

# (name, restype, argtypes) of every entry point in include/sph_rt.h
_P = C.c_void_p
_SIGNATURES = [
    ("sph_rt_default_config", None, [_P]),
    ("sph_rt_create", C.c_int, [_P, _P]),
    ("sph_rt_set_particles", C.c_int, [_P, C.c_int64] + [_P] * 9),
    ("sph_rt_set_particles_device", C.c_int, [_P, C.c_int64] + [_P] * 9),
    ("sph_rt_step", C.c_int, [_P, C.c_double, _P, _P, _P, _P, _P]),
    ("sph_rt_step_device", C.c_int, [_P, C.c_double, _P, _P, _P, _P, _P]),
    ("sph_rt_get_energies", C.c_int, [_P, _P, _P, _P]),
    ("sph_rt_get_history", C.c_int, [_P, _P, _P, _P]),
    ("sph_rt_extrapolation_weights", C.c_int, [C.c_int32, C.c_double, _P, _P]),
    ("sph_rt_set_history", C.c_int, [_P, C.c_int32, _P, _P]),
    ("sph_rt_get_energies_device", C.c_int, [_P, _P, _P]),
    ("sph_rt_get_sizes", C.c_int, [_P, _P, _P, _P]),
    ("sph_rt_adapt_smoothing_lengths", C.c_int, [_P, C.c_double, C.c_double, C.c_int32, _P]),
    ("sph_rt_get_smoothing_lengths", C.c_int, [_P, _P]),
    ("sph_rt_move_particles", C.c_int, [_P, _P]),
    ("sph_rt_move_particles_device", C.c_int, [_P, _P]),
    ("sph_rt_get_neighbors", C.c_int, [_P, _P, _P]),
    ("sph_rt_get_operator", C.c_int, [_P, _P, _P, _P, _P, _P]),
    ("sph_rt_get_properties", C.c_int, [_P] * 7),
    ("sph_rt_kernel_stats", C.c_int, [_P, _P, _P, _P, C.c_int]),
    ("sph_rt_get_amg_info", C.c_int, [_P, _P, _P, _P, C.c_int32]),
    ("sph_rt_loop_graph_info", C.c_int, [_P, _P, _P]),
    ("sph_rt_get_config", C.c_int, [_P, _P]),
    ("sph_rt_release_cached_memory", C.c_int, [C.c_int32]),
    ("sph_rt_get_solver_tuning", C.c_int, [_P, _P, C.c_int32, _P]),
    ("sph_rt_kernel_stats_kind", C.c_int, [_P, C.c_int32, _P, _P, _P]),
    ("sph_rt_launch_count", C.c_int64, [_P]),
    ("sph_rt_last_error", C.c_char_p, [_P]),
    ("sph_rt_destroy", None, [_P]),
    ("sph_rt_srv_default_config", None, [_P]),
    ("sph_rt_srv_create", C.c_int, [_P, _P]),
    ("sph_rt_srv_submit", C.c_int, [_P, _P, C.c_int64] + [_P] * 11 + [C.c_int32, C.c_double, _P]),
    ("sph_rt_srv_poll", C.c_int, [_P, C.c_int64, _P, _P]),
    ("sph_rt_srv_wait", C.c_int, [_P, C.c_int64]),
    ("sph_rt_srv_result", C.c_int, [_P, C.c_int64, _P, _P, _P, _P, C.c_int64]),
    ("sph_rt_srv_info", C.c_int, [_P, _P]),
    ("sph_rt_srv_destroy", None, [_P]),
    ("sph_rt_batch_create", C.c_int, [_P, _P]),
    ("sph_rt_batch_add", C.c_int, [_P, C.c_int64] + [_P] * 10),
    ("sph_rt_batch_add_many", C.c_int, [_P, C.c_int32, _P, C.c_int32, _P]),
    ("sph_rt_batch_set_sources", C.c_int, [_P, C.c_int32, _P, _P]),
    ("sph_rt_batch_step", C.c_int, [_P, C.c_double, _P, _P, _P, _P]),
    ("sph_rt_batch_run", C.c_int, [_P, C.c_double, C.c_int32, _P, _P, _P]),
    ("sph_rt_batch_set_shape", C.c_int, [_P, _P]),
    ("sph_rt_batch_get_shape", C.c_int, [_P, _P]),
    ("sph_rt_batch_autotune", C.c_int, [_P, C.c_double, _P, _P]),
    ("sph_rt_batch_get_energies", C.c_int, [_P, C.c_int32, _P, _P]),
    ("sph_rt_batch_problem_info", C.c_int, [_P, C.c_int32, _P]),
    ("sph_rt_batch_size", C.c_int32, [_P]),
    ("sph_rt_batch_last_error", C.c_char_p, [_P]),
    ("sph_rt_batch_destroy", None, [_P]),
]
# include/sph_rt_noalloc.h
_SIGNATURES_NOALLOC = [
    ("sph_rt_energy_totals_noalloc", C.c_int, [C.c_int64] + [_P] * 7),
]


# Largest n_total of sph_rt_energy_totals_noalloc (SPH_RT_NOALLOC_MAX_N in
# include/sph_rt_noalloc.h): 4096 thread blocks of 8192 particles.
NOALLOC_MAX_N = 4096 * 8192


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsphrt.so (building it first if needed).  Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libsphrt.so not found at {path}; run paper_2001_11606_gb300.build")
    L = C.CDLL(path)
    for name, res, args in _SIGNATURES + _SIGNATURES_NOALLOC:
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def energy_totals_noalloc(n_total, kind, mass, rho, e, E, totals, stream=0):
    """sph_rt_energy_totals_noalloc (include/sph_rt_noalloc.h) with raw DEVICE
    pointers (ints, e.g. torch's data_ptr(); 0 = NULL) and a cudaStream_t
    handle; returns the status code.  The reason of a failure is in
    last_thread_error()."""
    fn = load().sph_rt_energy_totals_noalloc
    ptrs = [C.c_void_p(p) if p else None for p in (kind, mass, rho, e, E, totals)]
    return fn(int(n_total), *ptrs, C.c_void_p(stream) if stream else None)


def last_thread_error() -> str:
    """Message of the last failed handle-less call on this thread."""
    return load().sph_rt_last_error(None).decode()


def exported_symbols():
    return [name for name, _, _ in _SIGNATURES]


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def default_config(**overrides) -> Config:
    cfg = Config()
    load().sph_rt_default_config(C.byref(cfg))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise AttributeError(k)
        setattr(cfg, k, v)
    return cfg


class Solver:
    """One handle of the library (see sph_rt.h for the semantics of each call)."""

    def __init__(self, cfg: Config | None = None, **overrides):
        self._L = load()
        cfg = cfg or default_config()
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        h = C.c_void_p()
        rc = self._L.sph_rt_create(C.byref(cfg), C.byref(h))
        if rc != OK:
            raise SphRtError(rc, self._L.sph_rt_last_error(None).decode())
        self._h = h
        self.n = 0

    # -- plumbing --------------------------------------------------------------
    def _check(self, rc):
        if rc != OK:
            raise SphRtError(rc, self.last_error())
        return rc

    def last_error(self) -> str:
        return self._L.sph_rt_last_error(self._h).decode()

    def close(self):
        if getattr(self, "_h", None):
            self._L.sph_rt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- C ABI -----------------------------------------------------------------
    def set_particles(self, pos, mass, rho, h, sigma0, kind, copy_of, e0, E0):
        pos = _f64(pos)
        n = pos.shape[0] if pos.ndim == 2 else pos.size // self.cfg.dim
        kind = np.ascontiguousarray(kind, dtype=np.int32)
        copy_of = None if copy_of is None else np.ascontiguousarray(copy_of, dtype=np.int64)
        arrs = [_f64(a, n) for a in (mass, rho, h, sigma0)]
        e0, E0 = _f64(e0, n), _f64(E0, n)
        rc = self._L.sph_rt_set_particles(self._h, n, _ptr(pos), *[_ptr(a) for a in arrs],
                                          _ptr(kind), _ptr(copy_of), _ptr(e0), _ptr(E0))
        self._check(rc)
        self.n = n
        return rc

    def set_particles_device(self, n, pos, mass, rho, h, sigma0, kind, copy_of, e0, E0):
        ptrs = [C.c_void_p(p) if p else None for p in (pos, mass, rho, h, sigma0, kind, copy_of,
                                                      e0, E0)]
        self._check(self._L.sph_rt_set_particles_device(self._h, int(n), *ptrs))
        self.n = int(n)

    def step(self, dt, Qe=None, QE=None, ghost_e=None, ghost_E=None, raise_on_error=True):
        st = Stats()
        arrs = [_f64(a, self.n) for a in (Qe, QE, ghost_e, ghost_E)]
        rc = self._L.sph_rt_step(self._h, float(dt), *[_ptr(a) for a in arrs], C.byref(st))
        if raise_on_error:
            self._check(rc)
        return rc, st

    def step_host_ptrs(self, dt, Qe=0, QE=0, ghost_e=0, ghost_E=0):
        """Step with raw HOST pointers (e.g. pinned torch tensors)."""
        st = Stats()
        ptrs = [C.c_void_p(p) if p else None for p in (Qe, QE, ghost_e, ghost_E)]
        self._check(self._L.sph_rt_step(self._h, float(dt), *ptrs, C.byref(st)))
        return st

    def step_device(self, dt, Qe=0, QE=0, ghost_e=0, ghost_E=0, raise_on_error=True):
        st = Stats()
        ptrs = [C.c_void_p(p) if p else None for p in (Qe, QE, ghost_e, ghost_E)]
        rc = self._L.sph_rt_step_device(self._h, float(dt), *ptrs, C.byref(st))
        if raise_on_error:
            self._check(rc)
        return rc, st

    def get_energies(self):
        e = np.empty(self.n)
        E = np.empty(self.n)
        tot = np.empty(2)
        self._check(self._L.sph_rt_get_energies(self._h, _ptr(e), _ptr(E), _ptr(tot)))
        return e, E, tot

    def get_history(self):
        """(E_hist, dt_hist): the extrapolated Krylov start's history, rows
        E^{n-2}, E^{n-3}, ... in caller order and their steps' dt, as many rows as
        the next step reads (0 after new particles or a failed step)."""
        E = np.zeros((3, self.n))
        dt = np.zeros(3)
        d = C.c_int32()
        self._check(self._L.sph_rt_get_history(self._h, C.byref(d), _ptr(E), _ptr(dt)))
        return E[:d.value].copy(), dt[:d.value].copy()

    def set_history(self, E_hist, dt_hist):
        E = np.ascontiguousarray(E_hist, dtype=np.float64).reshape(-1, self.n)
        dt = np.ascontiguousarray(dt_hist, dtype=np.float64).ravel()
        if dt.size != E.shape[0]:
            raise ValueError("one dt per history row")
        self._check(self._L.sph_rt_set_history(self._h, E.shape[0], _ptr(E), _ptr(dt)))

    def get_energies_host_ptrs(self, e_ptr, E_ptr):
        self._check(self._L.sph_rt_get_energies(self._h, C.c_void_p(e_ptr), C.c_void_p(E_ptr),
                                                None))

    def get_energies_device(self, e_ptr, E_ptr):
        self._check(self._L.sph_rt_get_energies_device(self._h, C.c_void_p(e_ptr) if e_ptr else None,
                                                       C.c_void_p(E_ptr) if E_ptr else None))

    def adapt_smoothing_lengths(self, eta=4.0, tol=1e-13, max_iter=100):
        """Smoothing lengths by the iteration of Sec. 3.1; returns the largest
        number of updates."""
        it = C.c_int32()
        self._check(self._L.sph_rt_adapt_smoothing_lengths(self._h, float(eta), float(tol),
                                                           int(max_iter), C.byref(it)))
        return it.value

    def get_smoothing_lengths(self):
        h = np.empty(self.n)
        self._check(self._L.sph_rt_get_smoothing_lengths(self._h, _ptr(h)))
        return h

    def move_particles(self, pos):
        pos = _f64(pos)
        if pos.size != self.n * self.cfg.dim:
            raise ValueError(f"expected {self.n * self.cfg.dim} coordinates, got {pos.size}")
        self._check(self._L.sph_rt_move_particles(self._h, _ptr(pos)))

    def move_particles_device(self, pos_ptr):
        self._check(self._L.sph_rt_move_particles_device(self._h, C.c_void_p(pos_ptr)))

    def sizes(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self._L.sph_rt_get_sizes(self._h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def get_neighbors(self):
        rowptr = np.zeros(self.n + 1, dtype=np.int64)
        self._check(self._L.sph_rt_get_neighbors(self._h, _ptr(rowptr), None))
        cols = np.zeros(max(int(rowptr[-1]), 1), dtype=np.int64)
        self._check(self._L.sph_rt_get_neighbors(self._h, _ptr(rowptr), _ptr(cols)))
        return rowptr, cols[: rowptr[-1]]

    def get_operator(self):
        _, _, nnz = self.sizes()
        rowptr = np.zeros(self.n + 1, dtype=np.int64)
        cols = np.zeros(max(nnz, 1), dtype=np.int64)
        vals = np.zeros(max(nnz, 1))
        diag = np.zeros(self.n)
        gb = np.zeros(self.n)
        self._check(self._L.sph_rt_get_operator(self._h, _ptr(rowptr), _ptr(cols), _ptr(vals),
                                                _ptr(diag), _ptr(gb)))
        return rowptr, cols[:nnz], vals[:nnz], diag, gb

    def get_properties(self):
        out = {k: np.zeros(self.n) for k in ("T", "sigma", "f", "R", "lambda", "D")}
        self._check(self._L.sph_rt_get_properties(self._h, *[_ptr(out[k]) for k in
                                                             ("T", "sigma", "f", "R", "lambda",
                                                              "D")]))
        return out

    def kernel_stats(self, reset=False):
        n, ms, by = C.c_int64(), C.c_double(), C.c_double()
        self._check(self._L.sph_rt_kernel_stats(self._h, C.byref(n), C.byref(ms), C.byref(by),
                                                int(reset)))
        return n.value, ms.value, by.value

    def kernel_stats_by_kind(self):
        """{name: (launches, ms, bytes)} of the timed fine-operator kernels."""
        out = {}
        for kind, name in ((0, "spmv_pq"), (1, "resid"), (2, "cheb_step"), (3, "post_ap"),
                           (4, "true_resid")):
            n, ms, by = C.c_int64(), C.c_double(), C.c_double()
            self._check(self._L.sph_rt_kernel_stats_kind(self._h, kind, C.byref(n), C.byref(ms),
                                                         C.byref(by)))
            out[name] = (n.value, ms.value, by.value)
        return out

    def amg_info(self):
        nl = C.c_int32()
        rows = np.zeros(16, dtype=np.int64)
        nnz = np.zeros(16, dtype=np.int64)
        self._check(self._L.sph_rt_get_amg_info(self._h, C.byref(nl), _ptr(rows), _ptr(nnz), 16))
        k = min(nl.value, 16)
        return list(zip(rows[:k].tolist(), nnz[:k].tolist()))

    def launch_count(self) -> int:
        return int(self._L.sph_rt_launch_count(self._h))

    def loop_graph_info(self):
        """(captures, launches) of the device-driven outer-loop graph."""
        cap, lau = C.c_int64(), C.c_int64()
        self._check(self._L.sph_rt_loop_graph_info(self._h, C.byref(cap), C.byref(lau)))
        return cap.value, lau.value

    def get_config(self) -> "Config":
        """The handle's configuration as it stands (the autotuner's choice included)."""
        cfg = Config()
        self._check(self._L.sph_rt_get_config(self._h, C.byref(cfg)))
        return cfg

    def solver_tuning(self):
        """Trials of the solver autotuner: [(fine_post_smooth, cheb_degree,
        reliable_drop, ms or None if the step did not converge)]."""
        cnt = C.c_int32()
        self._check(self._L.sph_rt_get_solver_tuning(self._h, None, 0, C.byref(cnt)))
        arr = (TuneTrial * max(cnt.value, 1))()
        self._check(self._L.sph_rt_get_solver_tuning(self._h, arr, cnt.value, C.byref(cnt)))
        return [(t.fine_post_smooth, t.cheb_degree, t.reliable_drop,
                 t.ms if t.ms >= 0 else None) for t in arr[: cnt.value]]


def release_cached_memory(device: int = 0) -> None:
    """Return the library's cache of freed device buffers of `device` to CUDA."""
    rc = load().sph_rt_release_cached_memory(int(device))
    if rc != OK:
        raise SphRtError(rc, "sph_rt_release_cached_memory")


def config_from_params(params: dict, **overrides) -> Config:
    """Config from a workload parameter dict (inputs.Workload.params)."""
    cfg = default_config()
    for k, v in params.items():
        if hasattr(cfg, k):
            setattr(cfg, k, v)
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def solver_for(workload, **overrides) -> Solver:
    """Solver with the workload's particles set (host arrays)."""
    P = workload.particles
    S = Solver(config_from_params(workload.params, **overrides))
    S.set_particles(P.pos, P.mass, P.rho, P.h, P.sigma0, P.kind,
                    P.copy_of if np.any(P.kind == COPY) else None, workload.e0, workload.E0)
    return S


class Server:
    """Continuous-batching request loop (sph_rt_srv_* in sph_rt.h)."""

    def __init__(self, **overrides):
        self._L = load()
        cfg = SrvConfig()
        self._L.sph_rt_srv_default_config(C.byref(cfg))
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        h = C.c_void_p()
        rc = self._L.sph_rt_srv_create(C.byref(cfg), C.byref(h))
        if rc != OK:
            raise SphRtError(rc, "sph_rt_srv_create failed")
        self._h = h
        self._n = {}

    def submit(self, cfg: Config, particles, e0, E0, steps: int, dt: float, Qe=None, QE=None):
        P = particles
        n = P.pos.shape[0]
        pos = _f64(P.pos)
        arrs = [_f64(a, n) for a in (P.mass, P.rho, P.h, P.sigma0)]
        kind = np.ascontiguousarray(P.kind, dtype=np.int32)
        copy_of = (np.ascontiguousarray(P.copy_of, dtype=np.int64)
                   if np.any(kind == COPY) else None)
        e0, E0 = _f64(e0, n), _f64(E0, n)
        Qe, QE = _f64(Qe, n), _f64(QE, n)
        rid = C.c_int64()
        rc = self._L.sph_rt_srv_submit(self._h, C.byref(cfg), n, _ptr(pos),
                                       *[_ptr(a) for a in arrs], _ptr(kind), _ptr(copy_of),
                                       _ptr(e0), _ptr(E0), _ptr(Qe), _ptr(QE), int(steps),
                                       float(dt), C.byref(rid))
        if rc != OK:
            raise SphRtError(rc, "sph_rt_srv_submit failed")
        self._n[rid.value] = n
        return rid.value

    def poll(self, rid):
        st = C.c_int32()
        t = np.zeros(3)
        rc = self._L.sph_rt_srv_poll(self._h, int(rid), C.byref(st), _ptr(t))
        if rc != OK:
            raise SphRtError(rc, "unknown request")
        return st.value, t

    def wait(self, rid):
        return self._L.sph_rt_srv_wait(self._h, int(rid))

    def result(self, rid):
        n = self._n[rid]
        e = np.empty(n)
        E = np.empty(n)
        st = Stats()
        msg = C.create_string_buffer(512)
        rc = self._L.sph_rt_srv_result(self._h, int(rid), _ptr(e), _ptr(E), C.byref(st), msg, 512)
        if rc != OK:
            raise SphRtError(rc, msg.value.decode())
        return e, E, st

    def info(self):
        inf = SrvInfo()
        self._L.sph_rt_srv_info(self._h, C.byref(inf))
        return inf

    def close(self):
        if getattr(self, "_h", None):
            self._L.sph_rt_srv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Problem(C.Structure):
    """sph_rt_problem (arrays as for sph_rt_batch_add)."""
    _fields_ = [("n_total", C.c_int64)] + [(f, C.c_void_p) for f in
                                           ("pos", "mass", "rho", "h", "sigma0", "kind",
                                            "copy_of", "e0", "E0")]


class BatchShape(C.Structure):
    """sph_rt_batch_shape."""
    _fields_ = [("lanes_per_row", C.c_int32), ("cheb_degree", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("rows_per_cta", C.c_int32)]


class Batch:
    """Many small problems, one kernel launch per step (sph_rt_batch_* in sph_rt.h)."""

    def __init__(self, cfg: Config):
        self._L = load()
        h = C.c_void_p()
        rc = self._L.sph_rt_batch_create(C.byref(cfg), C.byref(h))
        if rc != OK:
            raise SphRtError(rc, self._L.sph_rt_last_error(None).decode())
        self._h = h
        self._n = []

    def _check(self, rc):
        if rc != OK:
            raise SphRtError(rc, self._L.sph_rt_batch_last_error(self._h).decode())
        return rc

    def add(self, particles, e0, E0):
        P = particles
        n = P.pos.shape[0]
        arrs = [_f64(a, n) for a in (P.mass, P.rho, P.h, P.sigma0)]
        kind = np.ascontiguousarray(P.kind, dtype=np.int32)
        copy_of = (np.ascontiguousarray(P.copy_of, dtype=np.int64)
                   if np.any(kind == COPY) else None)
        idx = C.c_int32()
        self._check(self._L.sph_rt_batch_add(self._h, n, _ptr(_f64(P.pos)), *[_ptr(a) for a in arrs],
                                             _ptr(kind), _ptr(copy_of), _ptr(_f64(e0, n)),
                                             _ptr(_f64(E0, n)), C.byref(idx)))
        self._n.append(n)
        return idx.value

    def add_many(self, problems, threads=1):
        """Add [(particles, e0, E0)] with their set-ups on `threads` host threads;
        returns the first index (problem k gets first + k)."""
        keep = []
        arr = (Problem * max(len(problems), 1))()
        for k, (P, e0, E0) in enumerate(problems):
            n = P.pos.shape[0]
            a = dict(pos=_f64(P.pos), mass=_f64(P.mass, n), rho=_f64(P.rho, n), h=_f64(P.h, n),
                     sigma0=_f64(P.sigma0, n), kind=np.ascontiguousarray(P.kind, dtype=np.int32),
                     copy_of=(np.ascontiguousarray(P.copy_of, dtype=np.int64)
                              if np.any(P.kind == COPY) else None),
                     e0=_f64(e0, n), E0=_f64(E0, n))
            keep.append(a)
            arr[k].n_total = n
            for f, v in a.items():
                setattr(arr[k], f, None if v is None else v.ctypes.data)
        first = C.c_int32()
        self._check(self._L.sph_rt_batch_add_many(self._h, len(problems), arr, int(threads),
                                                  C.byref(first)))
        self._n.extend(P.pos.shape[0] for P, _, _ in problems)
        return first.value

    def set_sources(self, index, Qe=None, QE=None):
        n = self._n[index]
        self._check(self._L.sph_rt_batch_set_sources(self._h, int(index), _ptr(_f64(Qe, n)),
                                                     _ptr(_f64(QE, n))))

    def step(self, dt, raise_on_error=True):
        K = len(self._n)
        st = np.zeros(K, dtype=np.int32)
        ou = np.zeros(K, dtype=np.int32)
        kr = np.zeros(K, dtype=np.int32)
        en = np.zeros(4 * K)
        rc = self._L.sph_rt_batch_step(self._h, float(dt), _ptr(st), _ptr(ou), _ptr(kr), _ptr(en))
        if raise_on_error:
            self._check(rc)
        return rc, st, ou, kr, en.reshape(K, 4)

    def run(self, dt, steps, raise_on_error=True):
        """`steps` steps of every problem in one CUDA-graph launch."""
        K = len(self._n)
        st = np.zeros(K, dtype=np.int32)
        ou = np.zeros(K, dtype=np.int32)
        kr = np.zeros(K, dtype=np.int32)
        rc = self._L.sph_rt_batch_run(self._h, float(dt), int(steps), _ptr(st), _ptr(ou),
                                      _ptr(kr))
        if raise_on_error:
            self._check(rc)
        return rc, st, ou, kr

    def set_shape(self, lanes_per_row, cheb_degree, blocks_per_sm=1, rows_per_cta=4096):
        """Lanes per row (1, 2, 4, 8), Chebyshev degree (1..16), resident blocks
        per SM (1, 2) and rows per CTA (0 = one block per problem, else >= 64) of
        the batched launch."""
        sh = BatchShape(int(lanes_per_row), int(cheb_degree), int(blocks_per_sm),
                        int(rows_per_cta))
        self._check(self._L.sph_rt_batch_set_shape(self._h, C.byref(sh)))

    def get_shape(self):
        """(lanes_per_row, cheb_degree, blocks_per_sm, rows_per_cta)."""
        sh = BatchShape()
        self._check(self._L.sph_rt_batch_get_shape(self._h, C.byref(sh)))
        return sh.lanes_per_row, sh.cheb_degree, sh.blocks_per_sm, sh.rows_per_cta

    def autotune(self, dt):
        """Time one step per candidate shape (the state does not advance); returns the
        chosen (lanes_per_row, cheb_degree, blocks_per_sm, rows_per_cta) and
        {shape: ms, or None if some problem did not converge}."""
        t = np.zeros(BATCH_TUNE_CANDIDATES, dtype=np.float32)
        sh = BatchShape()
        rows0 = self.get_shape()[3]
        self._check(self._L.sph_rt_batch_autotune(self._h, float(dt), _ptr(t), C.byref(sh)))
        table = {}
        c = 0
        best = None
        for b in BATCH_TUNE_BLOCKS:
            for w in BATCH_TUNE_LANES:
                for g in BATCH_TUNE_DEGREES:
                    ms = float(t[c])
                    table[(w, g, b, rows0)] = ms if ms >= 0 else None
                    if ms >= 0 and (best is None or ms < best[0]):
                        best = (ms, w, g, b)
                    c += 1
        if best is not None:
            for r in BATCH_TUNE_ROWS:
                ms = float(t[c])
                key = (best[1], best[2], best[3], r)
                if key not in table or table[key] is None or (ms >= 0 and ms < table[key]):
                    table[key] = ms if ms >= 0 else None
                c += 1
        chosen = (sh.lanes_per_row, sh.cheb_degree, sh.blocks_per_sm, sh.rows_per_cta)
        return chosen, table

    def problem_info(self, index):
        """{n_total, n_interior, nnz_operator, nnz_neighbours, cluster} of one problem
        (cluster: blocks it runs on with the current shape)."""
        a = np.zeros(5, dtype=np.int64)
        self._check(self._L.sph_rt_batch_problem_info(self._h, int(index), _ptr(a)))
        return dict(n_total=int(a[0]), n_interior=int(a[1]), nnz_operator=int(a[2]),
                    nnz_neighbours=int(a[3]), cluster=int(a[4]))

    def get_energies(self, index):
        n = self._n[index]
        e = np.empty(n)
        E = np.empty(n)
        self._check(self._L.sph_rt_batch_get_energies(self._h, int(index), _ptr(e), _ptr(E)))
        return e, E

    def close(self):
        if getattr(self, "_h", None):
            self._L.sph_rt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def extrapolation_weights(order, dt, dt_hist=()):
    """Weights of the extrapolated Krylov start: sum_j w[j] E^{n-1-j} is the value
    at t_{n-1} + dt of the polynomial of degree `order` through the last states;
    dt_hist holds the previous steps' sizes, newest first."""
    w = np.zeros(order + 1 if 0 <= order <= 3 else 1)
    d = np.ascontiguousarray(dt_hist, dtype=np.float64)
    if d.size < order:
        raise ValueError("need one previous step size per order")
    rc = load().sph_rt_extrapolation_weights(int(order), float(dt), _ptr(d) if d.size else None,
                                             _ptr(w))
    if rc:
        raise SphRtError(rc, "invalid order or step sizes")
    return w
