"""ctypes front end of the plain FP64 CPU oracle (sph_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg are the only users.  The product library never imports this
package, and this package never imports the product library.

`build()` compiles sph_oracle.c with gcc (-O2 -ffp-contract=off -fopenmp) into
oracle/_build/; the functions below marshal numpy arrays into the C calls.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libsph_oracle.so")
_lock = threading.Lock()
_lib = None


class Params(C.Structure):
    _fields_ = [
        ("dim", C.c_int32),
        ("a", C.c_double), ("c", C.c_double), ("cv", C.c_double),
        ("limiter", C.c_int32),
        ("larsen_k", C.c_double),
        ("opacity_exp", C.c_double),
        ("T_floor", C.c_double),
        ("tol_outer_e", C.c_double), ("tol_outer_E", C.c_double),
        ("tol_inner_e", C.c_double), ("tol_krylov", C.c_double),
        ("max_outer", C.c_int32), ("max_inner_e", C.c_int32), ("max_krylov", C.c_int32),
        ("kernel", C.c_int32),
        ("sigma_s", C.c_double),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("outer_iters", C.c_int32),
        ("krylov_total", C.c_int32),
        ("krylov_per_outer", C.c_int32 * 64),
        ("newton_max", C.c_int32),
        ("status", C.c_int32),
        ("energy_before", C.c_double), ("energy_after", C.c_double),
        ("source_energy", C.c_double), ("boundary_energy", C.c_double),
        ("last_change_e", C.c_double), ("last_change_E", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            i64, i32, dbl = C.c_int64, C.c_int, C.c_double
            L.orc_kernel.argtypes = [i32, dbl, dbl, P, P]
            L.orc_kernel_c4.argtypes = [i32, dbl, dbl, P, P]
            L.orc_neighbors.argtypes = [i64, i32, P, P, P, i32, i32, P, P]
            L.orc_neighbors.restype = i64
            L.orc_neighbors_rows.argtypes = [i64, i32, P, P, i32, i64, P, P, P]
            L.orc_neighbors_rows.restype = i64
            L.orc_properties.argtypes = [P, i64, P, P, P, P, P, P, P, P, P, dbl, P, P,
                                         P, P, P, P, P, P]
            L.orc_assemble.argtypes = [P, i64, P, P, P, P, P, P, dbl, P, P, P, P, P, P,
                                       P, P, P, P, P]
            L.orc_assemble.restype = i64
            L.orc_material_solve.argtypes = [P, i64, P, P, P, dbl, P, P, P, P]
            L.orc_material_solve.restype = i32
            L.orc_cg.argtypes = [i64, P, P, P, P, P, P, P, P, dbl, i32, P]
            L.orc_cg.restype = i32
            L.orc_step.argtypes = [P, i64, P, P, P, P, P, P, P, P, P, dbl, P, P, P, P, P, P, P]
            L.orc_step.restype = i32
            L.orc_totals.argtypes = [i64, P, P, P, P, P, P]
            L.orc_smoothing_lengths.argtypes = [P, i64, P, P, P, dbl, dbl, i32, P]
            L.orc_smoothing_lengths.restype = i32
            L.orc_limiter.argtypes = [P, dbl]
            L.orc_limiter.restype = dbl
            L.orc_num_threads.restype = i32
            L.orc_set_threads.argtypes = [i32]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def make_params(**kw) -> Params:
    p = Params()
    defaults = dict(dim=3, a=1.0, c=1.0, cv=1.0, limiter=0, larsen_k=2.0, opacity_exp=0.0,
                    T_floor=0.0, tol_outer_e=1e-8, tol_outer_E=1e-8, tol_inner_e=1e-13,
                    tol_krylov=1e-12, max_outer=50, max_inner_e=50, max_krylov=5000, kernel=0,
                    sigma_s=0.0)
    defaults.update(kw)
    for k, v in defaults.items():
        setattr(p, k, v)
    return p


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def kernel(dim: int, r: float, h: float, kern: int = 0):
    """(W, dW/dr) of the M4 cubic B-spline (kern 0, support 2h) or the Wendland
    C4 kernel (kern 1, support h; Sec. 2.4)."""
    W, dW = C.c_double(), C.c_double()
    fn = lib().orc_kernel_c4 if kern == 1 else lib().orc_kernel
    fn(dim, float(r), float(h), C.byref(W), C.byref(dW))
    return W.value, dW.value


def limiter(R: float, limiter: int, larsen_k: float = 2.0) -> float:
    """Flux limiter lambda(R) (Sec. 2.1): 0 none (1/3), 1 Levermore, 2 Larsen(k)."""
    p = make_params(limiter=int(limiter), larsen_k=float(larsen_k))
    return float(lib().orc_limiter(C.byref(p), float(R)))


def smoothing_lengths(particles, params: dict, eta: float = 4.0, tol: float = 1e-13,
                      max_iter: int = 100):
    """Smoothing lengths by the initialisation iteration of Sec. 3.1 (support
    radius = eta local point spacings), starting from particles.h.  Returns
    (h, largest number of updates)."""
    P = particles
    prm = make_params(**params)
    pos = _f64(P.pos)
    h = _f64(P.h).copy()
    kind = np.ascontiguousarray(P.kind, dtype=np.int32)
    copy_of = np.ascontiguousarray(P.copy_of, dtype=np.int64)
    it = lib().orc_smoothing_lengths(C.byref(prm), pos.shape[0], _p(pos), _p(kind), _p(copy_of),
                                     float(eta), float(tol), int(max_iter), _p(h))
    return h, int(it)


def neighbors(pos, h, kind, brute: bool = False, kernel: int = 0):
    """Neighbour CSR over all particles in caller order: (rowptr int64, cols int32).
    kernel 0: support 2h (M4); 1: support h (Wendland C4)."""
    pos = _f64(pos)
    n, dim = pos.shape
    h = _f64(h)
    kind = np.ascontiguousarray(kind, dtype=np.int32)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    L = lib()
    L.orc_neighbors(n, dim, _p(pos), _p(h), _p(kind), int(brute), int(kernel), _p(rowptr), None)
    cols = np.zeros(max(int(rowptr[-1]), 1), dtype=np.int32)
    L.orc_neighbors(n, dim, _p(pos), _p(h), _p(kind), int(brute), int(kernel), _p(rowptr),
                    _p(cols))
    return rowptr, cols[: rowptr[-1]]


def neighbors_of_rows(pos, h, rows, kernel: int = 0):
    """Brute-force neighbour lists (caller IDs, ascending) of the given rows."""
    pos = _f64(pos)
    n, dim = pos.shape
    h = _f64(h)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    L = lib()
    L.orc_neighbors_rows(n, dim, _p(pos), _p(h), int(kernel), len(rows), _p(rows), _p(rp), None)
    cols = np.zeros(max(int(rp[-1]), 1), dtype=np.int32)
    L.orc_neighbors_rows(n, dim, _p(pos), _p(h), int(kernel), len(rows), _p(rows), _p(rp),
                         _p(cols))
    return rp, cols[: rp[-1]]


class Problem:
    """Particle data plus neighbour lists, in caller order."""

    def __init__(self, particles, params: dict, brute: bool = False, nbrs=None):
        P = particles
        self.P = P
        self.params = make_params(**params)
        self.pos = _f64(P.pos)
        self.mass = _f64(P.mass)
        self.rho = _f64(P.rho)
        self.h = _f64(P.h)
        self.sigma0 = _f64(P.sigma0)
        self.kind = np.ascontiguousarray(P.kind, dtype=np.int32)
        self.copy_of = np.ascontiguousarray(P.copy_of, dtype=np.int64)
        self.n = self.pos.shape[0]
        if nbrs is None:
            nbrs = neighbors(self.pos, self.h, self.kind, brute=brute,
                             kernel=self.params.kernel)
        self.rowptr, self.cols = nbrs

    def properties(self, e, E, dt):
        n = self.n
        out = {k: np.zeros(n) for k in ("T", "sigma", "f", "R", "lambda", "D")}
        e, E = _f64(e), _f64(E)
        lib().orc_properties(C.byref(self.params), n, _p(self.pos), _p(self.mass), _p(self.rho),
                             _p(self.h), _p(self.sigma0), _p(self.kind), _p(self.copy_of),
                             _p(e), _p(E), float(dt), _p(self.rowptr), _p(self.cols),
                             *[_p(out[k]) for k in ("T", "sigma", "f", "R", "lambda", "D")])
        return out

    def assemble(self, props, dt, E_ghost):
        """Diffusion operator rows: (arow, acol, aval, adiag, gb) in caller order."""
        n = self.n
        nnz = max(int(self.rowptr[-1]), 1)
        arow = np.zeros(n + 1, dtype=np.int64)
        acol = np.zeros(nnz, dtype=np.int32)
        aval = np.zeros(nnz)
        adiag = np.zeros(n)
        gb = np.zeros(n)
        E_ghost = _f64(E_ghost)
        m = lib().orc_assemble(C.byref(self.params), n, _p(self.pos), _p(self.mass), _p(self.rho),
                               _p(self.h), _p(self.kind), _p(self.copy_of), float(dt),
                               _p(props["sigma"]), _p(props["f"]), _p(props["D"]), _p(E_ghost),
                               _p(self.rowptr), _p(self.cols), _p(arow), _p(acol), _p(aval),
                               _p(adiag), _p(gb))
        return arow, acol[:m], aval[:m], adiag, gb

    def material_solve(self, sigma, dt, e_old, P, e):
        e = _f64(e).copy()
        fails = C.c_int64()
        it = lib().orc_material_solve(C.byref(self.params), self.n, _p(self.kind), _p(self.rho),
                                      _p(_f64(sigma)), float(dt), _p(_f64(e_old)), _p(_f64(P)),
                                      _p(e), C.byref(fails))
        return e, int(it), int(fails.value)

    def cg(self, arow, acol, aval, adiag, b, x0, tol, maxit=5000):
        x = _f64(x0).copy()
        V = self.mass / self.rho
        rr = C.c_double()
        it = lib().orc_cg(self.n, _p(self.kind), _p(V), _p(arow), _p(acol), _p(aval), _p(adiag),
                          _p(_f64(b)), _p(x), float(tol), int(maxit), C.byref(rr))
        return x, int(it), rr.value

    def step(self, e, E, dt, Qe=None, QE=None, ghost_e=None, ghost_E=None):
        """One backward-Euler step; returns (status, e_new, E_new, stats)."""
        e = _f64(e).copy()
        E = _f64(E).copy()
        st = Stats()
        rc = lib().orc_step(C.byref(self.params), self.n, _p(self.pos), _p(self.mass),
                            _p(self.rho), _p(self.h), _p(self.sigma0), _p(self.kind),
                            _p(self.copy_of), _p(self.rowptr), _p(self.cols), float(dt),
                            _p(_f64(Qe)), _p(_f64(QE)), _p(_f64(ghost_e)), _p(_f64(ghost_E)),
                            _p(e), _p(E), C.byref(st))
        return int(rc), e, E, st

    def totals(self, e, E):
        out = np.zeros(2)
        lib().orc_totals(self.n, _p(self.kind), _p(self.mass), _p(self.rho), _p(_f64(e)),
                         _p(_f64(E)), _p(out))
        return out


def run(workload, steps: int | None = None, brute: bool = False, params: dict | None = None,
        problem: Problem | None = None):
    """Run `steps` steps of a workload from its initial state; returns (e, E, stats list)."""
    prm = dict(workload.params)
    if params:
        prm.update(params)
    pb = problem or Problem(workload.particles, prm, brute=brute)
    e, E = workload.e0.copy(), workload.E0.copy()
    stats = []
    for n in range(1, (steps if steps is not None else workload.steps) + 1):
        Qe, QE, ge, gE = workload.step_inputs(n)
        rc, e, E, st = pb.step(e, E, workload.dt, Qe, QE, ge, gE)
        if rc != 0:
            raise RuntimeError(f"oracle step {n} did not converge (status {rc})")
        stats.append(st)
    return e, E, stats


def fractional_change(x_new, x_old, V, target, interior, floor=1e-15):
    """Fractional energy change over a step (Sec. 3.3, Eq. energy-fractional):
    eta = max_i |x_i^n - x_i^{n-1}| / (x_i^n + target * xbar^n), where
    xbar^n = sum_i x_i^n V_i / sum_i V_i is the volume average over the
    interior particles.  `floor` is added to the denominator, as the paper
    suggests, for a state whose energy may be zero everywhere."""
    m = np.asarray(interior, dtype=bool)
    xn = np.asarray(x_new, dtype=np.float64)[m]
    xo = np.asarray(x_old, dtype=np.float64)[m]
    v = np.asarray(V, dtype=np.float64)[m]
    xbar = float(np.sum(xn * v) / np.sum(v))
    return float(np.max(np.abs(xn - xo) / (xn + target * xbar + floor)))


def next_dt(e_new, e_old, E_new, E_old, V, interior, dt, target=0.05, growth=10.0,
            dt_min=0.0, dt_max=np.inf):
    """Time step for the next step (Sec. 3.3): dt_x = dt (target / eta_x)^(1/2) for
    the material energy e and the radiation energy E, the more restrictive of
    the two, at most `growth` times the current step (the infinite-medium runs
    of Sec. 4.1 allow an order of magnitude per step), within [dt_min, dt_max].
    Returns (dt_next, eta_e, eta_E)."""
    eta_e = fractional_change(e_new, e_old, V, target, interior)
    eta_E = fractional_change(E_new, E_old, V, target, interior)
    cand = [dt * (target / eta) ** 0.5 if eta > 0.0 else np.inf for eta in (eta_e, eta_E)]
    dt_next = min(min(cand), growth * dt, dt_max)
    return max(dt_next, dt_min), eta_e, eta_E
