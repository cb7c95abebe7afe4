"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol declared in include/sph_rt.h, and rejects invalid input on the host
before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2001_11606_gb300 import inputs as I
from paper_2001_11606_gb300 import sphrt

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include")
HEADER = os.path.join(INCLUDE, "sph_rt.h")


def declared_functions(path=HEADER):
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_rt_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = sphrt.load()
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L, name), name
    assert sorted(sphrt.exported_symbols()) == names
    # every other public header's entry points are exported too
    for h in sorted(os.listdir(INCLUDE)):
        if h.endswith(".h"):
            for name in declared_functions(os.path.join(INCLUDE, h)):
                assert hasattr(L, name), (h, name)


def test_max_outer_beyond_recorded_stats_is_allowed():
    # the stats record the first 64 outer iterations; the limit itself is larger
    S = sphrt.Solver(sphrt.default_config(max_outer=1000))
    S.close()


def test_config_struct_matches_defaults():
    cfg = sphrt.default_config()
    assert cfg.dim == 3 and cfg.a == 1.0 and cfg.precond == sphrt.PRECOND_AMG
    assert cfg.amg_theta == 0.02 and cfg.cheb_degree == 1 and cfg.graphs == 1 and cfg.pdl == 1
    assert cfg.amg_tail == 0 and cfg.autotune == 0
    assert cfg.tol_outer_e == 1e-8 and cfg.tol_krylov == 1e-12 and cfg.tol_inner_e == 1e-13


@pytest.mark.parametrize("field,value", [("dim", 4), ("cv", 0.0), ("a", -1.0), ("limiter", 7),
                                         ("tol_krylov", -1.0), ("max_outer", 0),
                                         ("precond", 9), ("cheb_degree", 0),
                                         ("amg_theta", 1.5), ("graphs", 2), ("pdl", 2),
                                         ("amg_tail", -1), ("coarse_fp32", 2),
                                         ("fine_post_smooth", 2), ("reliable_drop", 0.0),
                                         ("reliable_drop", 1.0), ("dt_target", -0.1),
                                         ("dt_growth", 0.5), ("dt_min", -1.0),
                                         ("dt_max", 0.0), ("dt_eta_floor", -1.0),
                                         ("cell_list", 3), ("cell_list", -1),
                                         ("index64", 2), ("autotune", 3),
                                         ("krylov_start", 4)])
def test_create_rejects_bad_config(field, value):
    cfg = sphrt.default_config(**{field: value})
    with pytest.raises(sphrt.SphRtError) as ei:
        sphrt.Solver(cfg)
    assert ei.value.status == sphrt.EINVAL
    assert str(ei.value)


def test_vcycle_product_cg_needs_degree_one():
    with pytest.raises(sphrt.SphRtError) as ei:
        sphrt.Solver(sphrt.default_config(fine_post_smooth=0, cheb_degree=2))
    assert ei.value.status == sphrt.EINVAL and "cheb_degree" in str(ei.value)


def _particles():
    return I.make_lattice(2, (4, 4), 0.25, seed=1)


@pytest.mark.parametrize("mutate,msg", [
    (lambda P, e, E: P.mass.__setitem__(3, -1.0), "mass"),
    (lambda P, e, E: P.h.__setitem__(0, 0.0), "mass, rho and h"),
    (lambda P, e, E: P.pos.__setitem__((2, 1), np.nan), "position"),
    (lambda P, e, E: P.kind.__setitem__(5, 9), "kind"),
    (lambda P, e, E: P.sigma0.__setitem__(1, -2.0), "sigma0"),
    (lambda P, e, E: E.__setitem__(4, np.inf), "initial energy"),
])
def test_set_particles_rejects_bad_input_on_host(mutate, msg):
    P = _particles()
    e = np.ones(P.n)
    E = np.ones(P.n)
    mutate(P, e, E)
    S = sphrt.Solver(sphrt.default_config(dim=2))
    with pytest.raises(sphrt.SphRtError) as ei:
        S.set_particles(P.pos, P.mass, P.rho, P.h, P.sigma0, P.kind, None, e, E)
    assert ei.value.status == sphrt.EINVAL and msg in str(ei.value)
    S.close()


def test_copy_ghost_must_point_at_interior():
    P = I.make_lattice(2, (4, 4), 0.25, seed=1, faces=[("reflect", "reflect")] * 2)
    c = np.flatnonzero(P.kind == sphrt.COPY)[0]
    bad = P.copy_of.copy()
    bad[c] = c  # a ghost, not an interior particle
    S = sphrt.Solver(sphrt.default_config(dim=2))
    with pytest.raises(sphrt.SphRtError) as ei:
        S.set_particles(P.pos, P.mass, P.rho, P.h, P.sigma0, P.kind, bad, np.ones(P.n),
                        np.ones(P.n))
    assert "copy_of" in str(ei.value)
    with pytest.raises(sphrt.SphRtError):
        S.set_particles(P.pos, P.mass, P.rho, P.h, P.sigma0, P.kind, None, np.ones(P.n),
                        np.ones(P.n))
    S.close()


def test_step_before_particles_is_a_state_error():
    S = sphrt.Solver(sphrt.default_config(dim=2))
    with pytest.raises(sphrt.SphRtError) as ei:
        S.step(1e-3)
    assert ei.value.status == sphrt.ESTATE
    S.close()


def test_no_interior_particle():
    P = _particles()
    kind = np.full(P.n, sphrt.DIRICHLET, dtype=np.int32)
    S = sphrt.Solver(sphrt.default_config(dim=2))
    with pytest.raises(sphrt.SphRtError) as ei:
        S.set_particles(P.pos, P.mass, P.rho, P.h, P.sigma0, kind, None, np.ones(P.n),
                        np.ones(P.n))
    assert "interior" in str(ei.value)
    S.close()


@pytest.mark.parametrize("shape", [(3, 1, 1, 0), (16, 1, 1, 0), (0, 1, 1, 0), (4, 0, 1, 0),
                                   (4, 17, 1, 0), (4, 2, 0, 0), (4, 2, 3, 0), (4, 2, 1, -1),
                                   (4, 2, 1, 63)])
def test_batch_rejects_bad_shape(shape):
    B = sphrt.Batch(sphrt.default_config())
    with pytest.raises(sphrt.SphRtError) as ex:
        B.set_shape(*shape)
    assert ex.value.status == sphrt.EINVAL
    B.set_shape(2, 6, 2, 2048)
    assert B.get_shape() == (2, 6, 2, 2048)
    B.close()


def test_batch_tune_table_matches_header():
    src = open(HEADER).read()
    m = re.search(r"#define SPH_RT_BATCH_TUNE_CANDIDATES (\d+)", src)
    assert m and int(m.group(1)) == sphrt.BATCH_TUNE_CANDIDATES == 44


def test_release_cached_memory_needs_no_handle():
    sphrt.release_cached_memory(0)  # nothing cached in this process: no device call
    with pytest.raises(sphrt.SphRtError):
        sphrt.release_cached_memory(-1)


def test_extrapolation_weights_reproduce_polynomials():
    # the Krylov start's weights: exact at t_n for every polynomial in time of
    # degree <= order through the last states, on non-uniform steps
    rng = np.random.default_rng(5)
    for order in range(4):
        for _ in range(20):
            dt = rng.uniform(0.1, 2.0)
            d = rng.uniform(0.1, 2.0, size=3)
            w = sphrt.extrapolation_weights(order, dt, d[:order])
            tau = np.concatenate([[0.0], -np.cumsum(d[:order])])  # t_{n-1-j} - t_{n-1}
            for q in range(order + 1):
                assert abs(np.dot(w, tau ** q) - dt ** q) < 1e-11 * max(1.0, dt ** q)
            if order < 3:  # and not one degree beyond
                q = order + 1
                assert abs(np.dot(w, tau ** q) - dt ** q) > 1e-9
    assert np.allclose(sphrt.extrapolation_weights(1, 0.5, [2.0]), [1.25, -0.25])
    assert np.allclose(sphrt.extrapolation_weights(2, 1.0, [1.0, 1.0]), [3, -3, 1])
    assert np.allclose(sphrt.extrapolation_weights(3, 1.0, [1.0, 1.0, 1.0]), [4, -6, 4, -1])
    assert list(sphrt.extrapolation_weights(0, 1.0)) == [1.0]
    for bad in [(4, 1.0, [1.0] * 4), (1, 0.0, [1.0]), (2, 1.0, [1.0, -1.0])]:
        with pytest.raises(sphrt.SphRtError):
            sphrt.extrapolation_weights(*bad)


def test_history_calls_check_their_arguments_before_the_device():
    L = sphrt.load()
    S = sphrt.Solver(sphrt.default_config(dim=2))
    depth = np.zeros(1, dtype=np.int32)
    E = np.ones((3, 4))
    dt = np.ones(3)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert L.sph_rt_get_history(None, p(depth), p(E), p(dt)) == sphrt.EINVAL
    assert L.sph_rt_get_history(S._h, None, p(E), p(dt)) == sphrt.EINVAL
    assert L.sph_rt_set_history(S._h, 1, None, p(dt)) == sphrt.EINVAL
    # no particles yet: a state error, whatever the depth
    assert L.sph_rt_get_history(S._h, p(depth), p(E), p(dt)) == sphrt.ESTATE
    assert L.sph_rt_set_history(S._h, 1, p(E), p(dt)) == sphrt.ESTATE
    assert L.sph_rt_set_history(S._h, 9, p(E), p(dt)) == sphrt.ESTATE
    S.close()
