"""Device-driven outer loop: the step's loop as one CUDA graph with conditional
WHILE nodes gives bitwise the same results and statistics as the host-driven
loop, is captured once and replayed, and ends on every failure path."""
import numpy as np
import pytest

from paper_2001_11606_gb300 import inputs as I
from paper_2001_11606_gb300 import sphrt

pytestmark = pytest.mark.gpu


def _run(w, steps, **cfg):
    S = sphrt.solver_for(w, **cfg)
    stats = []
    for n in range(1, steps + 1):
        _, st = S.step(w.dt, *w.step_inputs(n))
        stats.append((st.outer_iters, st.krylov_iters_total,
                      tuple(st.krylov_iters_per_outer[:st.outer_iters]), st.newton_iters_max))
    e, E, _ = S.get_energies()
    info = S.loop_graph_info()
    launches = S.launch_count()
    S.close()
    return e, E, stats, info, launches


@pytest.mark.parametrize("precond,precision,post,n", [
    (sphrt.PRECOND_AMG, sphrt.FP64, 1, 12), (sphrt.PRECOND_AMG, sphrt.MIXED, 1, 12),
    (sphrt.PRECOND_CHEBYSHEV, sphrt.FP64, 1, 12), (sphrt.PRECOND_JACOBI, sphrt.FP64, 1, 12),
    # the CG whose product comes from the V-cycle, without and with A P (32^3)
    (sphrt.PRECOND_AMG, sphrt.FP64, 0, 12), (sphrt.PRECOND_AMG, sphrt.MIXED, 0, 12),
    (sphrt.PRECOND_AMG, sphrt.MIXED, 0, 32)])
def test_graph_loop_matches_host_loop_bitwise(precond, precision, post, n):
    w = I.mms_3d_lp(n=n, steps=3)
    kw = dict(precond=precond, precision=precision, fine_post_smooth=post)
    g = _run(w, 3, graphs=1, **kw)
    h = _run(w, 3, graphs=0, **kw)
    assert np.array_equal(g[0], h[0]) and np.array_equal(g[1], h[1])
    assert g[2] == h[2]
    assert g[3] == (1, 3)  # captured once, launched every step
    assert h[3] == (0, 0)


def test_graph_recaptured_when_dt_changes():
    w = I.mms_2d(n=16, steps=3)
    S = sphrt.solver_for(w)
    S.step(w.dt, *w.step_inputs(1))
    S.step(w.dt, *w.step_inputs(2))
    assert S.loop_graph_info() == (1, 2)
    S.step(0.5 * w.dt, *w.step_inputs(3))
    assert S.loop_graph_info() == (2, 3)
    S.close()


def test_graph_krylov_failure_ends_step_unchanged():
    w = I.mms_2d(n=16, steps=1)
    # Jacobi CG cannot reach 1e-15 in one iteration (AMG on this small problem can:
    # its single level is solved almost exactly)
    S = sphrt.solver_for(w, precond=sphrt.PRECOND_JACOBI, max_krylov=1, tol_krylov=1e-15)
    e0, E0, _ = S.get_energies()
    with pytest.raises(sphrt.SphRtError) as ei:
        S.step(w.dt, *w.step_inputs(1))
    assert ei.value.status == sphrt.ENOTCONV and "Krylov" in str(ei.value)
    e1, E1, _ = S.get_energies()
    assert np.array_equal(e0, e1) and np.array_equal(E0, E1)
    S.close()


def test_graph_outer_limit_ends_step_unchanged():
    w = I.mms_2d(n=16, steps=1)
    S = sphrt.solver_for(w, max_outer=2, tol_outer_e=1e-300, tol_outer_E=1e-300)
    e0, E0, _ = S.get_energies()
    with pytest.raises(sphrt.SphRtError) as ei:
        S.step(w.dt, *w.step_inputs(1))
    assert ei.value.status == sphrt.ENOTCONV and "max_outer" in str(ei.value)
    e1, E1, _ = S.get_energies()
    assert np.array_equal(e0, e1) and np.array_equal(E0, E1)
    S.close()


@pytest.mark.parametrize("precision", [sphrt.FP64, sphrt.MIXED])
def test_cluster_tail_vcycle_bitwise_and_fewer_launches(precision):
    # 32^3: levels of ~420k, 80k, 19k, 5k stored entries run in the cluster tail
    w = I.mms_3d_lp(n=32, steps=2)
    on = _run(w, 2, precision=precision, amg_tail=1)
    off = _run(w, 2, precision=precision, amg_tail=0)
    assert np.array_equal(on[0], off[0]) and np.array_equal(on[1], off[1])
    assert on[2] == off[2]
    assert on[4] < off[4]  # the tail replaces several launches per V-cycle


@pytest.mark.parametrize("precision,post", [(sphrt.FP64, 1), (sphrt.MIXED, 1), (sphrt.FP64, 0),
                                            (sphrt.MIXED, 0)])
def test_dependent_launch_changes_no_bit(precision, post):
    # programmatic dependent launch only lets a kernel's launch overlap its
    # predecessor's drain; every kernel waits for its predecessor's results
    w = I.mms_3d_lp(n=12, steps=3)
    on = _run(w, 3, precision=precision, pdl=1, fine_post_smooth=post)
    off = _run(w, 3, precision=precision, pdl=0, fine_post_smooth=post)
    assert np.array_equal(on[0], off[0]) and np.array_equal(on[1], off[1])
    assert on[2] == off[2]
