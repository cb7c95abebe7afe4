"""Solver autotuner (config.autotune = 1): the first step times one trial step
per smoother candidate from the same state, keeps the fastest, and leaves the
state where it was -- the tuned handle's results equal those of a handle set
to the chosen settings, bit for bit, and match the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2001_11606_gb300 import inputs as I
from paper_2001_11606_gb300 import sphrt

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_krylov=1e-14, tol_outer_e=1e-12, tol_outer_E=1e-12, tol_inner_e=1e-14)


def _run(w, steps, **cfg):
    S = sphrt.solver_for(w, **cfg)
    for k in range(1, steps + 1):
        S.step(w.dt, *w.step_inputs(k))
    e, E, _ = S.get_energies()
    return S, e, E


@pytest.mark.parametrize("over,ncand", [(dict(precision=sphrt.FP64), 4),
                                        (dict(precision=sphrt.MIXED), 5),
                                        (dict(precond=sphrt.PRECOND_CHEBYSHEV), 5)])
def test_tuned_solver_equals_its_choice_and_the_oracle(over, ncand):
    w = I.mms_3d_lp(n=20, steps=2)
    S, e, E = _run(w, 2, autotune=1, **over, **TIGHT)
    trials = S.solver_tuning()
    assert len(trials) == ncand
    assert all(t[3] is not None and t[3] > 0 for t in trials)
    c = S.get_config()
    chosen = (c.fine_post_smooth, c.cheb_degree, c.reliable_drop)
    best = min(trials, key=lambda t: t[3])
    assert chosen == best[:3]
    assert c.autotune == 1
    S.close()
    # the same settings without tuning: the same bits
    R, e2, E2 = _run(w, 2, autotune=2, fine_post_smooth=chosen[0], cheb_degree=chosen[1],
                     reliable_drop=chosen[2], **over, **TIGHT)
    assert R.solver_tuning() == []
    R.close()
    assert np.array_equal(e, e2) and np.array_equal(E, E2)
    # and the oracle
    pb = O.Problem(w.particles, dict(w.params, **TIGHT))
    eo, Eo = w.e0.copy(), w.E0.copy()
    for k in (1, 2):
        rc, eo, Eo, _ = pb.step(eo, Eo, w.dt, *w.step_inputs(k))
        assert rc == 0
    m = w.particles.kind == 0
    tol = 1e-8 if over.get("precision") == sphrt.MIXED else 1e-10
    assert np.max(np.abs(e[m] - eo[m]) / np.abs(eo[m])) < tol
    assert np.max(np.abs(E[m] - Eo[m]) / np.abs(Eo[m])) < tol


def test_tuning_keeps_host_staged_inputs_for_every_trial():
    # the host entry point stages the sources in buffers a step may use as
    # scratch (the Chebyshev preconditioner does); every trial must see them
    w = I.mms_2d(n=32, steps=2)
    S, e, E = _run(w, 1, autotune=1, precond=sphrt.PRECOND_CHEBYSHEV, **TIGHT)
    c = S.get_config()
    S.close()
    R, e2, E2 = _run(w, 1, precond=sphrt.PRECOND_CHEBYSHEV, cheb_degree=c.cheb_degree, **TIGHT)
    R.close()
    assert np.array_equal(e, e2) and np.array_equal(E, E2)


def test_jacobi_has_nothing_to_tune():
    w = I.mms_2d(n=16, steps=1)
    S, e, E = _run(w, 1, autotune=1, precond=sphrt.PRECOND_JACOBI)
    assert S.solver_tuning() == []
    S.close()
