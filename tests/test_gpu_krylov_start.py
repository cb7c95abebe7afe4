"""Extrapolated start of each step's first linear solve (config.krylov_start =
p > 0: the Lagrange extrapolation in time of order p through the last states):
only where the Krylov iteration starts changes, so the outer iteration of
Alg. 1 reaches the same fixed point -- the results match the oracle to the
same tolerance as the plain start, and a step with no converged previous step
of the same particle set (the first one, the first after new particles) is
bit-identical to the plain start."""
import numpy as np
import pytest

import oracle as O
from paper_2001_11606_gb300 import inputs as I
from paper_2001_11606_gb300 import sphrt

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_krylov=1e-14, tol_outer_e=1e-12, tol_outer_E=1e-12, tol_inner_e=1e-14)


def _oracle(w, steps):
    pb = O.Problem(w.particles, dict(w.params, **TIGHT))
    e, E = w.e0.copy(), w.E0.copy()
    for k in range(1, steps + 1):
        rc, e, E, _ = pb.step(e, E, w.dt, *w.step_inputs(k))
        assert rc == 0
    return e, E


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("prec,tol", [(sphrt.FP64, 1e-10), (sphrt.MIXED, 1e-8)])
def test_extrapolated_start_matches_the_oracle(prec, tol, order):
    w = I.mms_3d_lp(n=20, steps=4)
    runs = {}
    for ks in (0, order):
        S = sphrt.solver_for(w, krylov_start=ks, precision=prec, **TIGHT)
        kry, states = [], []
        for k in range(1, 5):
            _, st = S.step(w.dt, *w.step_inputs(k))
            kry.append(st.krylov_iters_total)
            states.append(S.get_energies()[:2])
        assert S.get_config().krylov_start == ks
        S.close()
        runs[ks] = (kry, states)
    # the first step has no previous one: the same start, the same bits
    (e0, E0), (e1, E1) = runs[0][1][0], runs[order][1][0]
    assert np.array_equal(e0, e1) and np.array_equal(E0, E1)
    assert runs[0][0][0] == runs[order][0][0]
    eo, Eo = _oracle(w, 4)
    m = w.particles.kind == 0
    e, E = runs[order][1][-1]
    assert np.max(np.abs(e[m] - eo[m]) / np.abs(eo[m])) < tol
    assert np.max(np.abs(E[m] - Eo[m]) / np.abs(Eo[m])) < tol


def test_new_particles_restart_from_the_state():
    # after set_particles there is no E^{n-2} of the new slot order: the next
    # step starts from E^{n-1} and equals a fresh handle's step bit for bit
    w = I.mms_3d_lp(n=16, steps=3)
    P = w.particles
    S = sphrt.solver_for(w, krylov_start=3, **TIGHT)
    for k in (1, 2):
        S.step(w.dt, *w.step_inputs(k))
    S.set_particles(P.pos, P.mass, P.rho, P.h, P.sigma0, P.kind, P.copy_of, w.e0, w.E0)
    S.step(w.dt, *w.step_inputs(1))
    e, E, _ = S.get_energies()
    S.close()
    R = sphrt.solver_for(w, krylov_start=0, **TIGHT)
    R.step(w.dt, *w.step_inputs(1))
    e2, E2, _ = R.get_energies()
    R.close()
    assert np.array_equal(e, e2) and np.array_equal(E, E2)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_batched_extrapolated_start_matches_the_oracle(order):
    # per problem: the first step starts from the state, the later ones from the
    # extrapolation; multi-step runs and single steps keep the same history
    probs = []
    for d in I.serving_stream(3, seed=70, n_min=500, n_max=4000):
        probs.append(I.heating_wave(2, d["n_target"], d["sigma0"], seed=d["seed"], steps=4))
    res = {}
    for ks in (0, order):
        cfg = sphrt.config_from_params(probs[0].params, krylov_start=ks, **TIGHT)
        B = sphrt.Batch(cfg)
        for w in probs:
            B.add(w.particles, w.e0, w.E0)
        kry, states = [], []
        for _ in range(4):
            rc, st, ou, kr, en = B.step(probs[0].dt)
            assert np.all(st == 0)
            kry.append(kr.copy())
            states.append([B.get_energies(k) for k in range(len(probs))])
        B.close()
        res[ks] = (kry, states)
    assert np.array_equal(res[0][0][0], res[order][0][0])
    for (e0, E0), (e1, E1) in zip(res[0][1][0], res[order][1][0]):
        assert np.array_equal(e0, e1) and np.array_equal(E0, E1)
    # one run of four steps: the same bits as four single steps
    cfg = sphrt.config_from_params(probs[0].params, krylov_start=order, **TIGHT)
    R = sphrt.Batch(cfg)
    for w in probs:
        R.add(w.particles, w.e0, w.E0)
    rc, st, ou, kr = R.run(probs[0].dt, 4)
    assert rc == sphrt.OK
    for k, w in enumerate(probs):
        e, E = R.get_energies(k)
        assert (np.array_equal(e, res[order][1][-1][k][0])
                and np.array_equal(E, res[order][1][-1][k][1]))
        pb = O.Problem(w.particles, dict(w.params, **TIGHT))
        eo, Eo = w.e0.copy(), w.E0.copy()
        for _ in range(4):
            rc2, eo, Eo, _ = pb.step(eo, Eo, w.dt)
            assert rc2 == 0
        m = w.particles.kind == 0
        assert np.max(np.abs(e[m] - eo[m]) / np.abs(eo[m])) < 1e-10
        assert np.max(np.abs(E[m] - Eo[m]) / np.abs(Eo[m])) < 1e-10
    R.close()


def test_varying_steps_match_the_oracle():
    # steps of changing size: the extrapolation weights follow the step sizes
    w = I.mms_3d_lp(n=16, steps=6)
    dts = [w.dt, 0.5 * w.dt, 0.5 * w.dt, 1.5 * w.dt, w.dt, 2.0 * w.dt]
    S = sphrt.solver_for(w, krylov_start=3, **TIGHT)
    pb = O.Problem(w.particles, dict(w.params, **TIGHT))
    eo, Eo = w.e0.copy(), w.E0.copy()
    for k, dt in enumerate(dts, start=1):
        S.step(dt, *w.step_inputs(k))
        rc, eo, Eo, _ = pb.step(eo, Eo, dt, *w.step_inputs(k))
        assert rc == 0
    e, E, _ = S.get_energies()
    assert list(S.get_history()[1]) == [dts[-1], dts[-2], dts[-3]]
    S.close()
    m = w.particles.kind == 0
    assert np.max(np.abs(e[m] - eo[m]) / np.abs(eo[m])) < 1e-10
    assert np.max(np.abs(E[m] - Eo[m]) / np.abs(Eo[m])) < 1e-10
