"""Batched form: many small problems in one launch per step.  Each problem's
result is the same alone (a batch of one) and in the batch, and matches the
CPU oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2001_11606_gb300 import inputs as I
from paper_2001_11606_gb300 import sphrt

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_krylov=1e-14, tol_outer_e=1e-12, tol_outer_E=1e-12, tol_inner_e=1e-14)


def _problems(dim, k=5, seed=60):
    out = []
    for d in I.serving_stream(k, seed=seed, n_min=500, n_max=6000):
        out.append(I.heating_wave(dim, d["n_target"], d["sigma0"], seed=d["seed"], steps=3))
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_batch_same_alone_and_in_the_batch(dim):
    probs = _problems(dim)
    cfg = sphrt.config_from_params(probs[0].params, **TIGHT)
    B = sphrt.Batch(cfg)
    for w in probs:
        B.add(w.particles, w.e0, w.E0)
    for _ in range(3):
        rc, st, ou, kr, en = B.step(probs[0].dt)
        assert np.all(st == 0) and np.all(ou >= 1)
    for k, w in enumerate(probs):
        e, E = B.get_energies(k)
        A = sphrt.Batch(cfg)
        A.add(w.particles, w.e0, w.E0)
        for _ in range(3):
            A.step(w.dt)
        ea, Ea = A.get_energies(0)
        assert np.array_equal(e, ea) and np.array_equal(E, Ea)
        A.close()
    B.close()


def test_batch_matches_oracle_and_conserves_energy():
    probs = _problems(2, k=3, seed=61)
    cfg = sphrt.config_from_params(probs[0].params, **TIGHT)
    B = sphrt.Batch(cfg)
    for w in probs:
        B.add(w.particles, w.e0, w.E0)
    oracles = [(O.Problem(w.particles, dict(w.params, **TIGHT)), w.e0.copy(), w.E0.copy())
               for w in probs]
    for _ in range(3):
        rc, st, ou, kr, en = B.step(probs[0].dt)
        for k in range(len(probs)):
            before, after, src, bnd = en[k]
            assert abs(after - before - src - bnd) < 1e-11 * abs(after)
        for k, (pb, e, E) in enumerate(oracles):
            rc2, e, E, _ = pb.step(e, E, probs[k].dt)
            assert rc2 == 0
            oracles[k] = (pb, e, E)
    for k, (pb, e, E) in enumerate(oracles):
        eg, Eg = B.get_energies(k)
        m = probs[k].particles.kind == 0
        assert np.max(np.abs(eg[m] - e[m]) / np.abs(e[m])) < 1e-10
        assert np.max(np.abs(Eg[m] - E[m]) / np.abs(E[m])) < 1e-10
    B.close()


def test_batch_with_sources_matches_single_problem_path():
    w = I.mms_2d(n=16, steps=2)
    cfg = sphrt.config_from_params(w.params, **TIGHT)
    B = sphrt.Batch(cfg)
    B.add(w.particles, w.e0, w.E0)
    # constant sources and ghost values of step 1 on both paths
    Qe, QE, ge, gE = w.step_inputs(1)
    B.set_sources(0, Qe, QE)
    S = sphrt.solver_for(w, **TIGHT)
    for _ in range(2):
        B.step(w.dt)
        S.step(w.dt, Qe, QE)
    eb, Eb = B.get_energies(0)
    es, Es, _ = S.get_energies()
    m = w.particles.kind == 0
    assert np.max(np.abs(eb[m] - es[m]) / np.abs(es[m])) < 1e-10
    assert np.max(np.abs(Eb[m] - Es[m]) / np.abs(Es[m])) < 1e-10
