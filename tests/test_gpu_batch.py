"""Batched form: many small problems in one launch per step and cluster size.
Each problem's result is the same alone (a batch of one) and in the batch, for
every launch shape it matches the CPU oracle, and the autotuner leaves the
state where it was."""
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


def _state(B, K):
    return [B.get_energies(k) for k in range(K)]


def test_batch_blocks_per_sm_do_not_change_a_bit():
    probs = _problems(3, k=4, seed=62)
    cfg = sphrt.config_from_params(probs[0].params, **TIGHT)
    out = []
    for bps in (1, 2):
        B = sphrt.Batch(cfg)
        for w in probs:
            B.add(w.particles, w.e0, w.E0)
        B.set_shape(4, 2, bps, 512)
        B.run(probs[0].dt, 3)
        out.append(_state(B, len(probs)))
        B.close()
    for (e1, E1), (e2, E2) in zip(*out):
        assert np.array_equal(e1, e2) and np.array_equal(E1, E2)


# rows per CTA 64..2048 put these problems (500..6000 particles) on clusters
# of 1 to 8 blocks; 0 gives each one block
@pytest.mark.parametrize("shape", [(2, 1, 1, 0), (8, 3, 2, 256), (4, 6, 1, 2048), (1, 2, 1, 64),
                                   (1, 1, 2, 1024)])
def test_batch_shapes_match_the_oracle(shape):
    probs = _problems(2, k=3, seed=63)
    cfg = sphrt.config_from_params(probs[0].params, **TIGHT)
    B = sphrt.Batch(cfg)
    for w in probs:
        B.add(w.particles, w.e0, w.E0)
    B.set_shape(*shape)
    rc, st, ou, kr = B.run(probs[0].dt, 2)
    assert np.all(st == 0)
    for k, w in enumerate(probs):
        pb = O.Problem(w.particles, dict(w.params, **TIGHT))
        e, E = w.e0.copy(), w.E0.copy()
        for _ in range(2):
            rc2, e, E, _ = pb.step(e, E, w.dt)
            assert rc2 == 0
        eg, Eg = B.get_energies(k)
        m = w.particles.kind == 0
        assert np.max(np.abs(eg[m] - e[m]) / np.abs(e[m])) < 1e-10
        assert np.max(np.abs(Eg[m] - E[m]) / np.abs(E[m])) < 1e-10
    B.close()


def test_batch_autotune_keeps_the_state_and_picks_a_converged_shape():
    probs = _problems(3, k=6, seed=64)
    cfg = sphrt.config_from_params(probs[0].params, **TIGHT)
    B = sphrt.Batch(cfg)
    for w in probs:
        B.add(w.particles, w.e0, w.E0)
    before = _state(B, len(probs))
    chosen, table = B.autotune(probs[0].dt)
    # the rows-per-CTA sweep repeats one shape of the grid
    assert len(table) == sphrt.BATCH_TUNE_CANDIDATES - 1
    assert table[chosen] is not None
    assert all(t is None or t >= table[chosen] for t in table.values())
    assert B.get_shape() == chosen
    for (e1, E1), (e2, E2) in zip(before, _state(B, len(probs))):
        assert np.array_equal(e1, e2) and np.array_equal(E1, E2)
    # the tuned shape stays set: a run with it equals a fresh batch set to it
    B.run(probs[0].dt, 2)
    A = sphrt.Batch(cfg)
    for w in probs:
        A.add(w.particles, w.e0, w.E0)
    A.set_shape(*chosen)
    A.run(probs[0].dt, 2)
    for (e1, E1), (e2, E2) in zip(_state(A, len(probs)), _state(B, len(probs))):
        assert np.array_equal(e1, e2) and np.array_equal(E1, E2)
    A.close()
    B.close()


def test_config_autotune_tunes_on_the_first_run():
    probs = _problems(2, k=4, seed=65)
    cfg = sphrt.config_from_params(probs[0].params, autotune=1, **TIGHT)
    B = sphrt.Batch(cfg)
    for w in probs:
        B.add(w.particles, w.e0, w.E0)
    rc, st, ou, kr = B.run(probs[0].dt, 2)
    assert np.all(st == 0)
    W, deg, bps, rows = B.get_shape()
    assert W in sphrt.BATCH_TUNE_LANES and deg in sphrt.BATCH_TUNE_DEGREES and bps in (1, 2)
    assert rows in sphrt.BATCH_TUNE_ROWS
    ref = sphrt.Batch(sphrt.config_from_params(probs[0].params, **TIGHT))
    for w in probs:
        ref.add(w.particles, w.e0, w.E0)
    ref.run(probs[0].dt, 2)
    for k, w in enumerate(probs):
        m = w.particles.kind == 0
        (e1, E1), (e2, E2) = B.get_energies(k), ref.get_energies(k)
        assert np.max(np.abs(e1[m] - e2[m]) / np.abs(e2[m])) < 1e-10
        assert np.max(np.abs(E1[m] - E2[m]) / np.abs(E2[m])) < 1e-10
    info = B.problem_info(0)
    assert info["n_total"] == probs[0].particles.n
    assert info["n_interior"] == probs[0].particles.n_interior
    assert info["nnz_operator"] > info["n_interior"] and info["nnz_neighbours"] > 0
    ref.close()
    B.close()


def test_add_many_equals_one_by_one_and_is_all_or_none():
    probs = _problems(3, k=6, seed=66)
    cfg = sphrt.config_from_params(probs[0].params, **TIGHT)
    A = sphrt.Batch(cfg)
    for w in probs:
        A.add(w.particles, w.e0, w.E0)
    B = sphrt.Batch(cfg)
    # a bad problem in the middle: nothing is added
    bad = probs[2].particles
    pos = bad.pos.copy()
    pos[5, 0] = np.nan
    Pbad = I.Particles(dim=bad.dim, dx=bad.dx, counts=bad.counts, pos=pos, kind=bad.kind,
                       copy_of=bad.copy_of, mass=bad.mass, rho=bad.rho, h=bad.h,
                       sigma0=bad.sigma0)
    with pytest.raises(sphrt.SphRtError) as ex:
        B.add_many([(w.particles, w.e0, w.E0) for w in probs[:2]] + [(Pbad, probs[2].e0,
                                                                      probs[2].E0)])
    assert ex.value.status == sphrt.EINVAL and "problem 2" in str(ex.value)
    B._n = []
    assert B.add_many([(w.particles, w.e0, w.E0) for w in probs], threads=3) == 0
    for X in (A, B):
        rc, st, ou, kr = X.run(probs[0].dt, 2)
        assert np.all(st == 0)
    for k in range(len(probs)):
        (e1, E1), (e2, E2) = A.get_energies(k), B.get_energies(k)
        assert np.array_equal(e1, e2) and np.array_equal(E1, E2)
    A.close()
    B.close()


def test_destroyed_buffers_are_cached_and_released_on_request():
    torch = pytest.importorskip("torch")
    probs = _problems(3, k=4, seed=67)
    cfg = sphrt.config_from_params(probs[0].params)
    sphrt.release_cached_memory(0)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    B = sphrt.Batch(cfg)
    B.add_many([(w.particles, w.e0, w.E0) for w in probs])
    B.run(probs[0].dt, 1)
    B.close()
    torch.cuda.synchronize()
    held = free0 - torch.cuda.mem_get_info()[0]
    assert held > 0  # the destroyed handles' buffers stay in the cache
    A = sphrt.Batch(cfg)  # and a new batch runs from them
    A.add_many([(w.particles, w.e0, w.E0) for w in probs])
    rc, st, ou, kr = A.run(probs[0].dt, 1)
    assert np.all(st == 0)
    A.close()
    sphrt.release_cached_memory(0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (256 << 20)  # module code loaded meanwhile
