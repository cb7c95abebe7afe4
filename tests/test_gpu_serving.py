"""Serving: each request's result is the same alone and in a mix of
concurrently resident requests (resident single-problem path, and small
requests fused into batched launches), and admission respects the HBM budget."""
import numpy as np
import pytest

from paper_2001_11606_gb300 import inputs as I
from paper_2001_11606_gb300 import sphrt

pytestmark = pytest.mark.gpu


def _requests(k=6, seed=40):
    reqs = []
    for i, d in enumerate(I.serving_stream(k, seed=seed, n_min=800, n_max=12000)):
        w = I.heating_wave(d["dim"], d["n_target"], d["sigma0"], seed=d["seed"], steps=4)
        reqs.append(w)
    return reqs


def _alone(w):
    S = sphrt.solver_for(w)
    for _ in range(w.steps):
        S.step(w.dt)
    e, E, _ = S.get_energies()
    S.close()
    return e, E


def _batch_of_one(w):
    B = sphrt.Batch(sphrt.config_from_params(w.params))
    B.add(w.particles, w.e0, w.E0)
    B.run(w.dt, w.steps)
    e, E = B.get_energies(0)
    B.close()
    return e, E


def test_results_same_alone_and_in_the_mix():
    reqs = _requests()
    srv = sphrt.Server(workers=4, max_resident=8, fuse_max_n=0)
    ids = [srv.submit(sphrt.config_from_params(w.params), w.particles, w.e0, w.E0, w.steps, w.dt)
           for w in reqs]
    for rid in ids:
        assert srv.wait(rid) == sphrt.OK
    info = srv.info()
    assert info.peak_resident >= 2  # requests really overlapped
    for w, rid in zip(reqs, ids):
        e, E, st = srv.result(rid)
        ea, Ea = _alone(w)
        assert np.array_equal(e, ea) and np.array_equal(E, Ea)
    srv.close()


def test_fused_small_requests_same_as_alone():
    reqs = _requests(k=10, seed=43)
    cut = 5000
    small = [w.particles.n <= cut for w in reqs]
    assert any(small) and not all(small)
    srv = sphrt.Server(workers=3, max_resident=16, fuse_max_n=cut, fuse_max_k=8)
    ids = [srv.submit(sphrt.config_from_params(w.params), w.particles, w.e0, w.E0, w.steps, w.dt)
           for w in reqs]
    for rid in ids:
        assert srv.wait(rid) == sphrt.OK
    info = srv.info()
    assert info.fused_requests == sum(small) and info.fused_batches >= 1
    for w, rid, fused in zip(reqs, ids, small):
        e, E, st = srv.result(rid)
        m = w.particles.kind == 0
        if fused:
            eb, Eb = _batch_of_one(w)  # same as in a batch of its own
            assert np.array_equal(e, eb) and np.array_equal(E, Eb)
            ea, Ea = _alone(w)  # and the single-problem path within the solver tolerance
            assert np.max(np.abs(E[m] - Ea[m]) / np.abs(Ea[m])) < 1e-7
            assert np.max(np.abs(e[m] - ea[m]) / np.abs(ea[m])) < 1e-7
        else:
            ea, Ea = _alone(w)
            assert np.array_equal(e, ea) and np.array_equal(E, Ea)
    srv.close()


def test_batch_run_equals_single_steps():
    w = _requests(k=1, seed=44)[0]
    cfg = sphrt.config_from_params(w.params)
    A = sphrt.Batch(cfg)
    A.add(w.particles, w.e0, w.E0)
    for _ in range(w.steps):
        A.step(w.dt)
    ea, Ea = A.get_energies(0)
    A.close()
    B = sphrt.Batch(cfg)
    B.add(w.particles, w.e0, w.E0)
    rc, st, ou, kr = B.run(w.dt, w.steps)
    assert rc == sphrt.OK and st[0] == 0 and ou[0] >= w.steps
    eb, Eb = B.get_energies(0)
    B.close()
    assert np.array_equal(ea, eb) and np.array_equal(Ea, Eb)


def test_budget_limits_residency():
    reqs = _requests(k=4, seed=41)
    srv = sphrt.Server(workers=4, max_resident=8, hbm_budget_bytes=1.0, fuse_max_n=0)
    ids = [srv.submit(sphrt.config_from_params(w.params), w.particles, w.e0, w.E0, w.steps, w.dt)
           for w in reqs]
    for rid in ids:
        assert srv.wait(rid) == sphrt.OK
    assert srv.info().peak_resident == 1  # a tiny budget admits one request at a time
    srv.close()


def test_failed_request_reports_error():
    w = _requests(k=1, seed=42)[0]
    srv = sphrt.Server(workers=1)
    cfg = sphrt.config_from_params(w.params, max_outer=1, tol_outer_e=1e-16, tol_outer_E=1e-16)
    rid = srv.submit(cfg, w.particles, w.e0, w.E0, w.steps, w.dt)
    assert srv.wait(rid) == sphrt.ENOTCONV
    with pytest.raises(sphrt.SphRtError):
        srv.result(rid)
    srv.close()
