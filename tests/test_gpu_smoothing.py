"""Per-particle smoothing lengths by the initialisation iteration of Sec. 3.1,
and moving particles (rows a1-a2 re-run with the state kept), on the device,
against the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2001_11606_gb300 import inputs as I
from paper_2001_11606_gb300 import sphrt

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_krylov=1e-14, tol_outer_e=1e-12, tol_outer_E=1e-12, tol_inner_e=1e-14)


def _lattice_workload(dim, n, kern, h_over_dx, seed=3, jitter=0.1, faces=None):
    sup = 1.0 if kern == 1 else 2.0
    P = I.make_lattice(dim, (n,) * dim, 1.0 / n, seed=seed, jitter=jitter, h_over_dx=h_over_dx,
                       support=sup * 1.5, faces=faces)
    m = I.Manufactured(dim=dim)
    e0, E0 = m.fields(P.pos, 0.0)
    prm = dict(dim=dim, kernel=kern, tol_outer_e=1e-10, tol_outer_E=1e-10)
    return I.Workload(f"lat{dim}d", P, prm, 1e-3, 2, mms=m, e0=e0, E0=E0)


@pytest.mark.parametrize("dim,n,kern,h0", [(2, 20, 1, 3.0), (3, 10, 1, 3.5), (2, 20, 0, 1.5),
                                           (1, 40, 1, 3.0)])
def test_adapted_smoothing_lengths_match_oracle(dim, n, kern, h0):
    w = _lattice_workload(dim, n, kern, h0)
    P = w.particles
    h_o, it_o = O.smoothing_lengths(P, w.params, eta=4.0, tol=1e-13)
    S = sphrt.solver_for(w)
    it = S.adapt_smoothing_lengths(eta=4.0, tol=1e-13)
    h_g = S.get_smoothing_lengths()
    m = P.kind == 0
    np.testing.assert_allclose(h_g[m], h_o[m], rtol=1e-11, atol=0)
    assert np.array_equal(h_g[~m], h_o[~m])  # Dirichlet ghosts keep theirs
    assert abs(it - it_o) <= 1
    # the set-up was rebuilt with the new h: neighbour lists bit-exact with the oracle's
    P.h = h_g
    rp, cols = S.get_neighbors()
    orp, ocols = O.neighbors(P.pos, P.h, P.kind, kernel=kern)
    assert np.array_equal(rp, orp) and np.array_equal(cols, ocols.astype(np.int64))


def test_step_after_adapting_matches_oracle():
    w = _lattice_workload(2, 24, 1, 3.0)
    P = w.particles
    S = sphrt.solver_for(w, **TIGHT)
    S.adapt_smoothing_lengths(eta=4.0, tol=1e-13)
    P.h = S.get_smoothing_lengths()  # the oracle takes the device's lengths as given
    pb = O.Problem(P, dict(w.params, **TIGHT))
    e, E = w.e0.copy(), w.E0.copy()
    for k in (1, 2):
        ins = w.step_inputs(k)
        S.step(w.dt, *ins)
        rc, e, E, _ = pb.step(e, E, w.dt, *ins)
        assert rc == 0
    eg, Eg, _ = S.get_energies()
    m = P.kind == 0
    assert np.max(np.abs(eg[m] - e[m]) / e[m]) < 1e-10
    assert np.max(np.abs(Eg[m] - E[m]) / E[m]) < 1e-10


def test_adapt_rejects_huge_starting_h():
    w = _lattice_workload(3, 18, 1, 3.0)  # ~10^4 particles
    w.particles.h[:] = 30.0  # the whole set within one support
    S = sphrt.solver_for(w)
    with pytest.raises(sphrt.SphRtError) as ei:
        S.adapt_smoothing_lengths()
    assert ei.value.status == sphrt.EINVAL


@pytest.mark.parametrize("make", [lambda: I.mms_3d_lp(n=12, steps=3),
                                  lambda: I.heating_wave(2, 2000, 5.0, seed=5, steps=3)])
def test_moving_particles_rebuilds_with_state_kept(make):
    w = make()
    P = w.particles
    prm = dict(w.params, **TIGHT)
    S = sphrt.solver_for(w, **prm)
    pb = O.Problem(P, prm)
    e, E = w.e0.copy(), w.E0.copy()
    ins = w.step_inputs(1)
    S.step(w.dt, *ins)
    rc, e, E, _ = pb.step(e, E, w.dt, *ins)
    # move the interior particles and Dirichlet ghosts by up to 0.05 dx (copy ghosts
    # keep their positions: a ghost's position is the caller's, whatever it copies)
    rng = np.random.default_rng(8)
    pos = P.pos + (rng.uniform(-0.05, 0.05, P.pos.shape) * P.dx)
    c = P.kind == sphrt.COPY
    pos[c] = P.pos[c]
    S.move_particles(pos)
    eg, Eg, _ = S.get_energies()
    assert np.array_equal(eg, S.get_energies()[0])
    P2 = I.Particles(dim=P.dim, dx=P.dx, counts=P.counts, pos=pos, kind=P.kind, copy_of=P.copy_of,
                     mass=P.mass, rho=P.rho, h=P.h, sigma0=P.sigma0)
    rp, cols = S.get_neighbors()
    orp, ocols = O.neighbors(P2.pos, P2.h, P2.kind)
    assert np.array_equal(rp, orp) and np.array_equal(cols, ocols.astype(np.int64))
    m = P.kind == 0
    # the state survived the rebuild
    assert np.max(np.abs(eg[m] - e[m]) / e[m]) < 1e-10
    pb2 = O.Problem(P2, prm)
    for k in (2, 3):
        ins = w.step_inputs(k)
        S.step(w.dt, *ins)
        rc, e, E, _ = pb2.step(e, E, w.dt, *ins)
        assert rc == 0
    eg, Eg, _ = S.get_energies()
    assert np.max(np.abs(eg[m] - e[m]) / e[m]) < 1e-10
    assert np.max(np.abs(Eg[m] - E[m]) / E[m]) < 1e-10


def test_move_rejects_non_finite_positions():
    w = I.mms_2d(n=8, steps=1)
    S = sphrt.solver_for(w)
    pos = w.particles.pos.copy()
    pos[3, 1] = np.inf
    with pytest.raises(sphrt.SphRtError) as ei:
        S.move_particles(pos)
    assert ei.value.status == sphrt.EINVAL
