"""Time step choice of Sec. 3.3 (Eq. energy-fractional) on the device.

With config.dt_target > 0 a converged step reports the fractional changes
eta_e, eta_E of the material and radiation energies (volume average in the
denominator) and the proposed next step.  Checked against the oracle's
next_dt on the oracle's own trajectory, against the closed form of an
absorbing infinite medium, and against the growth limit and cap at
equilibrium (the cases the oracle's own pins use).
"""
import numpy as np
import pytest

import oracle as O
from paper_2001_11606_gb300 import inputs as I
from paper_2001_11606_gb300 import sphrt

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_krylov=1e-14, tol_outer_e=1e-12, tol_outer_E=1e-12, tol_inner_e=1e-14)


def test_dt_choice_matches_oracle_on_manufactured_problem():
    w = I.mms_3d_lp(n=16, steps=3)
    P = w.particles
    prm = dict(w.params, **TIGHT)
    S = sphrt.solver_for(w, **prm, dt_target=0.05, dt_growth=10.0)
    pb = O.Problem(P, prm)
    V = P.mass / P.rho
    m = P.kind == 0
    e, E = w.e0.copy(), w.E0.copy()
    for n in (1, 2, 3):
        ins = w.step_inputs(n)
        _, st = S.step(w.dt, *ins)
        rc, e1, E1, _ = pb.step(e, E, w.dt, *ins)
        assert rc == 0
        dt_o, eta_e, eta_E = O.next_dt(e1, e, E1, E, V, m, w.dt, target=0.05, growth=10.0)
        # the changes are differences of nearly equal energies: each side's 1e-12
        # agreement on the energies becomes ~1e-9 on eta
        assert st.eta_e == pytest.approx(eta_e, rel=1e-7, abs=0)
        assert st.eta_E == pytest.approx(eta_E, rel=1e-7, abs=0)
        assert st.dt_next == pytest.approx(dt_o, rel=1e-7, abs=0)
        e, E = e1, E1


def _single_particle(e0, E0):
    P = I.make_lattice(1, (1,), 1.0, seed=0)
    keep = P.kind == 0
    P1 = I.Particles(dim=1, dx=1.0, counts=(1,), pos=P.pos[keep], kind=P.kind[keep],
                     copy_of=P.copy_of[keep], mass=P.mass[keep], rho=P.rho[keep],
                     h=P.h[keep], sigma0=P.sigma0[keep])
    prm = dict(dim=1, a=0.0, tol_outer_e=1e-12, tol_outer_E=1e-12, tol_krylov=1e-14,
               tol_inner_e=1e-14)
    return I.Workload("one", P1, prm, 0.1, 1, e0=np.array([e0]), E0=np.array([E0]))


@pytest.mark.parametrize("ratio", [1.0 / 50.0, 30.0])
def test_dt_choice_absorbing_medium_closed_form(ratio):
    # a = 0 (absorption only): E_n = E_{n-1} / (1 + dt), eta_E = dt / (1 + target)
    # exactly, so dt_{n+1} = sqrt(dt_n dt*) with dt* = target (1 + target)
    target = 0.05
    dt_star = target * (1.0 + target)
    w = _single_particle(1e12, 1.0)
    S = sphrt.solver_for(w, dt_target=target, dt_growth=1e30)
    dt = ratio * dt_star
    E_prev = 1.0
    for n in range(1, 9):
        _, st = S.step(dt)
        _, E, _ = S.get_energies()
        assert E[0] == pytest.approx(E_prev / (1.0 + dt), rel=1e-13, abs=0)
        assert st.eta_E == pytest.approx(dt / (1.0 + target), rel=1e-12, abs=0)
        assert st.eta_e < 1e-6 * st.eta_E
        assert st.dt_next == pytest.approx(dt_star * ratio ** (0.5**n), rel=1e-9, abs=0)
        E_prev, dt = E[0], st.dt_next


def test_dt_choice_growth_and_cap_at_equilibrium():
    # nothing changes at equilibrium (eta = 0): the step grows by dt_growth per step
    # up to dt_max, as in the infinite-medium runs of Sec. 4.1 (x10, cap 0.1)
    P = I.make_lattice(2, (6, 6), 1.0 / 6, seed=4)
    T = 1.4
    e0 = np.full(P.n, 1.3 * T)
    E0 = np.full(P.n, 0.7 * T**4)
    prm = dict(dim=2, a=0.7, c=2.0, cv=1.3, limiter=1, opacity_exp=-3.0)
    w = I.Workload("eq", P, prm, 1e-6, 1, e0=e0, E0=E0)
    S = sphrt.solver_for(w, dt_target=0.05, dt_growth=10.0, dt_max=0.1)
    dt, dts = 1e-6, []
    for _ in range(8):
        _, st = S.step(dt)
        assert st.eta_e < 1e-12 and st.eta_E < 1e-12
        dt = st.dt_next
        dts.append(dt)
    assert dts[:5] == pytest.approx([1e-5, 1e-4, 1e-3, 1e-2, 0.1], rel=1e-12, abs=0)
    assert dts[5:] == [0.1, 0.1, 0.1]


def test_dt_choice_off_reports_zero():
    w = I.mms_2d(n=16, steps=1)
    S = sphrt.solver_for(w)
    _, st = S.step(w.dt, *w.step_inputs(1))
    assert st.dt_next == 0.0 and st.eta_e == 0.0 and st.eta_E == 0.0
