"""Checks of the seeded input generators (not of the method)."""
import numpy as np

from paper_2001_11606_gb300 import inputs as I


def test_splitmix64_reference_values():
    # published splitmix64 outputs for state 0 (first three draws)
    z = I.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_lattice_layout_and_jitter_bounds():
    P = I.make_lattice(3, (4, 5, 6), 0.1, seed=3)
    assert P.n == 10 * 11 * 12 and P.n_interior == 4 * 5 * 6
    idx0 = np.floor(P.pos / 0.1)  # cell of each point
    frac = P.pos / 0.1 - idx0
    assert np.all(np.abs(frac - 0.5) <= 0.1 + 1e-12)
    # x runs fastest in the caller order
    assert P.pos[1, 0] > P.pos[0, 0] and abs(P.pos[1, 1] - P.pos[0, 1]) < 0.2 * 0.1 + 1e-12


def test_reflective_ghosts_mirror_their_source():
    P = I.make_lattice(2, (6, 4), 0.25, seed=2, faces=[("dirichlet", "dirichlet"),
                                                        ("reflect", "reflect")])
    c = np.flatnonzero(P.kind == I.COPY)
    assert len(c) > 0 and np.all(P.kind[P.copy_of[c]] == I.INTERIOR)
    src = P.pos[P.copy_of[c]]
    g = P.pos[c]
    assert np.allclose(g[:, 0], src[:, 0])
    lo = g[:, 1] < 0
    assert np.allclose(g[lo, 1], -src[lo, 1]) and np.allclose(g[~lo, 1], 2.0 - src[~lo, 1])


def _fd_sources(m: I.Manufactured, x, t, eps=1e-5):
    """Sources by finite differences of the continuum fields (independent check)."""
    d = m.dim

    def E(x, t):
        return m.a * m.T(x, t) ** 4

    def D(x, t):
        T = m.T(x, t)
        g = np.stack([(E(x + eps * np.eye(d)[k], t) - E(x - eps * np.eye(d)[k], t)) / (2 * eps)
                      for k in range(d)], axis=1)
        sig = m.sigma0 * T ** m.p
        R = np.sqrt(np.sum(g * g, axis=1)) / (sig * E(x, t))
        lam = I._limiter_value_and_slope(R, m.limiter, m.larsen_k)[0]
        return m.c * lam / sig

    div = np.zeros(x.shape[0])
    for k in range(d):
        ek = np.eye(d)[k] * eps
        fp = D(x + ek / 2, t) * (E(x + ek, t) - E(x, t)) / eps
        fm = D(x - ek / 2, t) * (E(x, t) - E(x - ek, t)) / eps
        div += (fp - fm) / eps
    dEdt = (E(x, t + eps) - E(x, t - eps)) / (2 * eps)
    dTdt = (m.T(x, t + eps) - m.T(x, t - eps)) / (2 * eps)
    return m.rho * m.cv * dTdt, dEdt - div


def test_manufactured_sources_match_finite_differences():
    rng = np.random.default_rng(0)
    for dim, p, lim in ((2, 0.0, 0), (3, -3.0, 1), (3, -3.0, 2)):
        m = I.Manufactured(dim=dim, p=p, limiter=lim)
        x = rng.uniform(0.05, 0.95, size=(40, dim))
        Qe, QE = m.sources(x, 0.3)
        Qe2, QE2 = _fd_sources(m, x, 0.3, eps=2e-4)
        assert np.allclose(Qe, Qe2, rtol=1e-6, atol=1e-8)
        assert np.allclose(QE, QE2, rtol=2e-3, atol=2e-3 * np.max(np.abs(QE)))


def test_source_series_equals_sources():
    # the per-step inputs of a workload come from SourceSeries (spatial factors
    # computed once); they equal Manufactured.sources / fields to rounding
    rng = np.random.default_rng(1)
    for dim, p, lim in ((2, 0.0, 0), (3, 0.0, 0), (3, -3.0, 1), (3, -3.0, 2), (2, -3.0, 2)):
        m = I.Manufactured(dim=dim, p=p, limiter=lim)
        x = rng.uniform(-0.1, 1.1, size=(300, dim))
        ser = m.series(x)
        for t in (0.0, 0.37, 2.0):
            Qe, QE = m.sources(x, t)
            Qe2, QE2 = ser.sources(t)
            assert np.allclose(Qe2, Qe, rtol=1e-14, atol=0)
            assert np.allclose(QE2, QE, rtol=1e-13, atol=1e-14 * np.max(np.abs(QE)))
            e, E = m.fields(x, t)
            e2, E2 = ser.fields(t)
            assert np.array_equal(e, e2) and np.array_equal(E, E2)


def test_travelling_cosine_sources_match_finite_differences():
    # the paper's cgs manufactured problem (Sec. 4.3): Q_e = rho de/dt - c sigma_a (E - aT^4),
    # Q_E = dE/dt - div(D grad E) + c sigma_a (E - aT^4), D from the Larsen limiter with
    # sigma_t = sigma_a + sigma_s; checked against central differences of the fields
    rng = np.random.default_rng(2)
    for dim in (1, 2, 3):
        m = I.TravellingCosine(dim=dim)
        x = rng.uniform(0.0, m.dm, size=(30, dim))
        t = 3e-10
        Qe, QE = m.sources(x, t)
        ht, hx = 1e-15, 1e-4
        e_p, E_p = m.fields(x, t + ht)
        e_m, E_m = m.fields(x, t - ht)
        e, E = m.fields(x, t)
        st = m.sigma_a + m.sigma_s

        def D(y):
            Ey = m.fields(y, t)[1]
            g = np.stack([(m.fields(y + hx * np.eye(dim)[k], t)[1]
                           - m.fields(y - hx * np.eye(dim)[k], t)[1]) / (2 * hx)
                          for k in range(dim)], axis=1)
            R = np.sqrt(np.sum(g * g, axis=1)) / (st * Ey)
            return m.c * I._limiter_value_and_slope(R, m.limiter, m.larsen_k)[0] / st

        div = np.zeros(len(x))
        for k in range(dim):
            ek = np.eye(dim)[k] * hx
            fp = D(x + ek / 2) * (m.fields(x + ek, t)[1] - E) / hx
            fm = D(x - ek / 2) * (E - m.fields(x - ek, t)[1]) / hx
            div += (fp - fm) / hx
        coup = m.c * m.sigma_a * (E - m.a * (e / m.cv) ** 4)
        Qe_fd = m.rho * (e_p - e_m) / (2 * ht) - coup
        QE_fd = (E_p - E_m) / (2 * ht) - div + coup
        assert np.allclose(Qe, Qe_fd, rtol=1e-5, atol=1e-6 * np.max(np.abs(Qe)))
        assert np.allclose(QE, QE_fd, rtol=1e-4, atol=1e-4 * np.max(np.abs(QE)))


def test_periodic_ghosts_are_translated_copies():
    w = I.mms_cgs(2, 12, steps=1)
    P = w.particles
    c = np.flatnonzero(P.kind == I.COPY)
    assert len(c) > 0 and np.all(P.kind == np.where(P.kind == I.COPY, I.COPY, I.INTERIOR))
    assert np.all(P.kind[P.copy_of[c]] == I.INTERIOR)
    off = (P.pos[c] - P.pos[P.copy_of[c]]) / 5.0
    assert np.allclose(off, np.round(off), atol=1e-12)
    assert np.all(np.abs(np.round(off)).sum(axis=1) >= 1)
