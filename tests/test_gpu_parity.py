"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: neighbour lists bit-exact; material data and operator entries
1e-13 relative (same formulas, different rounding order); FP64 energies after
full steps 1e-10 relative (both sides converge to the same discrete fixed
point; parity runs tighten the Krylov and outer tolerances on both sides so
that the iteration error is far below that); the mixed-precision form 1e-8.
"""
import numpy as np
import pytest

import oracle as O
from paper_2001_11606_gb300 import inputs as I
from paper_2001_11606_gb300 import sphrt

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_krylov=1e-14, tol_outer_e=1e-12, tol_outer_E=1e-12, tol_inner_e=1e-14)


def rel_err(a, b, mask):
    return float(np.max(np.abs(a[mask] - b[mask]) / np.maximum(np.abs(b[mask]), 1e-300)))


def run_both(w, steps, gpu_over=None, orc_over=None, check=True):
    gpu_over = dict(gpu_over or {})
    prm = dict(w.params, **(orc_over or {}))
    S = sphrt.solver_for(w, **dict(prm, **gpu_over))
    pb = O.Problem(w.particles, prm)
    e, E = w.e0.copy(), w.E0.copy()
    gstats, ostats = [], []
    for n in range(1, steps + 1):
        Qe, QE, ge, gE = w.step_inputs(n)
        rc, st = S.step(w.dt, Qe, QE, ge, gE)
        gstats.append(st)
        rc, e, E, so = pb.step(e, E, w.dt, Qe, QE, ge, gE)
        assert rc == 0
        ostats.append(so)
    eg, Eg, tot = S.get_energies()
    m = w.particles.kind == 0
    out = dict(err_e=rel_err(eg, e, m), err_E=rel_err(Eg, E, m), S=S, pb=pb, gstats=gstats,
               ostats=ostats, e=e, E=E, eg=eg, Eg=Eg, tot=tot)
    return out


# ---------------------------------------------------------------------------
# a1-a2: neighbour lists
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("make", [lambda: I.mms_2d(n=32), lambda: I.mms_3d_lp(n=12),
                                  lambda: I.heating_wave(2, 3000, 5.0, seed=9),
                                  lambda: I.heating_wave(3, 3000, 5.0, seed=9)])
def test_neighbors_bit_exact(make):
    w = make()
    P = w.particles
    S = sphrt.solver_for(w)
    rp, cols = S.get_neighbors()
    orp, ocols = O.neighbors(P.pos, P.h, P.kind)
    assert np.array_equal(rp, orp)
    assert np.array_equal(cols, ocols.astype(np.int64))


def test_neighbors_bit_exact_varied_h():
    w = I.mms_3d_lp(n=10)
    P = w.particles
    rng = np.random.default_rng(4)
    P.h = P.h * rng.uniform(0.7, 1.3, P.n)
    S = sphrt.solver_for(w)
    rp, cols = S.get_neighbors()
    orp, ocols = O.neighbors(P.pos, P.h, P.kind)
    assert np.array_equal(rp, orp) and np.array_equal(cols, ocols.astype(np.int64))


def test_neighbors_unjittered_lattice_edge_cases():
    # pairs at exactly r = 2h must be excluded on both sides (strict inequality)
    P = I.make_lattice(3, (9, 7, 5), 1.0 / 64, seed=0, jitter=0.0)
    w = I.Workload("lattice", P, I.mms_3d_lp(n=4).params, 1e-3, 1, e0=np.ones(P.n),
                   E0=np.ones(P.n))
    S = sphrt.solver_for(w)
    rp, cols = S.get_neighbors()
    orp, ocols = O.neighbors(P.pos, P.h, P.kind)
    assert np.array_equal(rp, orp) and np.array_equal(cols, ocols.astype(np.int64))
    interior = np.flatnonzero(P.kind == 0)
    assert np.all(np.diff(rp)[interior] == 92)


def test_single_interior_particle_without_neighbours():
    P = I.make_lattice(1, (1,), 1.0, seed=0)
    keep = P.kind == 0
    P1 = I.Particles(dim=1, dx=1.0, counts=(1,), pos=P.pos[keep], kind=P.kind[keep],
                     copy_of=P.copy_of[keep], mass=P.mass[keep], rho=P.rho[keep],
                     h=P.h[keep], sigma0=P.sigma0[keep])
    prm = dict(dim=1, tol_outer_e=1e-12, tol_outer_E=1e-12, tol_krylov=1e-14,
               tol_inner_e=1e-14)
    w = I.Workload("one", P1, prm, 0.1, 3, e0=np.array([1.0]), E0=np.array([1e-16]))
    r = run_both(w, 3)
    assert r["err_e"] < 1e-12 and r["err_E"] < 1e-10


# ---------------------------------------------------------------------------
# a3-a4: material data and operator of one step
# ---------------------------------------------------------------------------
def _operator_dict(rowptr, cols, vals, diag):
    d = {}
    for i in range(len(rowptr) - 1):
        for k in range(rowptr[i], rowptr[i + 1]):
            key = (i, int(cols[k]))
            d[key] = d.get(key, 0.0) + vals[k]
    return d


@pytest.mark.parametrize("make", [lambda: I.mms_2d(n=16), lambda: I.mms_3d_lp(n=8),
                                  lambda: I.heating_wave(2, 1200, 30.0, seed=3)])
def test_properties_and_operator_match_oracle(make):
    w = make()
    P = w.particles
    S = sphrt.solver_for(w, precond=sphrt.PRECOND_JACOBI)
    Qe, QE, ge, gE = w.step_inputs(1)
    S.step(w.dt, Qe, QE, ge, gE)
    pg = S.get_properties()
    pb = O.Problem(P, w.params)
    po = pb.properties(w.e0, w.E0, w.dt)
    live = P.kind != sphrt.COPY
    for k in ("T", "sigma", "f", "R", "lambda", "D"):
        np.testing.assert_allclose(pg[k][live], po[k][live], rtol=1e-13, atol=1e-300, err_msg=k)
    # operator of Eq. diffusion-solve, with the Dirichlet ghost values at t^1
    Eg = w.E0.copy()
    Eg[P.kind == sphrt.DIRICHLET] = gE[P.kind == sphrt.DIRICHLET]
    arow, acol, aval, adiag, gb = pb.assemble(po, w.dt, Eg)
    rowptr, cols, vals, diag, ggb = S.get_operator()
    m = P.kind == 0
    np.testing.assert_allclose(diag[m], adiag[m], rtol=1e-13)
    np.testing.assert_allclose(ggb[m], gb[m], rtol=1e-12, atol=1e-12 * np.max(np.abs(gb)))
    dg = _operator_dict(rowptr, cols, vals, diag)
    do = _operator_dict(arow, acol, aval, adiag)
    # self-copy entries fold into the diagonal on both sides
    dg = {k: v for k, v in dg.items() if k[0] != k[1]}
    assert set(dg) == set(do)
    keys = sorted(do)
    a = np.array([dg[k] for k in keys])
    b = np.array([do[k] for k in keys])
    # entries near the edge of the kernel's support, where W'(q) vanishes like
    # (2 - q)^2, lose relative precision to cancellation; bound every entry
    # relative to its row's diagonal
    scale = np.array([abs(adiag[k[0]]) for k in keys])
    assert np.all(np.abs(a - b) <= 1e-13 * scale)


# ---------------------------------------------------------------------------
# a5-a9: full steps
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precond", [sphrt.PRECOND_JACOBI, sphrt.PRECOND_CHEBYSHEV,
                                     sphrt.PRECOND_AMG])
def test_mms2d_full_run_parity(precond):
    # 2-D manufactured problem, 1,024 particles, 10 steps of dt = 1e-3
    w = I.mms_2d()
    r = run_both(w, w.steps, gpu_over=dict(precond=precond), orc_over=TIGHT)
    assert r["err_e"] < 1e-10 and r["err_E"] < 1e-10, (r["err_e"], r["err_E"])
    for g, o in zip(r["gstats"], r["ostats"]):
        assert g.outer_iters == o.outer_iters


def test_mms2d_parity_at_workload_tolerances():
    # the workload's own tolerances (outer 1e-10, Krylov 1e-12) on both sides
    w = I.mms_2d()
    r = run_both(w, w.steps)
    assert r["err_e"] < 1e-10 and r["err_E"] < 1e-10, (r["err_e"], r["err_E"])


@pytest.mark.parametrize("precond", [sphrt.PRECOND_CHEBYSHEV, sphrt.PRECOND_AMG])
def test_mms3d_levermore_parity(precond):
    w = I.mms_3d_lp(n=16, steps=3)
    r = run_both(w, 3, gpu_over=dict(precond=precond), orc_over=TIGHT)
    assert r["err_e"] < 1e-10 and r["err_E"] < 1e-10, (r["err_e"], r["err_E"])


def test_heating_wave_copy_ghosts_parity():
    w = I.heating_wave(3, 4000, 10.0, seed=21, steps=3)
    r = run_both(w, 3, orc_over=TIGHT)
    assert r["err_e"] < 1e-10 and r["err_E"] < 1e-10, (r["err_e"], r["err_E"])


def test_energy_balance_on_gpu():
    w = I.mms_2d(n=32, steps=3)
    r = run_both(w, 3, orc_over=TIGHT)
    for g, o in zip(r["gstats"], r["ostats"]):
        defect = g.energy_after - g.energy_before - g.source_energy - g.boundary_energy
        assert abs(defect) < 1e-11 * g.energy_after
        assert abs(g.energy_after - o.energy_after) < 1e-12 * o.energy_after


@pytest.mark.parametrize("precision,tol", [(sphrt.FP64, 1e-10), (sphrt.MIXED, 1e-8)])
def test_heterogeneous_sphere_parity(precision, tol):
    # dense opaque hot sphere (rho x10, sigma x1e3, T = 1) in a cold medium (T = 0.01): E spans
    # 8 decades.  Both solvers stop on ||b - A E|| <= tol ||b||, a norm-wise test, so the
    # cold entries (E ~ 1e-8) carry absolute errors ~tol ||b|| from either side: the
    # comparison is relative to max |E| (and elementwise for e, which spans 2 decades).
    w = I.sphere_3d(n=12, steps=2, dt=1e-4)
    r = run_both(w, 2, gpu_over=dict(precision=precision), orc_over=TIGHT)
    m = w.particles.kind == 0
    assert r["err_e"] < tol, r["err_e"]
    errE = np.max(np.abs(r["Eg"][m] - r["E"][m])) / np.max(np.abs(r["E"][m]))
    assert errE < tol, errE


@pytest.mark.parametrize("n,h,precond,precision,tol", [
    (10, 2.4, sphrt.PRECOND_JACOBI, sphrt.FP64, 1e-10),
    (10, 2.4, sphrt.PRECOND_CHEBYSHEV, sphrt.FP64, 1e-10),
    (10, 2.4, sphrt.PRECOND_AMG, sphrt.FP64, 1e-10),
    (10, 2.4, sphrt.PRECOND_AMG, sphrt.MIXED, 1e-8),
    (5, 1.5, sphrt.PRECOND_AMG, sphrt.FP64, 1e-10)])
def test_row_tile_shapes_parity(n, h, precond, precision, tol):
    # h = 2.4 dx: ~250 stored entries per row (84-463), so the SpMV-class sweeps, the
    # gradient and the assembly take their 8-lanes-per-row shape (8 rounds of 4 rows per
    # 32-row tile); 1,000 rows end in a ragged tile.  5^3 = 125 rows: 4 tiles, the last
    # with 29 rows, 4-lane shape.
    w = I.mms_3d_lp(n=n, steps=2, h_over_dx=h)
    r = run_both(w, 2, gpu_over=dict(precond=precond, precision=precision), orc_over=TIGHT)
    assert r["err_e"] < tol and r["err_E"] < tol, (r["err_e"], r["err_E"])


def _larsen_workload(n, k, steps):
    # 3-D manufactured problem with sigma = T^-3 and the Larsen limiter of exponent k
    # (Sec. 2.1; k = 2 is the paper's default), sources made with the same limiter
    w = I._mms_workload(f"mms3d-larsen{k:g}-{n}^3", 3, n, 2, -3.0, 2, 1e-3, steps)
    w.mms.larsen_k = k
    w.params["larsen_k"] = k
    return w


@pytest.mark.parametrize("k", [2.0, 3.0])
def test_larsen_properties_and_operator_match_oracle(k):
    # the Larsen branch of the limiter (k = 2: its square-root form) on the device
    w = _larsen_workload(8, k, 1)
    P = w.particles
    S = sphrt.solver_for(w, precond=sphrt.PRECOND_JACOBI)
    Qe, QE, ge, gE = w.step_inputs(1)
    S.step(w.dt, Qe, QE, ge, gE)
    pg = S.get_properties()
    po = O.Problem(P, w.params).properties(w.e0, w.E0, w.dt)
    m = P.kind == 0
    assert np.min(po["R"][m]) > 0.05  # the limiter is away from its R = 0 value
    for key in ("R", "lambda", "D"):
        np.testing.assert_allclose(pg[key][m], po[key][m], rtol=1e-13, atol=0, err_msg=key)


@pytest.mark.parametrize("k", [2.0, 3.0])
def test_larsen_full_steps_parity(k):
    w = _larsen_workload(16, k, 3)
    r = run_both(w, 3, orc_over=TIGHT)
    assert r["err_e"] < 1e-10 and r["err_E"] < 1e-10, (r["err_e"], r["err_E"])


@pytest.mark.parametrize("make,precision,tol", [
    (lambda: I.mms_3d(n=32, steps=3), sphrt.MIXED, 1e-8),
    (lambda: I.mms_3d_lp(n=32, steps=3), sphrt.MIXED, 1e-8),
    (lambda: I.mms_3d_lp(n=32, steps=3), sphrt.FP64, 1e-10)])
def test_parity_where_the_fine_level_takes_its_full_size_path(make, precision, tol):
    # 32^3 = 32,768 rows with ~101 stored entries each (3.3 M, above the 600k-entry
    # threshold): the finest level runs the A P post-smoothing sweep with the fused
    # inner product and the next level is summed from A P, in FP32 in the mixed
    # form -- the kernels of the 64^3 .. 256^3 workloads.  Element by element
    # against the oracle over 3 steps, for both manufactured physics (sigma = 1 with
    # lambda = 1/3, and sigma = T^-3 with the Levermore limiter).
    w = make()
    r = run_both(w, w.steps, gpu_over=dict(precision=precision, precond=sphrt.PRECOND_AMG),
                 orc_over=TIGHT)
    levels = r["S"].amg_info()
    assert levels[0][1] > 600_000 and len(levels) >= 3, levels
    assert r["err_e"] < tol and r["err_E"] < tol, (r["err_e"], r["err_E"])


@pytest.mark.parametrize("make,precision,tol", [
    (lambda: I.mms_2d(), sphrt.FP64, 1e-10),
    (lambda: I.mms_3d_lp(n=16, steps=3), sphrt.FP64, 1e-10),
    (lambda: I.mms_3d_lp(n=16, steps=3), sphrt.MIXED, 1e-8),
    (lambda: I.mms_3d(n=32, steps=3), sphrt.FP64, 1e-10),
    (lambda: I.mms_3d(n=32, steps=3), sphrt.MIXED, 1e-8),
    (lambda: I.mms_3d_lp(n=32, steps=3), sphrt.MIXED, 1e-8),
    (lambda: I.heating_wave(3, 4000, 10.0, seed=21, steps=3), sphrt.MIXED, 1e-8)])
def test_vcycle_product_cg_parity(make, precision, tol):
    # fine_post_smooth = 0: the finest level only pre-smooths and the CG takes
    # B p from the V-cycle's sweeps (flexible CG; in the mixed form FP32 vectors
    # with FP64 residual replacement).  16^3 takes the form without A P, 32^3
    # the A P sweep.  Same fixed point, same tolerances as the other forms.
    w = make()
    r = run_both(w, w.steps, gpu_over=dict(precision=precision, precond=sphrt.PRECOND_AMG,
                                           fine_post_smooth=0), orc_over=TIGHT)
    assert r["err_e"] < tol and r["err_E"] < tol, (r["err_e"], r["err_E"])
    for g, o in zip(r["gstats"], r["ostats"]):
        assert g.outer_iters == o.outer_iters


@pytest.mark.parametrize("drop", [0.5, 1e-2, 1e-4, 1e-6])
def test_vcycle_product_cg_stops_on_the_fp64_residual(drop):
    # whatever the replacement interval, the mixed solve stops only when the FP64
    # residual meets the tolerance: the energies agree with the FP64 form's
    w = I.mms_3d(n=32, steps=2)
    ref = run_both(w, 2, gpu_over=dict(precond=sphrt.PRECOND_AMG), orc_over=TIGHT)
    S = sphrt.solver_for(w, **dict(w.params, **TIGHT), precision=sphrt.MIXED,
                         fine_post_smooth=0, reliable_drop=drop)
    for n in (1, 2):
        S.step(w.dt, *w.step_inputs(n))
    eg, Eg, _ = S.get_energies()
    m = w.particles.kind == 0
    assert rel_err(eg, ref["e"], m) < 1e-8 and rel_err(Eg, ref["E"], m) < 1e-8


# ---------------------------------------------------------------------------
# the paper's discretisation: Wendland C4 with h = 4 dx (support h), the cgs
# manufactured problem of Sec. 4.3 with periodic copy ghosts, Larsen limiter,
# scattering opacity
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("make", [
    lambda: I.mms_cgs(2, 16, steps=3, jitter=0.0),
    lambda: I.mms_cgs(2, 16, steps=3),
    lambda: I.mms_cgs(3, 10, steps=2),
    lambda: I.mms_cgs(1, 64, steps=5)])
def test_wendland_neighbors_bit_exact(make):
    w = make()
    P = w.particles
    S = sphrt.solver_for(w)
    rp, cols = S.get_neighbors()
    orp, ocols = O.neighbors(P.pos, P.h, P.kind, kernel=1)
    assert np.array_equal(rp, orp) and np.array_equal(cols, ocols.astype(np.int64))


def test_wendland_properties_and_operator_match_oracle():
    w = I.mms_cgs(2, 16, steps=1)
    P = w.particles
    S = sphrt.solver_for(w, precond=sphrt.PRECOND_JACOBI)
    Qe, QE, ge, gE = w.step_inputs(1)
    S.step(w.dt, Qe, QE, ge, gE)
    pg = S.get_properties()
    pb = O.Problem(P, w.params)
    po = pb.properties(w.e0, w.E0, w.dt)
    m = P.kind == 0
    for k in ("sigma", "f", "R", "lambda", "D"):
        np.testing.assert_allclose(pg[k][m], po[k][m], rtol=1e-13, atol=0, err_msg=k)
    arow, acol, aval, adiag, gb = pb.assemble(po, w.dt, w.E0)
    rowptr, cols, vals, diag, ggb = S.get_operator()
    np.testing.assert_allclose(diag[m], adiag[m], rtol=1e-13)
    dg = {k: v for k, v in _operator_dict(rowptr, cols, vals, diag).items() if k[0] != k[1]}
    do = _operator_dict(arow, acol, aval, adiag)
    assert set(dg) == set(do)
    keys = sorted(do)
    err = np.array([abs(dg[k] - do[k]) / abs(adiag[k[0]]) for k in keys])
    assert np.all(err <= 1e-13)


@pytest.mark.parametrize("make,precision,tol", [
    (lambda: I.mms_cgs(2, 16, steps=4), sphrt.FP64, 1e-10),
    (lambda: I.mms_cgs(2, 32, steps=3), sphrt.FP64, 1e-10),
    (lambda: I.mms_cgs(3, 12, steps=2), sphrt.FP64, 1e-10),
    (lambda: I.mms_cgs(3, 12, steps=2), sphrt.MIXED, 1e-8),
    (lambda: I.mms_cgs(1, 64, steps=6), sphrt.FP64, 1e-10)])
def test_cgs_manufactured_parity(make, precision, tol):
    w = make()
    r = run_both(w, w.steps, gpu_over=dict(precision=precision), orc_over=TIGHT)
    assert r["err_e"] < tol and r["err_E"] < tol, (r["err_e"], r["err_E"])
    for g, o in zip(r["gstats"], r["ostats"]):
        assert g.outer_iters == o.outer_iters
        # periodic: no boundary flux; the energy changes by the sources alone
        assert abs(g.boundary_energy) <= 1e-14 * g.energy_after
        defect = g.energy_after - g.energy_before - g.source_energy
        assert abs(defect) <= 1e-12 * g.energy_after


def test_mixed_precision_parity():
    w = I.mms_3d_lp(n=16, steps=3)
    r = run_both(w, 3, gpu_over=dict(precision=sphrt.MIXED, precond=sphrt.PRECOND_AMG),
                 orc_over=TIGHT)
    assert r["err_e"] < 1e-8 and r["err_E"] < 1e-8, (r["err_e"], r["err_E"])


# ---------------------------------------------------------------------------
# determinism, restart, failure handling, device entry points
# ---------------------------------------------------------------------------
def test_repeat_is_bitwise_identical():
    w = I.mms_3d_lp(n=12, steps=2)
    outs = []
    for _ in range(2):
        S = sphrt.solver_for(w)
        for n in (1, 2):
            S.step(w.dt, *w.step_inputs(n))
        outs.append(S.get_energies())
        S.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("krylov_start", [0, 1, 2, 3])
def test_restart_continues_bitwise(krylov_start):
    # a checkpoint is the state (e, E) and, for the extrapolated Krylov start,
    # its history (E^{n-2}, E^{n-3}, ... and their steps' dt)
    w = I.mms_2d(n=16, steps=5)
    P = w.particles
    m = P.kind == 0

    def run(steps):
        S = sphrt.solver_for(w, amg_rebuild=1, krylov_start=krylov_start)
        for n in range(1, steps + 1):
            S.step(w.dt, *w.step_inputs(n))
        return S

    S = run(5)
    e5, E5, _ = S.get_energies()
    S2 = run(4)
    e4, E4, _ = S2.get_energies()
    Eh, dth = S2.get_history()
    assert len(dth) == krylov_start and Eh.shape == (krylov_start, P.n)
    assert np.all(dth == w.dt)
    S3 = sphrt.Solver(sphrt.config_from_params(w.params, amg_rebuild=1,
                                               krylov_start=krylov_start))
    S3.set_particles(P.pos, P.mass, P.rho, P.h, P.sigma0, P.kind, None, e4, E4)
    assert len(S3.get_history()[1]) == 0  # new particles: no history yet
    if krylov_start:
        S3.set_history(Eh, dth)
    S3.step(w.dt, *w.step_inputs(5))
    e5b, E5b, _ = S3.get_energies()
    assert np.array_equal(e5, e5b) and np.array_equal(E5, E5b)
    # row j is E^{n-2-j}: the state three, two, one steps in (interior entries)
    for j in range(krylov_start):
        R = run(3 - j)
        assert np.array_equal(Eh[j][m], R.get_energies()[1][m]) and np.all(Eh[j][~m] == 0.0)
        R.close()
    if krylov_start:
        with pytest.raises(sphrt.SphRtError) as ei:
            S3.set_history(Eh, np.zeros(krylov_start))
        assert ei.value.status == sphrt.EINVAL
        bad = Eh.copy()
        bad[0, 0] = np.nan
        with pytest.raises(sphrt.SphRtError) as ei:
            S3.set_history(bad, dth)
        assert ei.value.status == sphrt.EINVAL
    if krylov_start < 3:  # deeper than the configuration reads
        with pytest.raises(sphrt.SphRtError) as ei:
            S3.set_history(np.ones((krylov_start + 1, P.n)), np.ones(krylov_start + 1))
        assert ei.value.status == sphrt.EINVAL
    for h in (S, S2, S3):
        h.close()


def test_not_converged_leaves_state_unchanged():
    w = I.mms_2d(n=16)
    S = sphrt.solver_for(w, max_outer=1, tol_outer_e=1e-15, tol_outer_E=1e-15)
    e0, E0, _ = S.get_energies()
    rc, st = S.step(w.dt, *w.step_inputs(1), raise_on_error=False)
    assert rc == sphrt.ENOTCONV
    e1, E1, _ = S.get_energies()
    assert np.array_equal(e0, e1) and np.array_equal(E0, E1)
    # Krylov limit too
    S2 = sphrt.solver_for(w, max_krylov=1, precond=sphrt.PRECOND_JACOBI)
    rc, st = S2.step(w.dt, *w.step_inputs(1), raise_on_error=False)
    assert rc == sphrt.ENOTCONV and "Krylov" in S2.last_error()


def test_device_entry_points_match_host():
    torch = pytest.importorskip("torch")
    w = I.mms_2d(n=16, steps=2)
    P = w.particles
    S = sphrt.solver_for(w)
    for n in (1, 2):
        S.step(w.dt, *w.step_inputs(n))
    eh, Eh, _ = S.get_energies()
    dev = torch.device("cuda:0")
    T = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    arrs = [T(P.pos), T(P.mass), T(P.rho), T(P.h), T(P.sigma0), T(P.kind, torch.int32), None,
            T(w.e0), T(w.E0)]
    S2 = sphrt.Solver(sphrt.config_from_params(w.params))
    torch.cuda.synchronize()
    S2.set_particles_device(P.n, *[a.data_ptr() if a is not None else 0 for a in arrs])
    for n in (1, 2):
        ins = [T(a) for a in w.step_inputs(n)]
        torch.cuda.synchronize()
        S2.step_device(w.dt, *[a.data_ptr() for a in ins])
    e_out = torch.empty(P.n, dtype=torch.float64, device=dev)
    E_out = torch.empty(P.n, dtype=torch.float64, device=dev)
    S2.get_energies_device(e_out.data_ptr(), E_out.data_ptr())
    S2_e, S2_E, _ = S2.get_energies()
    assert np.array_equal(S2_e, eh) and np.array_equal(S2_E, Eh)
    torch.cuda.synchronize()
    assert np.array_equal(e_out.cpu().numpy(), eh)


# ---------------------------------------------------------------------------
# the benchmark's workload at full size: 64^3 manufactured problem, Levermore
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def full_size():
    w = I.mms_3d_lp(n=64, steps=100)
    S = sphrt.solver_for(w)
    return w, S


def test_full_size_neighbors_sampled(full_size):
    w, S = full_size
    P = w.particles
    rp, cols = S.get_neighbors()
    rng = np.random.default_rng(0)
    interior = np.flatnonzero(P.kind == 0)
    rows = np.concatenate([rng.choice(interior, 48, replace=False), interior[:8], interior[-8:]])
    orp, ocols = O.neighbors_of_rows(P.pos, P.h, rows)
    for k, i in enumerate(rows):
        assert np.array_equal(cols[rp[i]:rp[i + 1]], ocols[orp[k]:orp[k + 1]].astype(np.int64))
    n_int, nnz_nbr, nnz_op = S.sizes()
    assert n_int == 64**3 and 28_000_000 < nnz_nbr < 31_000_000


def test_full_size_two_steps_match_oracle(full_size):
    w, S = full_size
    prm = dict(w.params, **TIGHT)
    S2 = sphrt.solver_for(w, **TIGHT)
    pb = O.Problem(w.particles, prm)
    e, E = w.e0.copy(), w.E0.copy()
    for n in (1, 2):
        ins = w.step_inputs(n)
        S2.step(w.dt, *ins)
        rc, e, E, _ = pb.step(e, E, w.dt, *ins)
        assert rc == 0
    eg, Eg, _ = S2.get_energies()
    m = w.particles.kind == 0
    assert rel_err(eg, e, m) < 1e-10 and rel_err(Eg, E, m) < 1e-10


def test_non_finite_step_input_is_rejected_without_state_change():
    w = I.mms_2d(n=16)
    S = sphrt.solver_for(w)
    e0, E0, _ = S.get_energies()
    Qe, QE, ge, gE = w.step_inputs(1)
    QE = QE.copy()
    QE[np.flatnonzero(w.particles.kind == 0)[5]] = np.nan
    rc, st = S.step(w.dt, Qe, QE, ge, gE, raise_on_error=False)
    assert rc == sphrt.EINVAL and "non-finite" in S.last_error()
    e1, E1, _ = S.get_energies()
    assert np.array_equal(e0, e1) and np.array_equal(E0, E1)
    # a NaN on a ghost entry of a source array is ignored (ghost sources are unused)
    QE2 = w.step_inputs(1)[1].copy()
    QE2[np.flatnonzero(w.particles.kind == 1)[0]] = np.nan
    rc, st = S.step(w.dt, Qe, QE2, ge, gE, raise_on_error=False)
    assert rc == sphrt.OK
