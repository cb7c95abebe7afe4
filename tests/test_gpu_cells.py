"""Size limits.  Neighbour search cell lists (row a1): the sorted 64-bit-key
list (radix sort, hash table of occupied cells) gives the same slots,
neighbour lists and steps as the dense key table, bit for bit, and takes grids
the dense table refuses (more than 2^26 cells), where it still matches the
brute-force oracle.  The AMG set-up's 64-bit source lists (for more than
2^31 - 1 entries) change no bit."""
import numpy as np
import pytest

import oracle as O
from paper_2001_11606_gb300 import inputs as I
from paper_2001_11606_gb300 import sphrt

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_krylov=1e-14, tol_outer_e=1e-12, tol_outer_E=1e-12, tol_inner_e=1e-14)


@pytest.mark.parametrize("make", [lambda: I.mms_2d(n=32), lambda: I.mms_3d_lp(n=12),
                                  lambda: I.heating_wave(2, 3000, 5.0, seed=9, steps=2),
                                  lambda: I.heating_wave(3, 3000, 5.0, seed=9, steps=2),
                                  lambda: I.mms_cgs(3, 8, steps=2)])
def test_sorted_cells_equal_dense_table(make):
    w = make()
    out = []
    for cells in (sphrt.CELLS_DENSE, sphrt.CELLS_SORTED):
        S = sphrt.solver_for(w, cell_list=cells)
        rp, cols = S.get_neighbors()
        for n in range(1, 3):
            Qe, QE, ge, gE = w.step_inputs(n)
            S.step(w.dt, Qe, QE, ge, gE)
        e, E, _ = S.get_energies()
        out.append((rp, cols, e, E))
        S.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def _far_blocks(dim, shift_cells, seed=3):
    """Two 12^dim lattices (Dirichlet ghosts) shift_cells cell widths apart along x."""
    P = I.make_lattice(dim, (12,) * dim, 1.0 / 12, seed=seed)
    Q = I.make_lattice(dim, (12,) * dim, 1.0 / 12, seed=seed + 1)
    cell = 2.0 * float(np.max(P.h))
    off = np.zeros(dim)
    off[0] = shift_cells * cell
    cat = lambda a, b: np.concatenate([a, b])
    R = I.Particles(dim=dim, dx=P.dx, counts=P.counts, pos=cat(P.pos, Q.pos + off),
                    kind=cat(P.kind, Q.kind), copy_of=np.full(P.n + Q.n, -1, dtype=np.int64),
                    mass=cat(P.mass, Q.mass), rho=cat(P.rho, Q.rho), h=cat(P.h, Q.h),
                    sigma0=cat(P.sigma0, Q.sigma0))
    x = R.pos[:, 0] - np.floor(R.pos[:, 0])
    T = 1.0 + 0.3 * np.sin(np.pi * x)
    prm = dict(dim=dim, a=1.0, c=1.0, cv=1.0, limiter=1, larsen_k=2.0, opacity_exp=0.0,
               T_floor=0.0, max_outer=50, max_inner_e=50, max_krylov=4000, **TIGHT)
    return I.Workload(f"far{dim}d", R, prm, 1e-3, 2, e0=T.copy(), E0=T**4)


@pytest.mark.parametrize("dim,shift", [(2, 20000.0), (3, 70000.0)])
def test_sorted_cells_take_grids_beyond_the_dense_table(dim, shift):
    w = _far_blocks(dim, shift)
    P = w.particles
    with pytest.raises(sphrt.SphRtError) as ex:
        sphrt.solver_for(w, cell_list=sphrt.CELLS_DENSE)
    assert ex.value.status == sphrt.EINVAL and "dense cell table" in str(ex.value)
    S = sphrt.solver_for(w)  # AUTO takes the sorted list here
    rp, cols = S.get_neighbors()
    orp, ocols = O.neighbors(P.pos, P.h, P.kind)
    assert np.array_equal(rp, orp) and np.array_equal(cols, ocols.astype(np.int64))
    pb = O.Problem(P, w.params)
    e, E = w.e0.copy(), w.E0.copy()
    for _ in range(2):
        S.step(w.dt)
        rc, e, E, _ = pb.step(e, E, w.dt)
        assert rc == 0
    eg, Eg, _ = S.get_energies()
    m = P.kind == 0
    assert np.max(np.abs(eg[m] - e[m]) / np.abs(e[m])) < 1e-10
    assert np.max(np.abs(Eg[m] - E[m]) / np.abs(E[m])) < 1e-10
    S.close()


def test_grid_beyond_2_29_cells_along_an_axis_is_refused():
    w = _far_blocks(3, 2.0**30)
    with pytest.raises(sphrt.SphRtError) as ex:
        sphrt.solver_for(w)
    assert ex.value.status == sphrt.EINVAL and "2^29" in str(ex.value)


# 64-bit Galerkin source lists (taken automatically for a level with 2^31 - 1
# or more entries plus rows) give the same hierarchy and steps as 32-bit ones
@pytest.mark.parametrize("over", [dict(precision=sphrt.FP64),
                                  dict(precision=sphrt.MIXED),
                                  dict(precision=sphrt.MIXED, fine_post_smooth=0,
                                       reliable_drop=1e-6)])
def test_index64_source_lists_change_no_bit(over):
    w = I.mms_3d_lp(n=24, steps=2)
    out = []
    for wide in (0, 1):
        S = sphrt.solver_for(w, index64=wide, **over)
        for n in range(1, 3):
            Qe, QE, ge, gE = w.step_inputs(n)
            S.step(w.dt, Qe, QE, ge, gE)
        e, E, _ = S.get_energies()
        out.append((e, E))
        S.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_beyond_2_31_neighbour_pairs_and_operator_entries():
    """280^3 manufactured problem: 2.35e9 neighbour pairs and 2.32e9 operator
    entries (both past 2^31, so the AMG lists are 64-bit); sampled neighbour
    rows match the brute-force oracle bit for bit and a step converges.  Needs
    about 175 GB of device memory."""
    torch = pytest.importorskip("torch")
    free, _ = torch.cuda.mem_get_info()
    if free < 200e9:
        pytest.skip(f"needs ~175 GB of free device memory ({free / 1e9:.0f} GB free)")
    w = I.mms_3d(n=280, steps=1)
    P = w.particles
    S = sphrt.solver_for(w)
    n_int, nnz_nbr, nnz_op = S.sizes()
    assert n_int == 280**3 and nnz_nbr > 2**31 and nnz_op + n_int > 2**31
    rp, cols = S.get_neighbors()
    rng = np.random.default_rng(1)
    interior = np.flatnonzero(P.kind == 0)
    rows = np.concatenate([rng.choice(interior, 16, replace=False), interior[:4], interior[-4:]])
    orp, ocols = O.neighbors_of_rows(P.pos, P.h, rows)
    for k, i in enumerate(rows):
        assert np.array_equal(cols[rp[i]:rp[i + 1]], ocols[orp[k]:orp[k + 1]].astype(np.int64))
    del rp, cols
    rc, st = S.step(w.dt, *w.step_inputs(1))
    assert rc == 0 and 1 <= st.outer_iters <= 4
    e, E, _ = S.get_energies()
    assert np.all(np.isfinite(E)) and np.all(E[P.kind == 0] > 0)
    S.close()
