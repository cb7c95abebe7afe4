"""The allocation-free entry point (include/sph_rt_noalloc.h).

Callers that cannot let the library allocate device memory -- their framework
owns the device through its own allocator, or cudaMalloc/cudaFree (which
synchronise the device) are forbidden in the region they run in -- compute
the interior energy totals with sph_rt_energy_totals_noalloc, whose scratch
is a fixed array in the library's static device memory.  The GPU tests check
it, through the C ABI, against the totals of sph_rt_get_energies and against
float64 sums on the host, each on two calls in a row (the shared scratch must
be left ready for the next call), at sizes that use a few blocks, more blocks
than the combining block has threads, and the largest accepted size.  The
rejections need no GPU: they happen before any device call.  The file is
named to run last, so a failure here never hides the other GPU tests.
"""
import numpy as np
import pytest

from paper_2001_11606_gb300 import inputs as I
from paper_2001_11606_gb300 import sphrt

RTOL = 1e-12  # the same quantities summed in a different order


def _call(n, ptrs, out, stream):
    rc = sphrt.energy_totals_noalloc(n, *ptrs, out, stream)
    assert rc == sphrt.OK, sphrt.last_thread_error()


@pytest.mark.gpu
def test_noalloc_totals_match_get_energies_twice():
    torch = pytest.importorskip("torch")
    w = I.mms_3d_lp(n=24, steps=2)
    P = w.particles
    S = sphrt.solver_for(w)
    for n in (1, 2):
        S.step(w.dt, *w.step_inputs(n))
    e, E, totals = S.get_energies()  # existing entry point
    dev = torch.device("cuda:0")
    f64 = dict(dtype=torch.float64, device=dev)
    d = [torch.as_tensor(P.kind, dtype=torch.int32, device=dev)]
    d += [torch.as_tensor(a, **f64) for a in (P.mass, P.rho, e, E)]
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        out = torch.full((2,), float("nan"), **f64)
        _call(P.n, [t.data_ptr() for t in d], out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize(dev)
        np.testing.assert_allclose(out.cpu().numpy(), totals, rtol=RTOL, err_msg=f"call {call}")
    S.close()


@pytest.mark.gpu
@pytest.mark.parametrize("n", [3_000_001, sphrt.NOALLOC_MAX_N])
def test_noalloc_totals_on_large_grids(n):
    # 367 blocks (more than the 256 threads of the combining block, so each
    # folds several partials) and the full 4096-block grid of the largest size
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(n)
    kind = rng.choice(np.array([0, 0, 0, 1, 2], dtype=np.int32), size=n)
    mass, rho, e, E = (rng.uniform(0.5, 2.0, n) for _ in range(4))
    inner = kind == 0
    want = np.array([np.sum(mass[inner] * e[inner]), np.sum(mass[inner] / rho[inner] * E[inner])])
    dev = torch.device("cuda:0")
    d = [torch.from_numpy(kind).to(dev)] + [torch.from_numpy(a).to(dev) for a in (mass, rho, e, E)]
    del mass, rho, e, E
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
        _call(n, [t.data_ptr() for t in d], out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize(dev)
        np.testing.assert_allclose(out.cpu().numpy(), want, rtol=RTOL, err_msg=f"call {call}")


def test_noalloc_rejects_sizes_beyond_its_scratch():
    # n_total is checked before any pointer is touched or any device call is made
    for n in (sphrt.NOALLOC_MAX_N + 1, 0, -5):
        rc = sphrt.energy_totals_noalloc(n, 0, 0, 0, 0, 0, 0)
        assert rc == sphrt.EINVAL
        assert "n_total" in sphrt.last_thread_error()


def test_noalloc_rejects_null_arrays():
    # any NULL array is rejected before any device call (the other pointers are
    # never dereferenced on the host)
    for k in range(6):
        ptrs = [8] * 6
        ptrs[k] = 0
        rc = sphrt.energy_totals_noalloc(16, *ptrs)
        assert rc == sphrt.EINVAL
        assert "NULL" in sphrt.last_thread_error()
