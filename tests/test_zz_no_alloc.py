"""The allocation-free entry point (include/sph_rt_noalloc.h).

Callers that cannot let the library allocate device memory -- their framework
owns the device through its own allocator, or cudaMalloc/cudaFree (which
synchronise the device) are forbidden in the region they run in -- compute
the interior energy totals with sph_rt_energy_totals_noalloc, whose scratch
is a fixed array in the library's static device memory.  This checks it,
through the C ABI, against the totals of sph_rt_get_energies on two calls in a
row (the shared scratch must be left ready for the next call).  The file is
named to run last, so a failure here never hides the other GPU tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2001_11606_gb300 import inputs as I
from paper_2001_11606_gb300 import sphrt

pytestmark = pytest.mark.gpu

RTOL = 1e-12  # same quantities summed in a different order


def _lib():
    L = sphrt.load()
    fn = L.sph_rt_energy_totals_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_int64] + [C.c_void_p] * 7
    return fn


def test_noalloc_totals_match_get_energies_twice():
    torch = pytest.importorskip("torch")
    fn = _lib()
    w = I.mms_3d_lp(n=24, steps=2)
    P = w.particles
    S = sphrt.solver_for(w)
    for n in (1, 2):
        S.step(w.dt, *w.step_inputs(n))
    e, E, totals = S.get_energies()  # existing entry point
    dev = torch.device("cuda:0")
    f64 = dict(dtype=torch.float64, device=dev)
    d_kind = torch.as_tensor(P.kind, dtype=torch.int32, device=dev)
    d_mass, d_rho = torch.as_tensor(P.mass, **f64), torch.as_tensor(P.rho, **f64)
    d_e, d_E = torch.as_tensor(e, **f64), torch.as_tensor(E, **f64)
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        out = torch.full((2,), float("nan"), **f64)
        rc = fn(P.n, d_kind.data_ptr(), d_mass.data_ptr(), d_rho.data_ptr(), d_e.data_ptr(),
                d_E.data_ptr(), out.data_ptr(), stream.cuda_stream)
        assert rc == sphrt.OK, sphrt.load().sph_rt_last_error(None)
        torch.cuda.synchronize(dev)
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, totals, rtol=RTOL, err_msg=f"call {call}")
    S.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    fn = _lib()
    max_n = 4096 * 8192
    rc = fn(max_n + 1, 1, 1, 1, 1, 1, 1, None)  # rejected before any pointer is used
    assert rc == sphrt.EINVAL
    assert b"n_total" in sphrt.load().sph_rt_last_error(None)
