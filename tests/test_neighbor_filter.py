"""CPU check of the neighbour search's FP32 pre-filter (neighbors.cu).

The kernel decides a candidate pair in FP32 from cell-relative positions when
its squared distance is farther than kNbrBand cell^2 from the cut, and with the
exact FP64 predicate otherwise.  This restates that FP32 arithmetic in numpy
(float32, no fused multiply-add) on every candidate pair of sampled rows and
checks (a) that the FP32 squared distances stay far inside the band (the
bound derived in the kernel's comment is ~2.4e-6 cell^2; the band is 3e-5), and
(b) that no pair decided in FP32 disagrees with the exact predicate.
"""
import numpy as np
import pytest

from paper_2001_11606_gb300 import inputs as I

BAND = 3e-5  # kNbrBand


def _filter_stats(P, rows=300, seed=0):
    pos = P.pos
    n, dim = pos.shape
    p3 = np.zeros((n, 3))
    p3[:, :dim] = pos
    h = P.h
    lo = p3.min(axis=0)
    cell = 2.0 * h.max() * (1.0 + 1e-9)
    nc = [(int((p3[:, d].max() - lo[d]) / cell) + 1) if d < dim else 1 for d in range(3)]
    c = np.clip(np.floor((p3 - lo) * (1.0 / cell)).astype(np.int64), 0, np.array(nc) - 1)
    rel = (p3 - (lo + c * cell)).astype(np.float32)
    rel[:, dim:] = 0.0
    c2f = ((2.0 * h) * (2.0 * h)).astype(np.float32)
    cellf = np.float32(cell)
    band = np.float32(BAND) * cellf * cellf
    inter = np.flatnonzero(P.kind == 0)
    pick = np.random.default_rng(seed).choice(inter, min(rows, len(inter)), replace=False)
    worst, wrong, amb, tot = 0.0, 0, 0, 0
    for i in pick:
        o = c - c[i]
        near = np.all(np.abs(o) <= 1, axis=1)
        near[i] = False
        js = np.flatnonzero(near)
        d = ((rel[i] - rel[js]) + (-o[js].astype(np.float32) * cellf)).astype(np.float32)
        r2f = ((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]).astype(np.float32) + d[:, 2] * d[:, 2])
        r2f = r2f.astype(np.float32)
        dx = p3[i] - p3[js]
        r2 = dx[:, 0] * dx[:, 0] + dx[:, 1] * dx[:, 1] + dx[:, 2] * dx[:, 2]
        cut = 2.0 * np.maximum(h[i], h[js])
        exact = r2 < cut * cut
        cf = np.maximum(c2f[i], c2f[js])
        m = r2 < 1.5 * cut * cut
        if np.any(m):
            worst = max(worst, float(np.max(np.abs(r2f.astype(np.float64) - r2)[m]) / cell**2))
        sure_in = r2f < cf - band
        sure_out = r2f > cf + band
        wrong += int(np.count_nonzero(sure_in & ~exact) + np.count_nonzero(sure_out & exact))
        amb += int(np.count_nonzero(~sure_in & ~sure_out))
        tot += len(js)
    return worst, wrong, amb, tot


@pytest.mark.parametrize("make", [
    lambda: I.mms_3d_lp(n=24).particles,
    lambda: I.mms_2d(n=48).particles,
    lambda: I.heating_wave(3, 3000, 5.0, seed=9).particles,
    lambda: I.make_lattice(3, (9, 7, 5), 1.0 / 64, seed=0, jitter=0.0),
])
def test_fp32_prefilter_is_exact_and_inside_its_band(make):
    worst, wrong, amb, tot = _filter_stats(make())
    assert wrong == 0
    assert worst < BAND / 20, worst
    assert amb < 0.05 * tot


def test_fp32_prefilter_with_varied_h():
    P = I.mms_3d_lp(n=12).particles
    P.h = P.h * np.random.default_rng(4).uniform(0.7, 1.3, P.n)
    worst, wrong, amb, tot = _filter_stats(P)
    assert wrong == 0 and worst < BAND / 20 and amb < 1e-3 * tot
