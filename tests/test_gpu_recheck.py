"""The recheck tiers (certified FP32 -> double-word enclosure -> FP64) against
the FP64 oracle.

A `band` widens the FP32 undecided zone so that a large share of the extremes
goes through the double-word tier; the decisions must still equal the
oracle's bit for bit, and FP64 must be needed only where an enclosure holds a
grid line (exact ties, as in the doubling map)."""
import numpy as np
import pytest

from paper_2202_06111_gb300 import workloads as W
from test_gpu_parity import gis, run_both  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _totals(res):
    st = res[-1][1]
    return st["cum_recheck"], st["cum_recheck_fp64"], st["cum_recheck_samples"]


@pytest.mark.parametrize("band", [0.0, 0.2])
def test_cstr_band_double_word(gis, band):
    res = run_both(gis, dict(W.cstr_256(levels=2, n0=31), rule="inner"), 2, band=band)
    rc, r64, ns = _totals(res)
    assert rc > 0 and ns > 0
    assert r64 <= 0.02 * rc + 2, f"{r64} of {rc} rechecked pairs needed FP64"


def test_vdp_band_double_word(gis):
    res = run_both(gis, dict(W.vdp_64(), precision="fp32", rule="outer"), 1, band=0.2)
    rc, r64, _ = _totals(res)
    assert rc > 100
    assert r64 <= 0.02 * rc + 2


def test_cartpole_band_double_word(gis):
    """sin / cos enclosures (4-D)."""
    res = run_both(gis, dict(W.cartpole_48(levels=1, n0=6), rule="outer"), 1, band=0.2)
    rc, r64, _ = _totals(res)
    assert rc > 100
    assert r64 <= 0.02 * rc + 2


def test_cstr_paper_fp32(gis):
    """Eq. 4 CSTR, FP32 with the recheck tiers. In the hot corner the explicit
    RK4 step blows up (images of 1e17 .. 1e65): beyond the FP32 exponent range
    of the double words, so those pairs are computed in FP64, which also
    settles whether the FP64 image is finite."""
    prob = dict(W.cstr_paper_problem(n0=(16, 16), levels=1), precision="fp32", rule="outer")
    res = run_both(gis, prob, 1)
    rc, r64, _ = _totals(res)
    assert rc > 0 and r64 <= rc


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_linear_band_double_word(gis, n):
    rng = np.random.default_rng(100 + n)
    A = (np.eye(n) * 1.05 + rng.uniform(-0.2, 0.2, (n, n))).tolist()
    B = rng.uniform(-0.5, 0.5, (n, 1)).tolist()
    prob = W.problem(W.linmap(A, B), [-1.3] * n, [1.7] * n, [9, 7, 5, 3][:n], 3 if n < 4 else 2,
                     W.controls_grid(-0.4, 0.3, 4), 1.0, 0, rule="outer", precision="fp32")
    run_both(gis, prob, 1, band=0.2)


def test_doubling_map_ties_reach_fp64(gis):
    """x+ = 2x + u puts images exactly on grid lines: their enclosures hold the
    line, so those pairs are computed in FP64."""
    prob = W.problem(W.linmap([[2.0]], [[1.0]]), [-1.0], [1.0], 16, 2, [[-0.5], [0.0], [0.5]], 1.0, 0,
                     rule="outer", precision="fp32")
    res = run_both(gis, prob, 1)
    rc, r64, _ = _totals(res)
    assert r64 > 0


@pytest.mark.parametrize("store", [1, 2])
def test_enclosure_store_dense_and_compact(gis, store):
    """The FP64 enclosures of rechecked extremes, dense per (cell, control) or in
    the compact store, give the same graphs (band widens the recheck)."""
    res = run_both(gis, dict(W.cstr_256(levels=2, n0=23), rule="inner"), 2, band=0.2, enclosure_store=store)
    rc, _, _ = _totals(res)
    assert rc > 0


def test_cartpole_compact_store(gis):
    """4-D with the compact store (the default for large grids)."""
    run_both(gis, dict(W.cartpole_48(levels=1, n0=6), rule="outer"), 1, band=0.1, enclosure_store=2)
