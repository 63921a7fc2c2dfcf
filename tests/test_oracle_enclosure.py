"""Pins of the oracle's interval enclosure of a cell's image (NEXT f3): it
holds the images of every point of the closed cell (checked on corners and
random points, every model), is the exact affine image for a linear discrete
map (up to the outward ulps), and contains the sampled box, so the graph built
from it contains the sampled graph's edges."""
import numpy as np
import pytest

from paper_2202_06111_gb300 import workloads as W


def _cases():
    return [
        ("vdp", W.problem(W.vdp(1.0), [-3, -3], [3, 3], 8, 3, W.controls_grid(-1, 1, 3), 0.1, 10)),
        ("cstr_dl", W.cstr_256(levels=0, n0=16)),
        ("cartpole", W.cartpole_48(levels=0, n0=6)),
        ("cstr_paper", W.cstr_paper_problem(n0=(8, 8))),
        ("linear_rk4", W.problem(W.linmap([[0.1, 1.0], [-0.9, -0.2]], [[0.0], [1.0]]), [-1, -1], [1, 1], 6, 2,
                                 W.controls_grid(-0.5, 0.5, 3), 0.3, 3)),
    ]


def _cell(prob, L, idx):
    lo = np.array(prob["lo"], float)
    w = (np.array(prob["hi"], float) - lo) / (np.array(prob["n0"], float) * 2.0 ** L)
    return lo + np.asarray(idx) * w, lo + (np.asarray(idx) + 1) * w


@pytest.mark.parametrize("name,prob", _cases(), ids=[c[0] for c in _cases()])
def test_enclosure_holds_every_point_of_the_cell(orc, name, prob):
    rng = np.random.default_rng(3)
    p = dict(prob, enclosure="interval")
    n = prob["n"]
    checked = 0
    for trial in range(12):
        L = int(rng.integers(0, 3))
        idx = [int(rng.integers(0, prob["n0"][d] << L)) for d in range(n)]
        u = np.asarray(prob["controls"][int(rng.integers(len(prob["controls"])))], float)
        lo, hi, nf = orc.pair_bbox(p, L, idx, u)
        if nf:
            continue
        a, b = _cell(prob, L, idx)
        pts = [a + (b - a) * np.array([(c >> d) & 1 for d in range(n)], float) for c in range(1 << n)]
        pts += [a + (b - a) * rng.uniform(size=n) for _ in range(200)]
        for x in pts:
            y = np.asarray(orc.step(prob, x, u))
            tol = 1e-12 * (1.0 + np.abs(y))
            assert np.all(y >= lo - tol) and np.all(y <= hi + tol), (name, L, idx, x, y, lo, hi)
        slo, shi, snf = orc.pair_bbox(prob, L, idx, u)      # the sampled box lies inside
        if not snf:
            assert np.all(lo <= slo) and np.all(shi <= hi)
        checked += 1
    assert checked >= 6


def test_enclosure_of_a_linear_map_is_its_exact_image(orc):
    A = np.array([[0.7, -1.3], [0.4, 1.1]])
    B = np.array([[0.5], [-0.25]])
    prob = dict(W.problem(W.linmap(A.tolist(), B.tolist()), [-2, -1], [2, 3], [5, 7], 2, [[0.3]], 1.0, 0),
                enclosure="interval")
    for L, idx in [(0, [0, 0]), (1, [3, 9]), (2, [17, 5])]:
        lo, hi, nf = orc.pair_bbox(prob, L, idx, np.array([0.3]))
        a, b = _cell(prob, L, idx)
        c, r = (a + b) / 2, (b - a) / 2
        want_lo = A @ c - np.abs(A) @ r + B[:, 0] * 0.3
        want_hi = A @ c + np.abs(A) @ r + B[:, 0] * 0.3
        assert not nf
        assert np.all(lo <= want_lo + 1e-13) and np.all(hi >= want_hi - 1e-13)
        assert np.allclose(lo, want_lo, rtol=0, atol=1e-12) and np.allclose(hi, want_hi, rtol=0, atol=1e-12)


def test_interval_graph_contains_the_sampled_graph(orc):
    base = W.problem(W.vdp(1.0), [-3, -3], [3, 3], 10, 3, W.controls_grid(-1, 1, 3), 0.1, 10, rule="outer",
                     precision="fp64")
    g = {}
    for enc in ("samples", "interval"):
        s = orc.Solver(dict(base, enclosure=enc))
        s.build_graph()
        g[enc] = s.graph()
    (o1, t1, _, _), (o2, t2, _, _) = g["samples"], g["interval"]
    assert len(o1) == len(o2)
    grew = 0
    for p in range(len(o1) - 1):
        a, b = set(t1[o1[p]:o1[p + 1]].tolist()), set(t2[o2[p]:o2[p + 1]].tolist())
        assert a <= b
        grew += len(b) > len(a)
    assert grew > 0


def test_own_exp_error_bound(orc):
    """The interval mode's e^x (range reduction + Taylor) is within 2^-46 of
    e^x relative (its proven bound; the enclosure widens by 2^-40) over the
    whole domain, at the reduction's switch points and at exact values."""
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    rng = np.random.default_rng(11)
    xs = list(rng.uniform(-700.0, 709.0, 3000)) + list(rng.uniform(-2.0, 2.0, 2000))
    xs += [(k + 0.5) * 0.6931471805599453 for k in range(-1000, 1020, 7)] + [0.0, 1.0, -1.0, 709.0, -700.0]
    worst = 0.0
    for x in xs:
        v = orc.own_exp(x)
        ex = mp.exp(mp.mpf(x))
        worst = max(worst, float(abs((mp.mpf(v) - ex) / ex)))
    assert worst < 2.0 ** -46
    assert orc.own_exp(0.0) == 1.0
    assert orc.own_exp(710.0) == float("inf") and orc.own_exp(-701.0) == 0.0


def test_own_sincos_error_bound(orc):
    """sin / cos of the interval mode: within 2^-46 absolute for |x| <= 65536,
    quadrants and signs included (near multiples of pi/2 and far out), and
    refused beyond."""
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 160
    rng = np.random.default_rng(12)
    xs = list(rng.uniform(-4.0, 4.0, 2000)) + list(rng.uniform(-65536.0, 65536.0, 2000))
    xs += [k * 1.5707963267948966 + d for k in range(-40, 41) for d in (-1e-9, 0.0, 1e-9)]
    worst = 0.0
    for x in xs:
        s, c = orc.own_sincos(x)
        worst = max(worst, float(abs(mp.mpf(s) - mp.sin(mp.mpf(x)))), float(abs(mp.mpf(c) - mp.cos(mp.mpf(x)))))
    assert worst < 2.0 ** -46
    assert orc.own_sincos(0.0) == (0.0, 1.0)
    assert orc.own_sincos(65537.0) is None and orc.own_sincos(float("nan")) is None
