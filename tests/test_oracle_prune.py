"""Pins of the oracle's pruning fixed point (Sec. 2.3, Def. 3-5, Prop. 1):
brute force over all subsets, closed forms of a scalar linear system, the
kept-set invariants, and monotone shrinkage under refinement."""
import itertools
import os

import numpy as np
import pytest

from paper_2202_06111_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def _random_graph(rng, nc, nu, p_edge=0.25, inner_ok=True):
    off = [0]
    tgt, flag = [], []
    for p in range(nc * nu):
        t = sorted(j for j in range(nc) if rng.random() < p_edge)
        f = 0
        if rng.random() < 0.8:
            f |= 1                                  # inside X
        if rng.random() < 0.1:
            f |= 2                                  # touches a removed cell
        if inner_ok and (f & 1) and not t:
            t = [int(rng.integers(nc))]             # an image inside X has a target
        tgt += t
        flag.append(f)
        off.append(len(tgt))
    return np.array(off), np.array(tgt, np.int32), np.array(flag, np.uint8)


def _viable(off, tgt, flag, K, p, rule):
    t = tgt[off[p]:off[p + 1]]
    if rule == "outer":
        return any(K[j] for j in t)
    if not (flag[p] & 1) or (flag[p] & 6):
        return False
    return all(K[j] for j in t)


def _is_post_fixed(off, tgt, flag, nu, K, rule):
    return all(any(_viable(off, tgt, flag, K, i * nu + u, rule) for u in range(nu))
               for i in range(len(K)) if K[i])


@pytest.mark.parametrize("rule", ["inner", "outer"])
@pytest.mark.parametrize("seed", range(12))
def test_prune_is_greatest_fixed_point_bruteforce(orc, rule, seed):
    """The kept set is the union of all subsets closed under the rule (the
    greatest post-fixed point), enumerated over all 2^n subsets."""
    rng = np.random.default_rng(seed)
    nc, nu = int(rng.integers(4, 12)), int(rng.integers(1, 4))
    off, tgt, flag = _random_graph(rng, nc, nu, p_edge=float(rng.uniform(0.1, 0.4)))
    best = np.zeros(nc, bool)
    for bits in range(1 << nc):
        K = np.array([(bits >> i) & 1 for i in range(nc)], bool)
        if _is_post_fixed(off, tgt, flag, nu, K, rule):
            best |= K
    got = orc.prune_graph(nc, nu, off, tgt, flag, rule)
    assert list(got) == list(best)


@pytest.mark.parametrize("seed", range(20))
def test_inner_subset_of_outer(orc, seed):
    rng = np.random.default_rng(100 + seed)
    nc, nu = int(rng.integers(5, 60)), int(rng.integers(1, 5))
    off, tgt, flag = _random_graph(rng, nc, nu, p_edge=0.08)
    ki = orc.prune_graph(nc, nu, off, tgt, flag, "inner")
    ko = orc.prune_graph(nc, nu, off, tgt, flag, "outer")
    assert not np.any(ki & ~ko)


def _scalar(a, b, controls, n0, rule):
    return W.problem(W.linmap([[a]], [[1.0]]), [-1.0], [1.0], n0, 2, [[c] for c in controls],
                     1.0, 0, rule=rule)


@pytest.mark.parametrize("rule", ["inner", "outer"])
@pytest.mark.parametrize("n0", [2, 4, 8, 16, 64])
def test_closed_form_doubling_map_full_controls(orc, rule, n0):
    """x+ = 2x + u, |x| <= 1, u in {-1,-1/2,0,1/2,1}: the largest control
    invariant set is [-1, 1] itself and both rules keep every cell (corner
    samples of a monotone linear map give the exact image)."""
    s = orc.solve(_scalar(2.0, 0.0, [-1, -0.5, 0, 0.5, 1], n0, rule), 0)
    assert s.kept().all()


def test_closed_form_single_cell_inner_keeps_nothing(orc):
    """With one cell the image [-2+u, 2+u] never fits in X: INNER keeps nothing,
    OUTER keeps the cell (its image still meets it)."""
    assert not orc.solve(_scalar(2.0, 0.0, [-1, -0.5, 0, 0.5, 1], 1, "inner"), 0).kept().any()
    assert orc.solve(_scalar(2.0, 0.0, [-1, -0.5, 0, 0.5, 1], 1, "outer"), 0).kept().all()


@pytest.mark.parametrize("rule", ["inner", "outer"])
def test_closed_form_no_invariant_set(orc, rule):
    """x+ = 2x + 3 (u = 0): the only fixed point x = -3 lies outside X, every
    trajectory leaves [-1, 1]: nothing is kept."""
    p = W.problem(W.linmap([[2.0]], [[1.0]]), [-1.0], [1.0], 16, 2, [[3.0]], 1.0, 0, rule=rule)
    assert not orc.solve(p, 0).kept().any()


@pytest.mark.parametrize("n0", [8, 16, 32, 64, 128])
def test_closed_form_half_controls_sandwich(orc, n0):
    """x+ = 2x + u with u in {-1/2, 0, 1/2}: the largest control invariant set is
    [-1/2, 1/2]. With exact images INNER's cells form an invariant set inside it
    and OUTER's cells cover it (Prop. 1(iii)): INNER <= [-1/2,1/2] <= OUTER."""
    w = 2.0 / n0
    for rule in ("inner", "outer"):
        s = orc.solve(_scalar(2.0, 0.0, [-0.5, 0.0, 0.5], n0, rule), 0)
        lv, idx = s.kept_cells()
        lo = -1.0 + idx[:, 0] * w
        hi = lo + w
        if rule == "inner":
            assert len(lo) == 0 or (lo.min() >= -0.5 and hi.max() <= 0.5)
        else:
            covered = sorted(zip(lo, hi))
            assert covered[0][0] <= -0.5 and covered[-1][1] >= 0.5
            assert all(b[0] <= a[1] for a, b in zip(covered, covered[1:]))   # no gap


def test_closed_form_golden(orc):
    """Exact kept intervals of the doubling map derived by hand in
    tests/golden/closed_form_doubling.txt (INNER [-1/2+w, 1/2-w], OUTER
    [-1/2-2w, 1/2+2w]): pins the closed-touch rule to the cell."""
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "closed_form_doubling.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 10
    for rule, n0, lo_want, hi_want in rows:
        n0 = int(n0)
        w = 2.0 / n0
        s = orc.solve(_scalar(2.0, 0.0, [-0.5, 0.0, 0.5], n0, rule), 0)
        lv, idx = s.kept_cells()
        if lo_want == "empty":
            assert len(idx) == 0
            continue
        cells = sorted(idx[:, 0].tolist())
        assert cells == list(range(cells[0], cells[-1] + 1))        # one interval
        assert (-1.0 + cells[0] * w, -1.0 + (cells[-1] + 1) * w) == (float(lo_want), float(hi_want))


def _check_fixed_point(s, rule):
    """K = Phi(K): kept cells have a viable control, removed cells have none."""
    off, tgt, flag, _ = s.graph()
    K = s.kept()
    nu = s.n_u
    for i in range(len(K)):
        v = any(_viable(off, tgt, flag, K, i * nu + u, rule) for u in range(nu))
        assert v == bool(K[i])


@pytest.mark.parametrize("rule", ["inner", "outer"])
def test_invariants_after_solve(orc, rule):
    """The INNER invariant: every kept cell has a control whose image
    lies in X and whose image cells are all kept; for OUTER every kept cell has
    an edge to a kept cell; and the kept set is a fixed point at every level."""
    prob = dict(W.cstr_256(levels=2, n0=24), rule=rule)
    s = orc.Solver(prob)
    for L in range(3):
        s.build_graph()
        s.prune()
        _check_fixed_point(s, rule)
        if L < 2:
            s.subdivide()


def _kept_volume_mask(s, prob, fine):
    """Kept union rasterised on the finest grid (exact: cells are dyadic unions)."""
    n0 = prob["n0"][0]
    N = n0 << fine
    mask = np.zeros((N, N), bool)
    lv, idx = s.kept_cells()
    for L, (i, j) in zip(lv, idx):
        f = 1 << (fine - L)
        mask[i * f:(i + 1) * f, j * f:(j + 1) * f] = True
    return mask


@pytest.mark.parametrize("rule", ["inner", "outer"])
def test_monotone_shrinkage(orc, rule):
    """Refinement never grows the kept union (Sec. 2.1: subdivision keeps the union,
    removed cells stay removed) and never loses covered volume by splitting alone."""
    prob = dict(W.vdp_64(n0=16), rule=rule)
    s = orc.Solver(prob)
    prev = None
    for L in range(4):
        s.build_graph()
        s.prune()
        m = _kept_volume_mask(s, prob, 3)
        if prev is not None:
            assert not np.any(m & ~prev)
        prev = m
        if L < 3:
            s.subdivide()
